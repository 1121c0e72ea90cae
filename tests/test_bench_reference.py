"""The bench's reference arm (the CPU oracle on a bounded sample of the workload) on the host:
one JSON line with the contract's keys, the oracle described as its CPU baseline, and an
end-to-end block without host-device copies.  Small degree so that it runs in seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--L", "63",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in rec, k
    assert rec["impl"] == "reference" and rec["steps"] == 2 and rec["warmup"] == 1
    assert rec["unit"] == "fields/s" and rec["value"] > 0 and rec["higher_is_better"] is True
    assert rec["config"]["L"] == 63 and "workload" in rec["config"]
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"] and cb["sample"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_cpu_baseline_block():
    """The GPU arm's cpu_baseline object (all cores, one thread, the small configurations),
    built on the host alone."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.cpu_baseline(argparse.Namespace(L=31))
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1 and "L=31" in cb["sample"]
    assert cb["single_thread"]["cores"] == 1 and cb["single_thread"]["value"] > 0
    sc = cb["small_configs"]
    for k in ("L16", "L511"):
        assert sc[k]["separable_fields_per_s"] > 0 and sc[k]["direct_fields_per_s"] > 0
    # O(L^3) against O(N L^2): at L = 511 the separable form is far ahead whatever the noise;
    # at L = 16 both take well under a millisecond and their order is noise
    assert sc["L511"]["separable_fields_per_s"] > sc["L511"]["direct_fields_per_s"]


def test_reference_arm_under_torchrun_two_ranks():
    """Launched like the multi-GPU driver runs (torchrun, 2 ranks): rank 0 alone prints the
    line, the other rank exits 0 without work."""
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", "29531", os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--L", "31", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
