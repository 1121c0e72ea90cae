"""The bench's JSON line on the GPU: a small main workload with every form and the end-to-end
measurement, checked for the keys of the measurement contract (value, roofline, e2e, launches,
clocks, forms).  Guards the bench script itself against breaking."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_bench_json_line_small_workload():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--L", "255", "--batch", "8",
                          "--steps", "3", "--warmup", "3", "--no-cpu-baseline"], cwd=ROOT, capture_output=True,
                         text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "kernels", "e2e", "gpu_launches",
              "clocks", "errors", "forms"):
        assert k in rec, k
    assert rec["value"] > 0 and rec["steps"] == 3 and rec["warmup"] >= 3
    assert rec["gpu_launches"] > 0 and "workload" in rec["config"]
    rl = rec["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rl, k
    e2e = rec["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in rec["clocks"] and "reasons" in rec["clocks"]
    assert rec["errors"]["fwd_vs_fp64_max_rel"] < 1e-6
    assert rec["errors"]["vs_oracle_max_rel"] < 1e-6
    # one generator pass per step: adjoint, forward, 7 other kernels
    assert rec["gpu_launches"] == rec["steps"] * 8
    for form in ("fp64_same_workload", "fp64_L16_one_field", "fp64_L511_one_field", "ragged_batch",
                 "real_fields_B8", "field_a_tables", "cg_route_L511_one_field", "fp64_real_vs_complex_L511_B8",
                 "split_L1000_B8", "cg_stability_ratios", "table3_degrees"):
        assert form in rec["forms"], form
    for L in (250, 500, 750, 1000, 1250, 1500, 1750, 2000, 2250):
        row = rec["forms"]["table3_degrees"]["L%d" % L]
        assert row["split_batch"]["roundtrip_max_rel"] < 1e-6 and row["fp64_one_field"]["roundtrip_max_rel"] < 1e-12
    assert rec["forms"]["split_L1000_B8"]["generator_shape"][2] in (1, 2)
    st = rec["forms"]["cg_stability_ratios"]["series"]["L10_N100000"]
    assert 0 < st["r_hat"] <= 0.7072 and 0 < st["r_tilde"] <= 0.7072 and st["kappa_tilde"] <= 2.4495
