#!/usr/bin/env python3
"""Benchmark: forward + adjoint vector spherical harmonic transform throughput.

Workload (the precision form): L = 1023 on the 1024 x 2048 Gauss-Legendre grid, a
batch of 32 fields, coefficients with complex parts i.i.d. N(0,1)*(l+1)^-1.5 (seed 2),
tangent components complex64.  One step = AdjVSHT of the batch (coefficients -> grid)
followed by FwdVSHT of the synthesised fields (grid -> coefficients); the metric is
fields / (t_adj + t_fwd).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x6|fp64]
  python bench.py --impl reference ...     (the CPU oracle, timed on a bounded sample)

Under torchrun (N > 1) every rank runs the same batch on its own GPU (replicas, weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adj VSHT fields/s at L=1023 (split-prec vs FP64), max rel err vs FP64 oracle"
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default=None, choices=["bf16x6", "fp64"])
    ap.add_argument("--L", type=int, default=1023)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default generator shape (profiling runs: no tuner launches)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP64 / small-degree / ragged-batch form measurements")
    ap.add_argument("--no-share", action="store_true",
                    help="regenerate the Legendre operand in both calls of a step "
                         "(no FAVEST_FLAG_SHARE_LAMBDA)")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle comparison of one field (about 10-30 s of host time)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# per-kernel roofline
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1700.0, "fallback"


def ncu_traffic(kernel, L, B):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled to this
    workload; None when there is none or the kernel's source changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        rec = d[kernel]
        src = os.path.join(ROOT, "paper_1908_00041_gb300", "csrc", rec["source"])
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["sha256"]:
                return None
        if rec["L"] != L:
            return None
        return rec["dram_bytes_per_launch"] * B / rec["batch"]
    except Exception:
        return None


def alu_peaks():
    """FP64 and FP32 FMA peaks (TFLOP/s) from unit counts and the maximum SM clock: 152 SMs x
    2 FP64 FMA per clock (NVIDIA's 1.25 TFLOP/s FP64 figure for GB300 at 2.07 GHz: 1.25e12 /
    (2 x 152 x 2.07e9) = 1.99) and 128 FP32 FMA per clock per SM, an FMA counted as 2."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return sms * 2 * 2 * mhz * 1e6 / 1e12, sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


def kernel_rooflines(plan, prof, fp64_probe, fp32_probe, L, B):
    hbm, bf16, src = measured_peaks()
    f64, f32, sms, mhz = alu_peaks()
    units = {0: ("hbm", "GB/s", hbm, "HBM copy bandwidth, MEASURED_PEAKS.json (%s)" % src),
             1: ("alu", "TFLOP/s", f64, "FP64 FMA peak from unit counts: %d SMs x 2 FMA/clk x 2 flop x %.0f MHz "
                                        "(derived; probe-measured FMA stream %.3f)" % (sms, mhz, fp64_probe)),
             2: ("tensor", "TFLOP/s", bf16, "bf16 dense sustained, MEASURED_PEAKS.json (%s)" % src),
             3: ("alu", "TFLOP/s", f32, "FP32 FMA peak from unit counts: %d SMs x 128 FMA/clk x 2 flop x %.0f MHz "
                                        "(derived; probe-measured FMA stream %.2f)" % (sms, mhz, fp32_probe))}
    probes = {1: fp64_probe, 3: fp32_probe}
    total = sum(v[0] for v in prof.values())
    kernels = {}
    for name, (tot_ms, n) in prof.items():
        nbytes, flops, pipe = plan.kernel_work(name)
        t = tot_ms / n * 1e-3
        bound, unit, peak, psrc = units[pipe]
        achieved = nbytes / t / 1e9 if pipe == 0 else flops / t / 1e12
        kernels[name] = {"ms_per_launch": tot_ms / n, "launches": n, "share": tot_ms / total,
                         "bound": bound, "pipe": ["hbm", "fp64", "tensor", "fp32"][pipe],
                         "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                         "algorithmic_bytes": nbytes, "algorithmic_flops": flops,
                         "hbm_frac": nbytes / t / 1e9 / hbm}
        if pipe in probes:
            kernels[name]["frac_of_probe"] = achieved / probes[pipe]
    top = max(kernels, key=lambda k: kernels[k]["share"])
    k = kernels[top]
    roofline = {"kernel": top, "bound": k["bound"], "achieved": k["achieved"], "peak": k["peak"],
                "unit": k["unit"], "frac": k["frac"], "traffic": ncu_traffic(top, L, B),
                "peak_source": units[{"hbm": 0, "fp64": 1, "tensor": 2, "fp32": 3}[k["pipe"]]][3],
                "ms_per_launch": k["ms_per_launch"],
                "algorithmic_bytes_per_launch": k["algorithmic_bytes"],
                "algorithmic_flops_per_launch": k["algorithmic_flops"]}
    return kernels, roofline


# ---------------------------------------------------------------------------
# the other forms: FP64 path at the same workload, the two FP64 configurations, the
# ragged batch (each a few CUDA-event-timed steps after warm-up)
# ---------------------------------------------------------------------------
def max_over_ranks(value, dist, device):
    """The largest of the ranks' values (replicas: the job takes as long as its slowest
    rank); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each processed units_per_rank units
    in at most `seconds`."""
    return world * units_per_rank / seconds


def time_steps(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_split_other_length(L, B, stream):
    """The split path at a degree whose longitude count is not a power of two (L = 1000:
    n_phi = 2002 = 2*7*11*13, the paper's nearest timing row), B complex64 fields, a few
    CUDA-event-timed steps after warm-up (adjoint + forward sharing one generator pass, as in
    the headline step); per-kernel times from the plan's own events."""
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    p = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    shape = p.tune()
    a, b = synthetic.coefficients(L, B, seed=5, decay=1.5)
    a = torch.as_tensor(a).to(torch.complex64).cuda()
    b = torch.as_tensor(b).to(torch.complex64).cuda()
    tt = torch.empty(p.field_shape(), dtype=torch.complex64, device="cuda")
    tp = torch.empty_like(tt)
    a2 = torch.empty_like(a)
    b2 = torch.empty_like(b)

    def st():
        p.adj(a, b, tt, tp, stream=stream, share_lambda=True)
        p.fwd(tt, tp, a2, b2, stream=stream, share_lambda=True)
    ms = time_steps(st, 5, 3, stream)
    p.profile(True)
    time_steps(st, 2, 0, stream)
    prof = p.profile_read()
    p.profile(False)
    err = max(float((a2 - a).abs().max() / a.abs().max()), float((b2 - b).abs().max() / b.abs().max()))
    shape = list(shape) + [p.gen_chains()]
    p.close()
    return {"value": B / (ms * 1e-3), "unit": "fields/s", "ms_per_step": ms, "L": L, "nphi": 2 * (L + 1),
            "generator_shape": shape, "roundtrip_max_rel": err,
            "kernel_ms": {k: v[0] / v[1] for k, v in prof.items()}}


# Table 3 of the paper (one field, CPU with MATLAB + NFFT): seconds per FwdVSHT and AdjVSHT
PAPER_TABLE3 = {250: (0.40, 0.83), 500: (1.81, 3.87), 750: (4.22, 9.52), 1000: (7.2903, 17.89),
                1250: (15.16, 33.97), 1500: (22.30, 50.32), 1750: (32.87, 73.94), 2000: (41.51, 97.32),
                2250: (62.74, 144.70)}


def measure_table3(stream, batch=32):
    """The paper's timing degrees (Table 3: L = 250 .. 2250; nphi = 2(L+1) with prime factors
    151..2251 above 128 for most of them, taken by the Bluestein stage of the FP32 DFT).  Per
    degree: the split path on one field (adjoint and forward each with its own generator
    pass, like the paper's per-transform times), the split path's throughput on `batch`
    fields (adjoint + forward sharing one generator pass), and the FP64 path on one field;
    roundtrip errors of the batch; the paper's CPU seconds beside them for context."""
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    out = {}
    for L in sorted(PAPER_TABLE3):
        row = {"nphi": 2 * (L + 1), "paper_cpu_s": {"fwd": PAPER_TABLE3[L][0], "adj": PAPER_TABLE3[L][1]}}
        for B, key in ((1, "split_one_field"), (batch, "split_batch")):
            p = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
            p.tune()
            a, b = synthetic.coefficients(L, B, seed=7, decay=1.5)
            a = torch.as_tensor(a).to(torch.complex64).cuda()
            b = torch.as_tensor(b).to(torch.complex64).cuda()
            tt = torch.empty(p.field_shape(), dtype=torch.complex64, device="cuda")
            tp = torch.empty_like(tt)
            a2 = torch.empty_like(a)
            b2 = torch.empty_like(b)
            if B == 1:
                adj_ms = time_steps(lambda: p.adj(a, b, tt, tp, stream=stream), 5, 2, stream)
                fwd_ms = time_steps(lambda: p.fwd(tt, tp, a2, b2, stream=stream), 5, 2, stream)
                row[key] = {"adj_ms": adj_ms, "fwd_ms": fwd_ms}
            else:
                def st():
                    p.adj(a, b, tt, tp, stream=stream, share_lambda=True)
                    p.fwd(tt, tp, a2, b2, stream=stream, share_lambda=True)
                ms = time_steps(st, 5, 2, stream)
                err = max(float((a2 - a).abs().max() / a.abs().max()), float((b2 - b).abs().max() / b.abs().max()))
                row[key] = {"fields": B, "ms_per_step": ms, "fields_per_s": B / (ms * 1e-3), "roundtrip_max_rel": err}
            p.close()
            del a, b, tt, tp, a2, b2
            torch.cuda.empty_cache()
        p64 = api.Plan(L, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
        a, b = synthetic.coefficients(L, 1, seed=7)
        a = torch.as_tensor(a).cuda()
        b = torch.as_tensor(b).cuda()
        tt = torch.empty(p64.field_shape(), dtype=torch.complex128, device="cuda")
        tp = torch.empty_like(tt)
        a2 = torch.empty_like(a)
        b2 = torch.empty_like(b)
        adj_ms = time_steps(lambda: p64.adj(a, b, tt, tp, stream=stream), 2, 1, stream)
        fwd_ms = time_steps(lambda: p64.fwd(tt, tp, a2, b2, stream=stream), 2, 1, stream)
        err = max(float((a2 - a).abs().max() / a.abs().max()), float((b2 - b).abs().max() / b.abs().max()))
        row["fp64_one_field"] = {"adj_ms": adj_ms, "fwd_ms": fwd_ms, "roundtrip_max_rel": err}
        p64.close()
        out["L%d" % L] = row
    return out


def measure_forms(L, B, a, b, split_value, fp64_peak):
    import numpy as np
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    stream = torch.cuda.current_stream()
    forms = {}
    # FP64 path, same workload (complex64 fields in and out)
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C64)
    tt = torch.empty(p64.field_shape(), dtype=torch.complex64, device="cuda")
    tp = torch.empty_like(tt)
    a2 = torch.empty_like(a)
    b2 = torch.empty_like(b)

    def st64():
        p64.adj(a, b, tt, tp, stream=stream)
        p64.fwd(tt, tp, a2, b2, stream=stream)
    p64.profile(True)
    ms = time_steps(st64, 2, 1, stream)
    prof = p64.profile_read()
    p64.profile(False)
    kern = {}
    for name, (tot, n) in prof.items():
        nb, fl, pipe = p64.kernel_work(name)
        t = tot / n * 1e-3
        kern[name] = {"ms_per_launch": tot / n, "fp64_frac": (fl / t / 1e12 / fp64_peak) if pipe == 1 else None}
    v64 = B / (ms * 1e-3)
    forms["fp64_same_workload"] = {"value": v64, "unit": "fields/s", "ms_per_step": ms, "kernels": kern}
    forms["split_speedup_over_fp64"] = split_value / v64
    p64.close()
    del tt, tp, a2, b2
    # C1: FP64, L = 16, one field (complex128)
    for name, Lc, seed in (("fp64_L16_one_field", 16, 0), ("fp64_L511_one_field", 511, 1)):
        ca, cb = synthetic.coefficients(Lc, 1, seed=seed, decay=1.0)
        pc = api.Plan(Lc, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
        da = torch.as_tensor(ca).cuda()
        db = torch.as_tensor(cb).cuda()
        xt = torch.empty(pc.field_shape(), dtype=torch.complex128, device="cuda")
        xp = torch.empty_like(xt)
        ra = torch.empty_like(da)
        rb = torch.empty_like(db)
        nst = 200 if Lc == 16 else 5
        t_adj = time_steps(lambda: pc.adj(da, db, xt, xp, stream=stream), nst, 3, stream)
        t_fwd = time_steps(lambda: pc.fwd(xt, xp, ra, rb, stream=stream), nst, 3, stream)
        torch.cuda.synchronize()
        rt = float(np.max(np.abs(ra.cpu().numpy() - ca)) / np.max(np.abs(ca)))
        forms[name] = {"adj_ms": t_adj, "fwd_ms": t_fwd, "fields_per_s": 1.0 / ((t_adj + t_fwd) * 1e-3),
                       "roundtrip_max_rel": rt}
        pc.close()
    # ragged batch: 256 fields, L uniform over {31, 63, 127, 255, 511} (seed 3), (l+1)^-1
    Ls, rng = synthetic.ragged_degrees(256, [31, 63, 127, 255, 511], seed=3)
    Ls = [int(x) for x in Ls]
    bp = api.BatchPlan(Ls, api.FAVEST_BF16X6, api.FAVEST_IO_C64, autotune=True, graph=True)
    ga = torch.zeros(bp.coef_elems, dtype=torch.complex64, device="cuda")
    gb = torch.zeros_like(ga)
    for i, Lr in enumerate(Ls):
        ca, cb = synthetic.coefficients(Lr, 1, seed=None, decay=1.0, rng=rng)
        bp.coef(ga, i).copy_(torch.as_tensor(ca[0]).to(torch.complex64))
        bp.coef(gb, i).copy_(torch.as_tensor(cb[0]).to(torch.complex64))
    gt = torch.empty(bp.field_elems, dtype=torch.complex64, device="cuda")
    gp = torch.empty_like(gt)
    fa = torch.empty_like(ga)
    fb = torch.empty_like(gb)

    def stb():
        bp.adj(ga, gb, gt, gp, stream=stream)
        bp.fwd(gt, gp, fa, fb, stream=stream)
    ms = time_steps(stb, 10, 3, stream)     # warm-up includes the eager run and the capture
    assert bp.status() == 0
    forms["ragged_batch"] = {"value": len(Ls) / (ms * 1e-3), "unit": "fields/s", "ms_per_step": ms,
                             "fields": len(Ls), "graph": True, "groups": bp.groups(),
                             "launches_per_step": None}
    forms["ragged_batch"].update(ragged_bounds(bp.groups(), stream))
    bp.close()
    del ga, gb, gt, gp, fa, fb
    # real fields (half-spectrum coefficients), L as the main workload, 32 and 64 fields
    for Br in (B, 2 * B):
        forms["real_fields_B%d" % Br] = measure_real(L, Br, stream)
    forms["field_a_tables"] = measure_field_a()
    forms["cg_stability_ratios"] = measure_stability()
    forms["cg_route_L511_one_field"] = measure_cg_route(511, stream)
    forms["fp64_real_vs_complex_L511_B8"] = measure_fp64_real(511, 8, stream)
    forms["split_L1000_B%d" % B] = measure_split_other_length(1000, B, stream)
    forms["table3_degrees"] = measure_table3(stream, B)
    forms["scatter_L127_N32768_B2"] = measure_scatter(127, 32768, 2, stream)
    return forms


def measure_scatter(L, npts, B, stream):
    """Transforms at arbitrary points (Sec. 4.4's FaVeST_fwd(T, L, X, w) / FaVeST_adj(a, b, X)):
    npts area-uniform random points (z ~ U[-1, 1], phi ~ U[0, 2 pi), seed 4), unit weights,
    B fields of Cartesian components; CUDA-event times of the forward and the adjoint, the
    rate in point x coefficient pairs per second (both families), and the adjoint identity
    <A c, T> = <c, A^H T> of the measured pair as a check."""
    import numpy as np
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    rng = np.random.default_rng(4)
    z = rng.uniform(-1.0, 1.0, npts)
    ph = rng.uniform(0.0, 2.0 * np.pi, npts)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    X = np.stack([r * np.cos(ph), r * np.sin(ph), z], -1)
    p = api.ScatterPlan(L, X, None, batch=B)
    a, b = synthetic.coefficients(L, B, seed=6)
    a = torch.as_tensor(a).cuda()
    b = torch.as_tensor(b).cuda()
    T = torch.as_tensor(rng.standard_normal((B, npts, 3)) + 1j * rng.standard_normal((B, npts, 3))).cuda()
    ga = torch.empty_like(a)
    gb = torch.empty_like(b)
    gT = torch.empty_like(T)
    fwd_ms = time_steps(lambda: p.fwd(T, ga, gb, stream=stream), 5, 2, stream)
    adj_ms = time_steps(lambda: p.adj(a, b, gT, stream=stream), 5, 2, stream)
    lhs = torch.vdot(gT.ravel(), T.ravel())
    rhs = torch.vdot(a.ravel(), ga.ravel()) + torch.vdot(b.ravel(), gb.ravel())
    pairs = 2.0 * B * npts * (L * L + 2 * L)
    p.close()
    return {"L": L, "points": npts, "fields": B, "fwd_ms": fwd_ms, "adj_ms": adj_ms,
            "fwd_pairs_per_s": pairs / (fwd_ms * 1e-3), "adj_pairs_per_s": pairs / (adj_ms * 1e-3),
            "adjoint_identity_rel": float(abs(lhs - rhs) / abs(rhs)), "points_recipe":
            "area-uniform random, numpy default_rng(4), unit weights"}


def ragged_bounds(groups, stream):
    """Where a single persistent launch could take the ragged batch: each degree group as a
    plan of its own, run alone (adj + fwd, tuned generator, every kernel on the whole GPU) one
    after another, and a lower bound for ANY schedule of the same kernels: each launch at its
    roofline (favest_kernel_work's algorithmic bytes at the measured HBM bandwidth, or its
    flops at the derived FP64 / FP32 peak), summed over the groups."""
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    hbm, _, _ = measured_peaks()
    f64, f32, _, _ = alu_peaks()
    seq_ms, lb_ms, per = 0.0, 0.0, []
    for g in groups:
        Lg, ng = g["L"], g["fields"]
        pg = api.Plan(Lg, ng, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
        pg.tune()
        ca, cb = synthetic.coefficients(Lg, ng, seed=Lg, decay=1.0)
        da = torch.as_tensor(ca).to(torch.complex64).cuda()
        db = torch.as_tensor(cb).to(torch.complex64).cuda()
        tt = torch.empty(pg.field_shape(), dtype=torch.complex64, device="cuda")
        tp = torch.empty_like(tt)
        ra = torch.empty_like(da)
        rb = torch.empty_like(db)

        def st():
            pg.adj(da, db, tt, tp, stream=stream)
            pg.fwd(tt, tp, ra, rb, stream=stream)
        t = time_steps(st, 10, 3, stream)
        pg.profile(True)
        pg.profile_read()
        st()
        prof = pg.profile_read()
        pg.profile(False)
        lb = 0.0
        for name, (_, n) in prof.items():
            nb, fl, pipe = pg.kernel_work(name)
            rate = {1: f64 * 1e12, 3: f32 * 1e12}.get(pipe)
            lb += n * max(nb / (hbm * 1e9), fl / rate if rate else 0.0) * 1e3
        seq_ms += t
        lb_ms += lb
        per.append({"L": Lg, "fields": ng, "alone_ms": t, "roofline_ms": lb})
        pg.close()
    return {"groups_one_after_another_ms": seq_ms, "every_kernel_at_roofline_ms": lb_ms, "per_group": per}


def measure_fp64_real(L, B, stream):
    """The FP64 path on B real fields (FAVEST_IO_R64, half-spectrum coefficients) against
    the same fields as complex ones (FAVEST_IO_C128): fields/s of adj + fwd steps."""
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    out = {}
    for name, io in (("real", api.FAVEST_IO_R64), ("complex", api.FAVEST_IO_C128)):
        p = api.Plan(L, B, api.FAVEST_FP64, io)
        if p.real:
            ha, hb = synthetic.half_coefficients(L, B, seed=1, decay=1.0)
        else:
            ha, hb = synthetic.coefficients(L, B, seed=1, decay=1.0)
        a = torch.as_tensor(ha).cuda()
        b = torch.as_tensor(hb).cuda()
        tt = torch.empty(p.field_shape(), dtype=p.fdtype, device="cuda")
        tp = torch.empty_like(tt)
        ra, rb = torch.empty_like(a), torch.empty_like(b)

        def step():
            p.adj(a, b, tt, tp, stream=stream)
            p.fwd(tt, tp, ra, rb, stream=stream)
        ms = time_steps(step, 5, 2, stream)
        err = float(max((ra - a).abs().max() / a.abs().max(), (rb - b).abs().max() / b.abs().max()))
        out[name] = {"fields_per_s": B / (ms * 1e-3), "ms_per_step": ms, "roundtrip_max_rel": err}
        p.close()
    out["real_speedup"] = out["real"]["fields_per_s"] / out["complex"]["fields_per_s"]
    return out


def measure_cg_route(L, stream):
    """The paper's Clebsch-Gordan route (Thm. 1, Thm. 2) on the FP64 path: one field of
    degree L from Cartesian components, forward and adjoint timed separately; checked
    against the theta/phi FP64 path on the same field (same coefficients, and the same
    field in Cartesian components)."""
    import numpy as np
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    ca, cb = synthetic.coefficients(L, 1, seed=1, decay=1.0)
    da, db = torch.as_tensor(ca).cuda(), torch.as_tensor(cb).cuda()
    p64 = api.Plan(L, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    cp = api.CgPlan(L, 1)
    tt, tp = p64.adj(da, db)
    x, _ = api.favest_gl_grid(L + 1)
    th = torch.as_tensor(np.arccos(x)).cuda()[:, None]
    ph = torch.as_tensor(2 * np.pi * np.arange(2 * (L + 1)) / (2 * (L + 1))).cuda()[None, :]
    ct, st, cph, sph = torch.cos(th), torch.sin(th), torch.cos(ph), torch.sin(ph)
    T = torch.stack([tt[0] * ct * cph - tp[0] * sph, tt[0] * ct * sph + tp[0] * cph,
                     -tt[0] * st.expand_as(tt[0])])[None].contiguous()
    a, b = cp.fwd(T)
    Tr = torch.empty_like(T)
    t_fwd = time_steps(lambda: cp.fwd(T, a, b, stream=stream), 5, 2, stream)
    t_adj = time_steps(lambda: cp.adj(da, db, Tr, stream=stream), 5, 2, stream)
    cp.profile(True)
    cp.fwd(T, a, b, stream=stream)
    cp.adj(da, db, Tr, stream=stream)
    prof = {k: v[0] / v[1] for k, v in cp.profile_read().items()}
    cp.profile(False)
    torch.cuda.synchronize()

    def nerr(g, r):
        return float((g - r).abs().max() / r.abs().max())
    out = {"fwd_ms": t_fwd, "adj_ms": t_adj, "fields_per_s": 1.0 / ((t_fwd + t_adj) * 1e-3),
           "fwd_vs_synthesising_coefficients": max(nerr(a, da), nerr(b, db)),
           "adj_vs_theta_phi_path": nerr(Tr, T), "kernel_ms": prof,
           "input": "coefficients N(0,1)(l+1)^-1, seed 1; T = the theta/phi FP64 adjoint in Cartesian components"}
    cp.close()
    p64.close()
    return out


def measure_stability():
    """Stability ratios of the forward CG route (Sec. 5.5, eq. r_stable) at L = 5 and 10 for
    N from 100 to 100,000 points, the ranges of the paper's stability figures.  Area-uniform
    random points (cos(theta) uniform, seed 2019) stand in for the paper's spherical designs;
    the ratios depend on the colatitude only.  Timed through the C-ABI call from host
    arrays (copy, three kernels, read-back) at L = 10, N = 100,000."""
    import numpy as np
    from paper_1908_00041_gb300 import api
    out = {"points": "cos(theta) uniform on (-1, 1), numpy default_rng(2019)", "series": {}}
    for L, Ns in ((5, (100, 1000, 10000)), (10, (100, 1000, 10000, 100000))):
        for N in Ns:
            z = np.random.default_rng(2019).uniform(-1.0, 1.0, N)
            r = api.favest_cg_stability(L, z)
            out["series"]["L%d_N%d" % (L, N)] = {"r_hat": r[0], "kappa_hat": r[1], "r_tilde": r[2],
                                                 "kappa_tilde": r[3], "r_hat_over_N": r[0] / N,
                                                 "r_tilde_over_N": r[2] / N}
    z = np.random.default_rng(2019).uniform(-1.0, 1.0, 100000)
    api.favest_cg_stability(10, z)
    reps = 10
    t0 = time.perf_counter()
    for _ in range(reps):
        api.favest_cg_stability(10, z)
    ms = (time.perf_counter() - t0) * 1e3 / reps
    out["L10_N100000_ms_per_call"] = ms
    out["L10_N100000_point_coefficients_per_s"] = 100000 * 120 / (ms * 1e-3)
    return out


def measure_field_a():
    """Tangent Field A (Sec. 5.2), the paper's GL-row experiments on the FP64 path:
    Table 1 (relative L2 error of AdjVSHT(FwdVSHT(T)), L = 10..150) and Table 2 (repeated
    transforms at L = 40).  T0 is synthesised by the FP64 path from the field's exact
    coefficients (tests/golden/field_a.txt, which also holds the paper's values; the GPU
    test samples T0 with the oracle instead)."""
    import numpy as np
    import torch
    from paper_1908_00041_gb300 import api
    coefs, t1, t2 = [], {}, None
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "field_a.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] in ("a", "b"):
            coefs.append((line[0], int(line[1]), int(line[2]), float(line[3]) + 1j * float(line[4])))
        elif line[0] == "table1":
            t1[int(line[1])] = float(line[2])
        elif line[0] == "table2":
            t2 = [float(v) for v in line[2:]]

    def exact(L):
        a = torch.zeros((1, L * L + 2 * L), dtype=torch.complex128, device="cuda")
        b = torch.zeros_like(a)
        for fam, l, m, v in coefs:
            (a if fam == "a" else b)[0, l * l + l + m - 1] = v
        return a, b
    out = {"T0": "synthesised from the exact coefficients by the FP64 path", "table1_gl": {}}
    for L in sorted(t1):
        p = api.Plan(L, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
        x, W = api.favest_gl_grid(L + 1)
        w = torch.as_tensor(np.repeat(W, 2 * (L + 1)) * (np.pi / (L + 1))).cuda()
        tt, tp = p.adj(*exact(L))
        rt, rp = p.adj(*p.fwd(tt, tp))
        num = (w * ((rt - tt).abs() ** 2 + (rp - tp).abs() ** 2).reshape(-1)).sum()
        den = (w * (tt.abs() ** 2 + tp.abs() ** 2).reshape(-1)).sum()
        out["table1_gl"][str(L)] = {"fp64": float(torch.sqrt(num / den)), "paper": t1[L]}
        p.close()
    p = api.Plan(40, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    T0 = p.adj(*exact(40))
    c0 = p.fwd(*T0)
    T1 = p.adj(*c0)
    c1 = p.fwd(*T1)
    T2 = p.adj(*c1)

    def sup(u, v):
        return max(float((u[0] - v[0]).abs().max()), float((u[1] - v[1]).abs().max()))
    out["table2_gl_L40"] = {"fp64": [sup(T1, T0), sup(T2, T0), sup(T2, T1), sup(c1, c0)], "paper": t2,
                            "columns": ["|T1-T0|inf", "|T2-T0|inf", "|T2-T1|inf", "max coefficient difference"]}
    p.close()
    return out


def measure_real(L, B, stream):
    """Split form on real fields: B fields, coefficients m >= 0 drawn as for the main
    workload ((l+1)^-1.5, seed 2, m = 0 entries real), adj + fwd per step sharing one
    generator pass; errors of two
    sampled fields against the FP64 complex path on the Hermitian-extended input."""
    import numpy as np
    import torch
    from paper_1908_00041_gb300 import api, synthetic
    ha, hb = synthetic.half_coefficients(L, B, seed=2, decay=1.5)
    pr = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    pr.tune()
    da = torch.as_tensor(ha).to(torch.complex64).cuda()
    db = torch.as_tensor(hb).to(torch.complex64).cuda()
    tt = torch.empty(pr.field_shape(), dtype=torch.float32, device="cuda")
    tp = torch.empty_like(tt)
    ra = torch.empty_like(da)
    rb = torch.empty_like(db)

    def step():
        pr.adj(da, db, tt, tp, stream=stream, share_lambda=True)
        pr.fwd(tt, tp, ra, rb, stream=stream, share_lambda=True)
    ms = time_steps(step, 10, 3, stream)
    pr.profile(True)
    time_steps(step, 3, 0, stream)
    prof = {k: v[0] / v[1] for k, v in pr.profile_read().items()}
    pr.profile(False)
    assert pr.status() == 0
    # accuracy: sampled fields against the FP64 complex path
    pick = [0, B - 1]
    ls = np.concatenate([np.full(l + 1, l) for l in range(1, L + 1)])
    ms_ = np.concatenate([np.arange(l + 1) for l in range(1, L + 1)])
    full = ls * ls + ls + ms_ - 1
    neg = ls * ls + ls - ms_ - 1
    sg = np.where(ms_ % 2 == 1, -1.0, 1.0)

    def extend(h):
        out = np.zeros(h.shape[:-1] + (L * L + 2 * L,), np.complex128)
        out[..., full] = h
        out[..., neg[ms_ > 0]] = (sg * np.conj(h))[..., ms_ > 0]
        return out
    p64 = api.Plan(L, len(pick), api.FAVEST_FP64, api.FAVEST_IO_C128)
    h32a = da.cpu().numpy()[pick].astype(np.complex128)
    h32b = db.cpu().numpy()[pick].astype(np.complex128)
    ct, cp = p64.adj(torch.as_tensor(extend(h32a)).cuda(), torch.as_tensor(extend(h32b)).cuda())
    xt = tt[pick].to(torch.float64).to(torch.complex128).contiguous()
    xp = tp[pick].to(torch.float64).to(torch.complex128).contiguous()
    ca, cb = p64.fwd(xt, xp)
    torch.cuda.synchronize()

    def nerr(g, r):
        g = np.asarray(g).reshape(len(pick), -1)
        r = np.asarray(r).reshape(len(pick), -1)
        return float(np.max(np.max(np.abs(g - r), axis=1) / np.max(np.abs(r), axis=1)))
    err_adj = max(nerr(tt[pick].cpu().numpy(), ct.real.cpu().numpy()),
                  nerr(tp[pick].cpu().numpy(), cp.real.cpu().numpy()))
    err_fwd = max(nerr(ra[pick].cpu().numpy(), ca.cpu().numpy()[:, full]),
                  nerr(rb[pick].cpu().numpy(), cb.cpu().numpy()[:, full]))
    p64.close()
    pr.close()
    return {"value": B / (ms * 1e-3), "unit": "fields/s", "ms_per_step": ms, "fields": B,
            "coefficients_per_family": L * (L + 3) // 2, "max_rel_err_adj_vs_fp64": err_adj,
            "max_rel_err_fwd_vs_fp64": err_fwd, "sampled_fields": pick, "kernel_ms": prof}


# ---------------------------------------------------------------------------
def reference_arm(args, rank):
    """The CPU oracle (separable FP64 form) on a bounded sample: each step computes
    one field's AdjVSHT + FwdVSHT restricted to every 64th order (1/64 of the
    orders), i.e. 1/64 of one field; value = sampled fraction / time."""
    import numpy as np
    import oracle
    from paper_1908_00041_gb300 import synthetic
    if rank != 0:
        return None
    L = args.L
    x, W, theta, phi = oracle.grid(L)
    a, b = synthetic.coefficients(L, 1, seed=2, decay=1.5)
    mstep = 64
    starts = list(range(mstep))
    nm = 2 * L + 1

    def step(i):
        s0 = starts[i % mstep]
        tt, tp = oracle.adj_sep_orders(L, x, a[0], b[0], 2 * (L + 1), s0, mstep)
        tt = tt.astype(np.complex64).astype(np.complex128)
        tp = tp.astype(np.complex64).astype(np.complex128)
        oracle.fwd_sep_orders(L, x, W, tt, tp, s0, mstep)
        return len(range(s0, nm, mstep)) / nm

    steps = args.steps or 5
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    frac = 0.0
    for i in range(steps):
        frac += step(args.warmup + i)
    dt = time.perf_counter() - t0
    val = frac / dt
    cores = oracle.num_threads()
    sample = ("one field, every 64th order of the L=1023 adjoint+forward (separable FP64 "
              "oracle, exact per-ring DFT), %d steps" % steps)
    return {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "fields/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "L=%d GL %dx%d, coefficients N(0,1)(l+1)^-1.5, seed 2 "
                               "(bounded sample of the batch-32 precision form)" % (L, L + 1, 2 * (L + 1)),
                   "L": L, "batch": 1, "sample_orders_step": mstep},
        "cpu_baseline": {"value": val, "unit": "fields/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "fields/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def oracle_errors(L, a0, b0, tt0, tp0, ga0, gb0):
    """Field 0 of the timed step against the FP64 oracle (separable form, every coefficient
    and grid value): the adjoint's field against the oracle's synthesis of the drawn
    coefficients, and the forward's coefficients against the oracle's analysis of the
    field the adjoint wrote (the forward's own input).  Normwise maxima per family
    (max |difference| / max |reference|), outside the timed region."""
    import numpy as np
    import oracle
    x, W, _, _ = oracle.grid(L)
    t0 = time.perf_counter()
    rt, rp = oracle.adj_sep(L, x, a0, b0, 2 * (L + 1))
    tt0 = tt0.astype(np.complex128)
    tp0 = tp0.astype(np.complex128)
    ra, rb = oracle.fwd_sep(L, x, W, tt0, tp0)

    def nerr(g, r):
        return float(np.max(np.abs(g - r)) / np.max(np.abs(r)))

    e_adj = max(nerr(tt0, rt), nerr(tp0, rp))
    e_fwd = max(nerr(ga0, ra), nerr(gb0, rb))
    return {"vs_oracle_max_rel": max(e_adj, e_fwd), "adj_vs_oracle_max_rel": e_adj,
            "fwd_vs_oracle_max_rel": e_fwd,
            "vs_oracle_sample": "field 0 of the batch, all coefficients and grid points, oracle O3 on %d "
                                "host threads (%.1f s)" % (oracle.num_threads(), time.perf_counter() - t0)}


def cpu_baseline(args):
    """Oracle O3 on the host cores, one field, every 2nd order (half of the work)."""
    import numpy as np
    import oracle
    from paper_1908_00041_gb300 import synthetic
    L = args.L
    x, W, theta, phi = oracle.grid(L)
    a, b = synthetic.coefficients(L, 1, seed=2, decay=1.5)
    mstep = 2
    nm = 2 * L + 1
    t0 = time.perf_counter()
    tt, tp = oracle.adj_sep_orders(L, x, a[0], b[0], 2 * (L + 1), 0, mstep)
    oracle.fwd_sep_orders(L, x, W, tt, tp, 0, mstep)
    dt = time.perf_counter() - t0
    frac = len(range(0, nm, mstep)) / nm
    cores = oracle.num_threads()
    # the same oracle on one thread, over every 32nd order (a sixteenth of the sample above)
    m1 = 32
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        tt, tp = oracle.adj_sep_orders(L, x, a[0], b[0], 2 * (L + 1), 0, m1)
        oracle.fwd_sep_orders(L, x, W, tt, tp, 0, m1)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    frac1 = len(range(0, nm, m1)) / nm
    return {"value": frac / dt, "unit": "fields/s", "cores": cores, "kind": "oracle",
            "sample": "one field of the L=%d workload, adjoint+forward over every 2nd order "
                      "(%.4f of the orders) with the separable FP64 oracle, %.1f s" % (L, frac, dt),
            "single_thread": {"value": frac1 / dt1, "unit": "fields/s", "cores": 1,
                              "sample": "every 32nd order (%.4f of the orders), %.1f s" % (frac1, dt1)},
            "small_configs": cpu_small_configs()}


def cpu_small_configs():
    """The oracle at the one-field FP64 configurations, L = 16 (17 x 34 grid) and L = 511
    (512 x 1024), adjoint + forward in fields/s: the separable form (O3) and the direct
    definition (every coefficient a sum over all grid points, every grid value a sum over all
    coefficients) on samples scaled to the whole transform."""
    import numpy as np
    import oracle
    from paper_1908_00041_gb300 import synthetic
    out = {}
    for L, mstep, ncoef_s, npts_s in ((16, 1, None, None), (511, 8, 16, 16)):
        x, W, _, _ = oracle.grid(L)
        nlat, nphi = L + 1, 2 * (L + 1)
        a, b = synthetic.coefficients(L, 1, seed=1, decay=1.0)
        nm = 2 * L + 1
        t0 = time.perf_counter()
        tt, tp = oracle.adj_sep_orders(L, x, a[0], b[0], nphi, 0, mstep)
        oracle.fwd_sep_orders(L, x, W, tt, tp, 0, mstep)
        t_sep = (time.perf_counter() - t0) / (len(range(0, nm, mstep)) / nm)
        K = L * L + 2 * L
        ls = np.array([l for l in range(1, L + 1) for _ in range(-l, l + 1)])
        ms = np.array([m for l in range(1, L + 1) for m in range(-l, l + 1)])
        js, ks = np.divmod(np.arange(nlat * nphi), nphi)
        if ncoef_s:
            pick = np.random.default_rng(0).choice(K, ncoef_s, replace=False)
            ls, ms = ls[pick], ms[pick]
            pt = np.random.default_rng(1).choice(nlat * nphi, npts_s, replace=False)
            js, ks = js[pt], ks[pt]
        t0 = time.perf_counter()
        oracle.fwd_literal_grid_coefs(L, x, W, tt, tp, ls, ms)
        t_f = (time.perf_counter() - t0) * K / len(ls)
        t0 = time.perf_counter()
        oracle.adj_literal_grid_points(L, nlat, nphi, x, a[0], b[0], js, ks)
        t_a = (time.perf_counter() - t0) * nlat * nphi / len(js)
        out["L%d" % L] = {"separable_fields_per_s": 1.0 / t_sep, "direct_fields_per_s": 1.0 / (t_f + t_a),
                          "sample": "separable over every %d%s order; direct over %s" % (
                              mstep, {1: "st", 8: "th"}[mstep],
                              "all coefficients and grid points" if not ncoef_s else
                              "%d coefficients and %d grid points, scaled" % (ncoef_s, npts_s))}
    return out


def bind_to_gpu_cpus(dev):
    """Run this process on the CPUs local to GPU `dev` (its PCI device's local_cpulist), so
    that the pinned host buffers of the end-to-end measurement are allocated on the GPU's own
    memory node; returns the number of CPUs kept, or None when the list is unavailable."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (
            pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open(path) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return len(cpus)
    except Exception:
        return None


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        rec = reference_arm(args, rank)
        if rec is not None:
            print(json.dumps(rec), flush=True)
        return

    import numpy as np
    import torch
    from paper_1908_00041_gb300 import api, synthetic

    torch.cuda.set_device(local)
    host_cpus = bind_to_gpu_cpus(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    api.lib(build_if_missing=True)
    prec_name = args.precision
    if prec_name is None:
        prec_name = "bf16x6"
        try:
            p = api.Plan(16, 1, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
            p.close()
        except api.FavestError:
            prec_name = "fp64"
    prec = api.FAVEST_BF16X6 if prec_name == "bf16x6" else api.FAVEST_FP64
    L, B = args.L, args.batch
    steps = args.steps or (200 if prec_name == "bf16x6" else 10)

    plan = api.Plan(L, B, prec, api.FAVEST_IO_C64)
    # plan set-up (untimed): the generator's block shape picked by the autotuner
    gen_shape = None
    if prec == api.FAVEST_BF16X6:
        gen_shape = list(plan.gen_shape() if args.no_tune else plan.tune()) + [plan.gen_chains()]
    a_h, b_h = synthetic.coefficients(L, B, seed=2, decay=1.5)
    a = torch.as_tensor(a_h).to(torch.complex64).cuda()
    b = torch.as_tensor(b_h).to(torch.complex64).cuda()
    tt = torch.empty(plan.field_shape(), dtype=torch.complex64, device="cuda")
    tp = torch.empty_like(tt)
    a2 = torch.empty_like(a)
    b2 = torch.empty_like(b)
    stream = torch.cuda.current_stream()

    # one recurrence pass per step: the adjoint generates the Legendre operand in the
    # layouts of both directions and the forward call uses it (FAVEST_FLAG_SHARE_LAMBDA)
    share = not args.no_share

    def step():
        plan.adj(a, b, tt, tp, stream=stream, share_lambda=share)
        plan.fwd(tt, tp, a2, b2, stream=stream, share_lambda=share)

    args.warmup = max(args.warmup, 3)      # at least three untimed warm-up steps
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    plan.profile(True)
    plan.profile_read()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    prof = plan.profile_read()
    plan.profile(False)
    assert plan.status() == 0
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, "cuda")
    value = replica_throughput(B, world, ms * 1e-3)
    # the library's own kernel launches in the timed region, as its event records count them
    launches = int(sum(n for _, n in prof.values()))

    # roofline: every kernel's algorithmic work (favest_kernel_work) per launch over its
    # CUDA-event duration, against the peak of the unit that binds it; the line's
    # roofline object is the kernel with the largest share of the timed region
    fp64_probe, fp32_probe = api.favest_probe_peaks()
    kernels, roofline = kernel_rooflines(plan, prof, fp64_probe, fp32_probe, L, B)
    fp64_peak, fp32_peak = alu_peaks()[:2]

    # end-to-end through the public API with host buffers (pinned), per step:
    # H2D of the coefficients, adjoint + forward, D2H of the recovered coefficients
    # end-to-end through the public API with host buffers (pinned), per step: H2D of the
    # step's coefficients, adjoint + forward, D2H of the recovered coefficients.  Steps
    # are pipelined as a user would: two buffer slots, the copy-in of step k+1 and the
    # copy-out of step k-1 run on their own streams while step k computes (the plan's
    # workspace is used by one step at a time, on the compute stream).
    e2e = None
    if not args.no_e2e:
        ha = torch.as_tensor(a_h).to(torch.complex64).pin_memory()
        hb = torch.as_tensor(b_h).to(torch.complex64).pin_memory()
        oa = [torch.empty_like(ha).pin_memory() for _ in range(2)]
        ob = [torch.empty_like(hb).pin_memory() for _ in range(2)]
        da = [torch.empty_like(a) for _ in range(2)]
        db = [torch.empty_like(b) for _ in range(2)]
        ra = [torch.empty_like(a) for _ in range(2)]
        rb = [torch.empty_like(b) for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_comp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        # 20..50 steps: the first copy-in and the last copy-out (about 5 ms together at
        # L = 1023, B = 32) are not overlapped, so few steps would mostly measure the fill
        ke = max(20, min(steps, 50))

        def e2e_step(k):
            q = k % 2
            s_in.wait_event(ev_comp[q])            # slot q's inputs consumed by step k-2
            with torch.cuda.stream(s_in):
                da[q].copy_(ha, non_blocking=True)
                db[q].copy_(hb, non_blocking=True)
            ev_in[q].record(s_in)
            stream.wait_event(ev_in[q])
            stream.wait_event(ev_out[q])           # slot q's results read back (step k-2)
            plan.adj(da[q], db[q], tt, tp, stream=stream, share_lambda=share)
            plan.fwd(tt, tp, ra[q], rb[q], stream=stream, share_lambda=share)
            ev_comp[q].record(stream)
            s_out.wait_event(ev_comp[q])
            with torch.cuda.stream(s_out):
                oa[q].copy_(ra[q], non_blocking=True)
                ob[q].copy_(rb[q], non_blocking=True)
            ev_out[q].record(s_out)

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(ke):
            e2e_step(k)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / ke, dist, "cuda")
        nbytes = ha.numel() * 8 * 2
        assert torch.equal(oa[(ke - 1) % 2], ra[(ke - 1) % 2].cpu())
        # copy rates of this machine (outside the timed region): one step's H2D alone, its D2H
        # alone, and both at once on their two streams, CUDA events on each stream
        def copy_ms(h2d, d2h, reps=3):
            evs = []
            for _ in range(reps):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                if h2d:
                    e[0].record(s_in)
                    with torch.cuda.stream(s_in):
                        da[0].copy_(ha, non_blocking=True)
                        db[0].copy_(hb, non_blocking=True)
                    e[1].record(s_in)
                if d2h:
                    e[2].record(s_out)
                    with torch.cuda.stream(s_out):
                        oa[0].copy_(ra[0], non_blocking=True)
                        ob[0].copy_(rb[0], non_blocking=True)
                    e[3].record(s_out)
                torch.cuda.synchronize()
                evs.append(max(e[0].elapsed_time(e[1]) if h2d else 0.0, e[2].elapsed_time(e[3]) if d2h else 0.0))
            return min(evs)
        h2d_ms, d2h_ms, both_ms = copy_ms(True, False), copy_ms(False, True), copy_ms(True, True)
        e2e = {"value": replica_throughput(B, world, dt), "unit": "fields/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": dt * 1e3, "steps": ke,
               "pipelined": "copy-in / compute / copy-out on three streams, two buffer slots",
               "copy_ms": {"h2d": h2d_ms, "d2h": d2h_ms, "h2d_and_d2h_together": both_ms,
                           "h2d_gbs": nbytes / h2d_ms * 1e-6, "d2h_gbs": nbytes / d2h_ms * 1e-6}}
        del da, db, ra, rb

    # accuracy (outside the timed region): recovered vs drawn coefficients, and the
    # split form against the FP64 path on the same complex64 field
    errors = None
    if not args.no_check and rank == 0:
        ra = a2.cpu().numpy().astype(np.complex128)
        rb = b2.cpu().numpy().astype(np.complex128)

        def nerr(g, r):
            return float(np.max(np.max(np.abs(g - r), axis=-1) / np.max(np.abs(r), axis=-1)))

        def rerr(g, r):
            return float(np.linalg.norm(g - r) / np.linalg.norm(r))
        errors = {"roundtrip_max_rel": max(nerr(ra, a_h), nerr(rb, b_h)),
                  "roundtrip_rms_rel": max(rerr(ra, a_h), rerr(rb, b_h))}
        if prec_name != "fp64":
            p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C64)
            fa, fb = p64.fwd(tt, tp)
            torch.cuda.synchronize()
            fa = fa.cpu().numpy().astype(np.complex128)
            fb = fb.cpu().numpy().astype(np.complex128)
            errors["fwd_vs_fp64_max_rel"] = max(nerr(ra, fa), nerr(rb, fb))
            errors["fwd_vs_fp64_rms_rel"] = max(rerr(ra, fa), rerr(rb, fb))
            p64.close()
        if not args.no_oracle_check:
            errors.update(oracle_errors(L, a_h[0], b_h[0], tt[0].cpu().numpy(), tp[0].cpu().numpy(),
                                        ra[0], rb[0]))

    forms = None
    if not args.no_forms and rank == 0 and prec_name == "bf16x6":
        forms = measure_forms(L, B, a, b, value, fp64_peak)

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        cpu = cpu_baseline(args)

    if rank == 0:
        ws = plan.workspace_bytes()
        rec = {
            "metric": METRIC, "value": value, "unit": "fields/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x6" if prec_name == "bf16x6" else "f64",
            "data": "synthetic",
            "config": {"workload": "precision form: L=%d, Gauss-Legendre grid %dx%d, batch %d "
                                   "fields, coefficients N(0,1)(l+1)^-1.5 seed 2, complex64 tangent "
                                   "components; step = AdjVSHT then FwdVSHT" % (L, L + 1, 2 * (L + 1), B),
                       "L": L, "batch": B, "precision": prec_name, "io": "complex64",
                       "l2": "inputs larger than L2 (%.2f GB per step vs 129 MB L2)"
                             % ((a.numel() * 16 + tt.numel() * 16) / 1e9),
                       "parallelism": "replicas x%d" % world, "workspace_bytes": ws,
                       "generator_shape": list(gen_shape) if gen_shape else None,
                       "host_cpus_local_to_gpu": host_cpus},
            "roofline": roofline, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "errors": errors, "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak,
            "fp64_probe_tflops": fp64_probe, "fp32_probe_tflops": fp32_probe,
            "forms": forms,
        }
        print(json.dumps(rec), flush=True)
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
