"""Benchmark of the band-limited FMM product u = A lambda on GB300.

Workload: N = 2^20 centres uniform in [0,1]^3 (seed 1), inverse multiquadric
Phi(r) = 1/sqrt(1+(eps r)^2), eps = 2, lambda ~ N(0,1), octree depth 5 (32
points per leaf on average), M = 32 nodes per dimension, period L = 4, taper
alpha = 4.5.  One step = one full product (gather, near field, P2M, M2M
upsweep, coupling + downsweep, L2P, scatter) in FP32 arithmetic.  The metric
is points per second (N / step time).

Default: 1 GPU, 10 timed steps after 3 warm-up steps.  Under torchrun (N > 1)
every rank runs an independent replica (the product does not shard; weak
scaling) and rank 0 prints the aggregate over the slowest rank's time.

`--impl reference` times the FP64 CPU oracle instead, on a bounded sample of
the same workload (the centres of one level-1 box, same tree and expansion
parameters), and prints its own line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvec throughput, 3D N=2^20 IMQ eps=2 (FP32 product)"
UNIT = "points/s"
FP32_LANES_PER_SM = 128


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "sm_max_mhz": p.get("sm_max_mhz", 2070.0),
                "bf16_tflops": p.get("bf16_tflops", 1900.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops": 1900.0,
            "source": "fallback"}


def fp32_peak_tflops(sm_mhz, n_sm):
    """FP32 FMA peak from unit counts: SMs x 128 lanes x 2 flop x clock (context only;
    the fractions use the measured rates of measured_unit_peaks)."""
    return n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def measured_unit_peaks(rbf, seconds=0.4):
    """Issue rates of the arithmetic units measured on this device by the library's own
    probe (rbf_peak_probe): FP32 and FP64 FMA in TFLOP/s, MUFU ex2 and rsqrt in T results/s."""
    from paper_1606_07652_gb300 import _lib
    return {"fp32_tflops": _lib.peak_probe(_lib.PROBE_FFMA, seconds) / 1e12,
            "fp64_tflops": _lib.peak_probe(_lib.PROBE_DFMA, seconds) / 1e12,
            "mufu_ex2_tops": _lib.peak_probe(_lib.PROBE_EX2, seconds) / 1e12,
            "mufu_rsqrt_tops": _lib.peak_probe(_lib.PROBE_RSQRT, seconds) / 1e12,
            "source": "rbf_peak_probe: 32 warps per SM of independent FFMA / DFMA / "
                      "ex2.approx / rsqrt.approx chains, CUDA events, %.1f s each" % seconds}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                for r in csv.reader(f):
                    if len(r) >= 9:
                        rows.append([c.strip() for c in r])
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _traffic(kernel_pass):
    """DRAM bytes per launch of a pass from the committed ncu summary, if the kernel
    source has not changed since the counters were taken (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        tab = json.load(f)
    ent = tab.get(kernel_pass)
    if not ent:
        return None
    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return ent["bytes_per_launch"] if sha == ent["source_sha"] else None


def near_pairs(tree):
    e = tree.export()
    n = np.diff(e["leaf_off"])
    tot = 0
    for a in range(len(n)):
        nb = e["near_idx"][e["near_off"][a]:e["near_off"][a + 1]]
        tot += int(n[a]) * int(n[nb].sum())
    return tot


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the job's time is its slowest rank's);
    the value itself when not distributed."""
    if dist is None:
        return float(value)
    import torch
    tt = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def pg_timeout(args):
    """Process-group timeout: a rank that fails or leaves makes the others' next
    collective raise after this long instead of waiting for the library default."""
    import datetime
    return datetime.timedelta(seconds=float(getattr(args, "pg_timeout", 600.0)))


def job_throughput(units_per_rank, world, steps, t_max_ms):
    """Whole-job rate: units every rank processed per step, over the slowest rank's time."""
    return world * units_per_rank * steps / (t_max_ms / 1e3)


def run_ours(args):
    import torch
    import paper_1606_07652_gb300 as rbf
    import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", timeout=pg_timeout(args))
    dev = torch.device("cuda", local)
    X, lam, targets, p = workloads.config2(n=args.n) if args.n else workloads.config2()
    N = len(X)
    Xd = torch.as_tensor(X, device=dev)
    ld = torch.as_tensor(lam, device=dev)
    unit_peaks = None
    if rank == 0:
        unit_peaks = (measured_unit_peaks(rbf) if args.peaks else
                      {"fp32_tflops": 78.5, "fp64_tflops": 1.06, "mufu_ex2_tops": 10.0,
                       "mufu_rsqrt_tops": 5.0,
                       "source": "not measured in this run (--peaks 0): earlier probe values"})
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    tree = rbf.tree_build(Xd, lo=np.zeros(3), side=1.0, depth=p["depth"])
    info = tree.info()
    kw = dict(M=p["M"], period_L=p["L"], window_alpha=p["alpha"])
    prec = rbf.FP32
    u = torch.empty_like(ld)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step():
        rbf.fmm_matvec(tree, p["kernel"], p["eps"], ld, u, prec=prec, **kw)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    rbf.profile(tree, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))            # write > L2 between timed steps (untimed)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    prof = rbf.profile_read(tree)
    rbf.profile(tree, False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = float(np.sum(step_ms))
    t_max = max_over_ranks(t_local, dist, dev)
    ms_per_step = t_max / args.steps
    value = job_throughput(N, world, args.steps, t_max)
    clocks = clk.summary()

    # end to end through the host entry point: pinned host lambda in, host u out
    lam_h = torch.as_tensor(lam).pin_memory()
    u_h = torch.empty(N, dtype=torch.float64).pin_memory()
    rbf.fmm_matvec_host(tree, p["kernel"], p["eps"], lam_h, u_h, prec=prec, **kw)
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rbf.fmm_matvec_host(tree, p["kernel"], p["eps"], lam_h, u_h, prec=prec, **kw)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_t = max_over_ranks(float(np.sum(e2e_ms)), dist, dev)
    e2e = {"value": job_throughput(N, world, args.steps, e2e_t), "unit": UNIT,
           "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8}

    out = None
    if rank == 0:
        peaks = _peaks()
        nmode = (p["M"] // 2 + 1) * (p["M"] + 1) ** 2
        nleaf = info["n_leaf"]
        passes = {}
        for name, v in prof.items():
            if v["launches"]:
                passes[name] = {"ms_per_step": v["ms"] / args.steps, "launches": v["launches"]}
        # algorithmic work per launch: P2M/L2P 8 flops per point and mode, M2L one
        # read and one write of every leaf expansion plus the root, P2P per near pair
        flops_p2m = 8.0 * N * nmode
        bytes_m2l = (2.0 * nleaf + 1.0) * nmode * 8.0
        pairs = near_pairs(tree)
        fp32_peak = unit_peaks["fp32_tflops"]
        work = {
            "p2m": ("alu", flops_p2m / 1e12, fp32_peak, "TFLOP/s"),
            "l2p": ("alu", flops_p2m / 1e12, fp32_peak, "TFLOP/s"),
            "m2l": ("hbm", bytes_m2l / 1e9, peaks["hbm_gbs"], "GB/s"),
            "p2p": ("alu", 11.0 * pairs / 1e12, fp32_peak, "TFLOP/s"),
        }
        m2m_bytes = 0.0
        for l in range(info["depth"]):
            m2m_bytes += (info["n_box"][l] + info["n_box"][l + 1]) * nmode * 8.0
        work["m2m"] = ("hbm", m2m_bytes / 1e9, peaks["hbm_gbs"], "GB/s")
        for name, (bound, amount, peak, unit) in work.items():
            if name in passes:
                ms = passes[name]["ms_per_step"]
                ach = amount / (ms / 1e3)
                passes[name].update({"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                                     "frac": ach / peak})
        if "p2m" in passes:
            from paper_1606_07652_gb300 import _lib
            passes["p2m"]["launch_shape"] = {0: "by rule", 1: "dense (measured)",
                                             2: "wide (measured)"}[_lib.p2m_launch_shape(tree)]
        if "p2p" in passes:
            # one rsqrt per pair (IMQ) on the multi-function unit beside ~11 FP32 flops:
            # the pass is bound by whichever unit its work fills first
            ms = passes["p2p"]["ms_per_step"]
            f_fma = 11.0 * pairs / (ms / 1e3) / 1e12 / fp32_peak
            f_mufu = pairs / (ms / 1e3) / 1e12 / unit_peaks["mufu_rsqrt_tops"]
            passes["p2p"].update({"frac_fp32": f_fma, "frac_mufu": f_mufu,
                                  "mufu_achieved_tops": pairs / (ms / 1e3) / 1e12,
                                  "mufu_peak_tops": unit_peaks["mufu_rsqrt_tops"],
                                  "binding_unit": "fp32" if f_fma >= f_mufu else "mufu",
                                  "frac": max(f_fma, f_mufu)})
        dom = max((k for k in passes if k in work), key=lambda k: passes[k]["ms_per_step"])
        d = passes[dom]
        per_launch_ms = prof[dom]["ms"] / prof[dom]["launches"]
        launches_per_step = prof[dom]["launches"] / args.steps
        roof = {"kernel": dom, "bound": d["bound"],
                "achieved": work[dom][1] / launches_per_step / (per_launch_ms / 1e3),
                "peak": d["peak"], "unit": d["unit"],
                "peak_source": ("of measured FP32 FMA rate (rbf_peak_probe)"
                                if d["bound"] == "alu" else "of %s HBM copy bandwidth"
                                % peaks["source"]),
                "traffic": _traffic(dom)}
        roof["frac"] = roof["achieved"] / roof["peak"]
        gpu_launches = int(sum(v["launches"] for v in prof.values()))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32", "data": "synthetic (seeded uniform centres, N(0,1) coefficients)",
               "config": {"workload": "3D N=%s uniform, IMQ eps=2, depth %d, M=%d, L=4, alpha=4.5"
                                      % ("2^20" if N == 1 << 20 else str(N), info["depth"], p["M"]),
                          "N": N, "d": 3, "depth": info["depth"], "M": p["M"], "modes_per_leaf":
                          nmode, "n_leaf": nleaf, "near_pairs": pairs,
                          "parallelism": "replicas" if world > 1 else "single GPU",
                          "l2": "256 MB buffer written between timed steps"},
               "clocks": clocks, "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roof,
               "passes": passes,
               "unit_peaks": dict(unit_peaks, fp32_unit_count_tflops=fp32_peak_tflops(
                   peaks["sm_max_mhz"], n_sm), n_sm=n_sm)}
        if not args.skip_extra:
            out.update(extra_measurements(rbf, tree, Xd, ld, targets, p, kw, dev, unit_peaks))
        if args.nested:
            out["nested_grid"] = nested_measurement(rbf, tree, Xd, ld, targets, p, kw, dev)
        if args.evaluate:
            out["evaluation"] = evaluation_measurement(rbf, tree, ld, p, kw, dev)
        if args.kernels:
            out["three_kernels"] = kernels_measurement(rbf, dev)
        if args.batch:
            out["batch"] = batch_measurement(rbf, dev)
        if args.solve:
            out["solve"] = solve_measurement(rbf, dev, big=args.solve > 1 or args.solve_big)
        if args.mrhs:
            out["multi_rhs"] = multi_rhs_measurement(rbf, dev, nrhs=args.mrhs_cols, n=args.mrhs_n,
                                                     M=args.mrhs_M)
        if not args.skip_cpu and world == 1:
            out["cpu_baseline"] = cpu_baseline(X, lam, p, budget_s=args.cpu_budget)
            iters = None
            if "solve" in out:
                iters = out["solve"]["n262144"]["fp64_plain"]["iters"]
            out["cpu_baseline_suite"] = cpu_baseline_suite(iters)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    tree.free()
    return out


def extra_measurements(rbf, tree, Xd, ld, targets, p, kw, dev, unit_peaks):
    """FP64 product throughput (with its P2M/L2P fractions of the measured FP64 FMA rate)
    and the error of both products against the FP64 direct sum."""
    import torch
    N = ld.shape[0]
    u32 = torch.empty_like(ld)
    u64 = torch.empty_like(ld)
    rbf.fmm_matvec(tree, p["kernel"], p["eps"], ld, u32, prec=rbf.FP32, **kw)
    rbf.fmm_matvec(tree, p["kernel"], p["eps"], ld, u64, prec=rbf.FP64, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rbf.profile(tree, True)
    e0.record()
    rbf.fmm_matvec(tree, p["kernel"], p["eps"], ld, u64, prec=rbf.FP64, **kw)
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    prof = rbf.profile_read(tree)
    rbf.profile(tree, False)
    nmode = (p["M"] // 2 + 1) * (p["M"] + 1) ** 2
    fp64_passes = {}
    for name, v in prof.items():
        if v["launches"]:
            fp64_passes[name] = {"ms": v["ms"]}
            if name in ("p2m", "l2p"):
                tf = 8.0 * N * nmode / (v["ms"] / 1e3) / 1e12
                fp64_passes[name].update({"achieved_tflops": tf,
                                          "peak_tflops": unit_peaks["fp64_tflops"],
                                          "frac": tf / unit_peaks["fp64_tflops"]})
    tg = torch.as_tensor(np.asarray(targets, dtype=np.int64), device=dev)
    ud = torch.empty(len(targets), dtype=torch.float64, device=dev)
    rbf.direct_sum(Xd, p["kernel"], p["eps"], ld, tg, ud)
    torch.cuda.synchronize()
    ud = ud.cpu().numpy()

    def err(u):
        v = u.cpu().numpy()[targets]
        return {"rel_l2": float(np.linalg.norm(v - ud) / np.linalg.norm(ud)),
                "max_abs": float(np.max(np.abs(v - ud))),
                "max_rel_to_max": float(np.max(np.abs(v - ud)) / np.max(np.abs(ud)))}

    return {"fp64": {"value": N / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                     "passes": fp64_passes},
            "error_vs_direct_4096_targets": {"fp32": err(u32), "fp64": err(u64)}}


def nested_measurement(rbf, tree, Xd, ld, targets, p, kw, dev, steps=5, K=8):
    """The same workload on the nested (scale-invariant) grids of Sec. 4.1.1: FP32
    products timed with CUDA events, per-pass device times, and the error of the
    FP32 and FP64 nested products against the FP64 direct sum on the same targets."""
    import torch
    info = tree.info()
    N = ld.shape[0]
    kwn = dict(kw, grid=rbf.GRID_NESTED, lagrange_K=K)
    u = torch.empty_like(ld)
    for _ in range(2):
        rbf.fmm_matvec(tree, p["kernel"], p["eps"], ld, u, prec=rbf.FP32, **kwn)
    torch.cuda.synchronize()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rbf.profile(tree, True)
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rbf.fmm_matvec(tree, p["kernel"], p["eps"], ld, u, prec=rbf.FP32, **kwn)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = rbf.profile_read(tree)
    rbf.profile(tree, False)
    u64 = torch.empty_like(ld)
    rbf.fmm_matvec(tree, p["kernel"], p["eps"], ld, u64, prec=rbf.FP64, **kwn)
    tg = torch.as_tensor(np.asarray(targets, dtype=np.int64), device=dev)
    ud = torch.empty(len(targets), dtype=torch.float64, device=dev)
    rbf.direct_sum(Xd, p["kernel"], p["eps"], ld, tg, ud)
    torch.cuda.synchronize()
    ud_h = ud.cpu().numpy()

    def err(v):
        v = v.cpu().numpy()[targets]
        return float(np.linalg.norm(v - ud_h) / np.linalg.norm(ud_h))

    # algorithmic HBM bytes of the translation passes (FP32 complex = 8 B per mode)
    nmode = (p["M"] // 2 + 1) * (p["M"] + 1) ** 2
    nb = info["n_box"]
    D = info["depth"]
    up = sum((nb[l] + 2 * nb[l - 1]) * nmode * 8.0 for l in range(2, D + 1))
    cpl = sum((2 * nb[l] + nb[l - 1]) * nmode * 8.0 for l in range(2, D + 1))
    cpl += sum((nb[l - 1] + 2 * nb[l]) * nmode * 8.0 for l in range(3, D + 1))
    hbm = _peaks()["hbm_gbs"]
    passes = {}
    for name, v in prof.items():
        if v["launches"]:
            passes[name] = {"ms_per_step": v["ms"] / steps, "launches": v["launches"] // steps}
    for name, b in (("m2m", up), ("m2l", cpl)):
        if name in passes:
            gbs = b / 1e9 / (passes[name]["ms_per_step"] / 1e3)
            passes[name].update({"algorithmic_GB": b / 1e9, "achieved_GBs": gbs,
                                 "frac_of_hbm": gbs / hbm})
    t = float(np.mean(ms))
    return {"workload": "same tree and M; nested grids, Lagrange stencil K=%d" % K,
            "ms_per_step": t, "points_per_s": N / (t / 1e3),
            "rel_err_vs_direct": {"fp32": err(u), "fp64": err(u64)},
            "passes": passes}


def evaluation_measurement(rbf, tree, ld, p, kw, dev, nt=1 << 20, steps=5):
    """The interpolant at nt new uniform points (rbf_eval_*): the one-off set-up
    (tree over centres and new points) and the FP32 evaluation per call."""
    import torch
    Y = torch.as_tensor(np.random.default_rng(404).random((nt, 3)), device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = rbf.Evaluator(tree, Y)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    s = torch.empty(nt, dtype=torch.float64, device=dev)
    ev.apply(p["kernel"], p["eps"], ld, s, prec=rbf.FP32, **kw)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ev.apply(p["kernel"], p["eps"], ld, s, prec=rbf.FP32, **kw)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    ev.free()
    t = float(np.mean(ms))
    return {"workload": "2^20 centres (the product's tree) evaluated at %d new uniform points" % nt,
            "setup_ms": setup_ms, "ms_per_evaluation": t, "new_points_per_s": nt / (t / 1e3)}


def kernels_measurement(rbf, dev, n=1 << 20, depths=(4, 5), Ms=(16, 24, 32)):
    """The three kernels of the paper's numerical examples (Sec. 5): IMQ and MQ with
    eps = 1, Wendland (1 - eps r)_+^3 (3 eps r + 1) with eps = 0.5, on 3-D uniform
    centres in the unit cube: for each tree depth and M, the FP32 product time and its
    max-norm error on 1024 targets relative to max |u| of the FP64 direct sum."""
    import torch
    import workloads
    X, lam = workloads.uniform(n, 3, 77)
    Xd = torch.as_tensor(X, device=dev)
    ld = torch.as_tensor(lam, device=dev)
    tg_h = np.random.default_rng(78).choice(n, 1024, replace=False)
    tg = torch.as_tensor(tg_h.astype(np.int64), device=dev)
    kernels = (("IMQ", rbf.IMQ, 1.0, 4.5), ("MQ", rbf.MQ, 1.0, 4.5),
               ("Wendland", rbf.WENDLAND, 0.5, 0.0))
    out = {}
    u = torch.empty_like(ld)
    for name, k, eps, alpha in kernels:
        ud = torch.empty(1024, dtype=torch.float64, device=dev)
        rbf.direct_sum(Xd, k, eps, ld, tg, ud)
        torch.cuda.synchronize()
        umax = float(ud.abs().max())
        rows = []
        for D in depths:
            t = rbf.tree_build(Xd, lo=np.zeros(3), side=1.0, depth=D)
            for M in Ms:
                kw = dict(prec=rbf.FP32, M=M, period_L=4.0, window_alpha=alpha)
                rbf.fmm_matvec(t, k, eps, ld, u, **kw)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                rbf.fmm_matvec(t, k, eps, ld, u, **kw)
                e1.record()
                torch.cuda.synchronize()
                err = float((u[tg] - ud).abs().max()) / umax
                rows.append({"depth": D, "M": M, "ms": e0.elapsed_time(e1), "linf_rel": err})
            t.free()
        out[name] = {"eps": eps, "window_alpha": alpha, "results": rows}
    return {"workload": "3D N=%d uniform in [0,1]^3, L=4, FP32 products, 1024 targets" % n,
            "kernels": out}


def batch_measurement(rbf, dev, n_problems=256, steps=5):
    """256 problems, N log-uniform in [2048, 65536], d in {2,3}, Gaussian or IMQ,
    eps ~ U[1,5], 4 right-hand sides: the cost model sends each problem to the
    direct sum (one persistent launch for all of them), the near field alone or the
    FMM; one graph launch of all FP32 products per step; aggregate points/s =
    sum_p N_p * nrhs_p / product time.  A few lockstep GMRES steps, each one graph
    launch on the device, give the step time."""
    import torch
    import workloads
    from paper_1606_07652_gb300 import _lib
    probs = workloads.config4(n_problems)
    t0 = time.perf_counter()
    tensors = [dict(X=torch.as_tensor(q["X"], device=dev), kernel=q["kernel"], eps=q["eps"],
                    nrhs=q["U"].shape[1]) for q in probs]
    B = _lib.Batch(tensors, tol_kernel=1e-6)
    lay = B.layout()
    setup = time.perf_counter() - t0
    total = lay["total"]
    lam = torch.as_tensor(np.random.default_rng(31).standard_normal(total), device=dev)
    u = torch.empty_like(lam)
    B.matvec(lam, u, rbf.FP32)          # capture
    for _ in range(3):
        B.matvec(lam, u, rbf.FP32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        B.matvec(lam, u, rbf.FP32)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # a few lockstep GMRES steps on the data values
    U = np.concatenate([q["U"].T.ravel() for q in probs])
    ud = torch.as_tensor(U, device=dev)
    x = torch.zeros_like(ud)
    rep = B.solve(ud, x, restart_m=20, max_iters=10, rtol=1e-12, prec=rbf.FP32)
    parts = B.time_parts(rbf.FP32, reps=3)
    st = B.stats()
    B.free()
    tree = lay["depth"] > 0
    dps = st["direct_pairs"] / (parts["direct_ms"] * 1e-3) if parts["direct_ms"] > 0 else None
    return {"problems": n_problems, "systems": int(sum(q["U"].shape[1] for q in probs)),
            "points_x_rhs": int(total), "setup_s": setup,
            "matvec_ms": ms, "value": total / (ms / 1e3), "unit": "points/s (all problems and RHS)",
            "gmres_step_ms": rep["step_ms"], "gmres_steps": rep["iters"],
            "step_over_product": rep["step_ms"] / ms,
            "choice": {"direct": st["n_direct"], "near_field_only": st["n_near_only"],
                       "fmm": st["n_fmm"]},
            "direct_work_items": st["direct_items"],
            "parts_ms": parts,
            "direct_launch": {"pairs": st["direct_pairs"], "pairs_per_s": dps,
                              "fp32_tflops_at_18_flops_per_pair": dps * 18e-12 if dps else None},
            "graph_kernel_nodes": {"product": st["product_nodes"], "gmres_step": st["step_nodes"]},
            "predicted_ms": st["predicted_ms"], "cost_model_s": st["model"],
            "M_range_tree_problems": ([int(lay["M"][tree].min()), int(lay["M"][tree].max())]
                                      if tree.any() else None),
            "depth_range_tree_problems": ([int(lay["depth"][tree].min()),
                                           int(lay["depth"][tree].max())] if tree.any() else None)}


def _curve(hist, every=5):
    """Residual history as compact [iterations, seconds, residual] rows: every FP64
    true residual and every `every`-th inner restart residual."""
    out, k = [], 0
    for it, sec, r, kind in hist:
        if kind == 0 or k % every == 0:
            out.append([it, round(sec, 4), r, "fp64" if kind == 0 else "inner"])
        if kind == 1:
            k += 1
    return out


def _time_to(hist, target, inner_true=False):
    """Seconds at which the true residual first reached target (None if never); with an
    FP64 inner product the restart residuals of a cold start are true residuals too."""
    for it, sec, r, kind in hist:
        if (kind == 0 or inner_true) and r <= target:
            return sec
    return None


def _floor(hist, inner_true=False):
    return min(r for it, sec, r, kind in hist if kind == 0 or inner_true)


def solve_leg(rbf, dev, n, depth, fp64_iters, fp32_iters):
    """The clustered 3-D Gaussian workload (8 Gaussians, sd 0.05, eps = 3, M = 24, L = 3) at n
    centres: plain FP64 FMM-GMRES(50) for at most fp64_iters iterations, FP32 products with
    FP64 refinement, and FP32 with the learned preconditioner (trained on 16,384 of the
    centres, judged by its trial cycle), all asked for 1e-8; residual against wall time for
    each, the floor each reaches and the time each takes to the common reachable residual."""
    import torch
    import workloads
    from paper_1606_07652_gb300 import _lib
    X, u, p = workloads.config3(n)
    Xd = torch.as_tensor(X, device=dev)
    ud = torch.as_tensor(u, device=dev)
    t = rbf.tree_build(Xd, lo=np.zeros(3), side=1.0, depth=depth)
    kw = dict(M=p["M"], period_L=p["L"], window_alpha=p["alpha"], history=4096)
    res = {"workload": "3D N=%d clustered (8 Gaussians, sd 0.05), Gaussian eps=3, depth %d, M=24, "
                       "L=3, u = sin(2 pi x) cos(2 pi y) exp(-z), target 1e-8" % (len(X), depth)}
    lam = torch.zeros_like(ud)
    r64 = rbf.interp_solve(t, p["kernel"], p["eps"], ud, lam, restart_m=50, max_iters=fp64_iters,
                           max_refine=1, rtol=1e-8, inner_prec=rbf.FP64, precond=0, **kw)
    lam.zero_()
    r32 = rbf.interp_solve(t, p["kernel"], p["eps"], ud, lam, restart_m=50, max_iters=fp32_iters,
                           max_refine=8, rtol=1e-8, inner_prec=rbf.FP32, precond=0, **kw)
    net = _lib.Mlp(96, 128, 32, seed=3)
    train = _lib.precond_train(t, p["kernel"], p["eps"], net, n_train=16384, epochs=40,
                               batch=1024, lr=1e-3, delta_rel=1e-12)
    t0 = time.perf_counter()
    _lib.precond_build(t, p["kernel"], p["eps"], net)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    lam.zero_()
    rl = rbf.interp_solve(t, p["kernel"], p["eps"], ud, lam, restart_m=50, max_iters=fp32_iters,
                          max_refine=8, rtol=1e-8, inner_prec=rbf.FP32, precond=1, **kw)
    t.free()
    net.free()
    legs = (("fp64_plain", r64, True), ("fp32_refined_plain", r32, False),
            ("fp32_refined_learned", rl, False))
    common = max(_floor(r["history"], tr) for _, r, tr in legs)
    for name, r, tr in legs:
        hist = r.pop("history")
        r["floor"] = _floor(hist, tr)
        r["seconds_to_common"] = _time_to(hist, common, tr)
        r["curve"] = _curve(hist, every=1 if len(hist) < 40 else 5)
        res[name] = r
    t64, t32 = res["fp64_plain"]["seconds_to_common"], res["fp32_refined_plain"]["seconds_to_common"]
    tl = res["fp32_refined_learned"]["seconds_to_common"]
    res["speedup_to_common"] = {"fp32_refined_plain": t64 / t32 if t64 and t32 else None,
                                "fp32_refined_learned": t64 / tl if t64 and tl else None}
    res["train"] = train
    res["precond_build_s"] = build_s
    res["common_rel_resid"] = common
    res["target_1e-8_reached"] = {k: res[k]["floor"] <= 1e-8
                                  for k in ("fp64_plain", "fp32_refined_plain",
                                            "fp32_refined_learned")}
    res["fp64_iteration_cap"] = fp64_iters
    return res


def learned_gain_leg(rbf, dev, n1=64, eh=1.2):
    """A regime where local cardinal functions are local: 3-D quasi-uniform centres (a
    jittered n1^3 grid, spacing h = 1/n1), Gaussian eps = eh / h.  The cost-model autotuner
    picks no far field (the kernel is below 1e-10 beyond one leaf) and the depth.  Solves to
    1e-8 with FP64 and with FP32 inner products: plain, learned P (a 3 x 256 network trained
    at this eps*h on 65,536 of the centres; the time to build P is counted with the solve,
    the one-off training is reported apart) and exact local cardinal P."""
    import torch
    import workloads
    from paper_1606_07652_gb300 import _lib
    X = workloads.jittered_grid(n1, 3, 12)
    n = len(X)
    u = np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1]) * np.exp(-X[:, 2])
    eps = eh * n1
    prm = _lib.autotune_cost(rbf.GAUSSIAN, eps, 3, n, 1, 1e-10, _lib.cost_calibrate())
    Xd = torch.as_tensor(X, device=dev)
    ud = torch.as_tensor(u, device=dev)
    t = rbf.tree_build(Xd, lo=np.zeros(3), side=1.0, depth=prm["depth"])
    kw = dict(M=prm["M"], period_L=prm["period_L"], window_alpha=prm["window_alpha"],
              restart_m=50, max_iters=3000, max_refine=10, rtol=1e-8)
    res = {"workload": "3D N=%d jittered grid, Gaussian eps=%.1f (eps*h=%.1f), autotuned depth %d, "
                       "M=%d (far-kernel error %.1e)" % (n, eps, eh, prm["depth"], prm["M"],
                                                         prm["err"])}
    net = _lib.Mlp(96, 256, 32, seed=3)
    res["train"] = _lib.precond_train(t, rbf.GAUSSIAN, eps, net, n_train=65536, epochs=200,
                                      batch=1024, lr=1e-3, delta_rel=1e-12)
    res["train"]["network"] = "96 -> 256 -> 256 -> 256 -> 32, BF16"

    def build(use_net):
        t0 = time.perf_counter()
        _lib.precond_build(t, rbf.GAUSSIAN, eps, net if use_net else None)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def solve(pc, inner):
        lam = torch.zeros_like(ud)
        r = rbf.interp_solve(t, rbf.GAUSSIAN, eps, ud, lam, precond=pc, inner_prec=inner, **kw)
        return {k: r[k] for k in ("status", "iters", "used_fallback", "rel_resid", "seconds",
                                  "matvecs_inner", "matvecs_fp64")}

    for tag, inner in (("fp64_inner", rbf.FP64), ("fp32_inner", rbf.FP32)):
        leg = {"plain": solve(0, inner)}
        leg["learned_build_s"] = build(True)
        leg["learned"] = solve(1, inner)
        leg["exact_build_s"] = build(False)
        leg["exact_local"] = solve(1, inner)
        pl, le = leg["plain"], leg["learned"]
        total = le["seconds"] + leg["learned_build_s"]
        leg["learned_vs_plain"] = {"iters": [le["iters"], pl["iters"]],
                                   "seconds_with_build": [total, pl["seconds"]],
                                   "fewer_iterations": le["iters"] < pl["iters"],
                                   "less_time": total < pl["seconds"]}
        res[tag] = leg
    t.free()
    net.free()
    return res


def solve_measurement(rbf, dev, big=True):
    """The solve half of the metric: the clustered workload at N = 262,144 and at
    N = 2^20 (FP64 capped to bound the run), and the learned-preconditioner leg."""
    out = {"n262144": solve_leg(rbf, dev, 262144, 6, fp64_iters=150, fp32_iters=1500)}
    if big:
        out["n1048576"] = solve_leg(rbf, dev, 1 << 20, 7, fp64_iters=60, fp32_iters=600)
    out["learned_gain"] = learned_gain_leg(rbf, dev)
    if big:   # the same regime at about 10^6 centres (a jittered 102^3 grid)
        out["learned_gain_1m"] = learned_gain_leg(rbf, dev, n1=102)
    return out


def multi_rhs_measurement(rbf, dev, tol=1.5e-7, nrhs=16, n=1 << 19, M=0):
    """d = 5, N = 2^19 uniform, Gaussian eps = 1.5, depth 2 (512 points per leaf), L = 4,
    M = the smallest even M whose measured far-kernel error is <= 1.5e-7.  Times one FP32
    product of a single column and one of the 16-column block (P2M and L2P of the block on
    the tensor cores, one multi-column near-field pass), checks the single column against
    the FP64 direct sum on 2048 targets and the block against single-column products."""
    import torch
    import workloads
    from paper_1606_07652_gb300 import _lib
    X, lam, lamb, targets, p = workloads.config5(n=n, nrhs=nrhs)
    N = len(X)
    if M <= 0:   # grow M to the error target
        M = 8
        err_k = _lib.kernel_error(p["kernel"], p["eps"], 5, M, p["L"], 0.0, 1.0, p["depth"])
        while err_k > tol and M < 24:
            M += 2
            err_k = _lib.kernel_error(p["kernel"], p["eps"], 5, M, p["L"], 0.0, 1.0, p["depth"])
    else:
        err_k = _lib.kernel_error(p["kernel"], p["eps"], 5, M, p["L"], 0.0, 1.0, p["depth"])
    Xd = torch.as_tensor(X, device=dev)
    t = rbf.tree_build(Xd, lo=np.zeros(5), side=1.0, depth=p["depth"])
    kw = dict(M=M, period_L=p["L"], window_alpha=0.0, prec=rbf.FP32)
    ld = torch.as_tensor(lam, device=dev)
    u = torch.empty_like(ld)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rbf.fmm_matvec(t, p["kernel"], p["eps"], ld, u, **kw)
    torch.cuda.synchronize()
    e0.record()
    rbf.fmm_matvec(t, p["kernel"], p["eps"], ld, u, **kw)
    e1.record()
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    tg = torch.as_tensor(np.asarray(targets, dtype=np.int64), device=dev)
    ud = torch.empty(len(targets), dtype=torch.float64, device=dev)
    rbf.direct_sum(Xd, p["kernel"], p["eps"], ld, tg, ud)
    torch.cuda.synchronize()
    err1 = float((u[tg] - ud).norm() / ud.norm())
    Lb = torch.as_tensor(np.ascontiguousarray(lamb.T), device=dev)      # (nrhs, N)
    Ub = torch.empty_like(Lb)
    rbf.fmm_matvec(t, p["kernel"], p["eps"], Lb, Ub, **kw)               # workspace
    torch.cuda.synchronize()
    rbf.profile(t, True)
    e0.record()
    rbf.fmm_matvec(t, p["kernel"], p["eps"], Lb, Ub, **kw)
    e1.record()
    torch.cuda.synchronize()
    msb = e0.elapsed_time(e1)
    prof = rbf.profile_read(t)
    rbf.profile(t, False)
    rbf.check_device_waits()
    us = torch.empty_like(ld)
    diffs = []
    for c in (0, nrhs - 1):
        rbf.fmm_matvec(t, p["kernel"], p["eps"], Lb[c], us, **kw)
        torch.cuda.synchronize()
        diffs.append(float((Ub[c] - us).norm() / us.norm()))
    nmode = (M // 2 + 1) * (M + 1) ** 4
    peaks = _peaks()
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25
    cmacs = float(N) * nmode * nrhs                   # useful complex MACs of P2M (and of L2P)
    passes = {k: v["ms"] for k, v in prof.items() if v["launches"]}
    tc = {}
    for name in ("p2m", "l2p"):
        if name in passes:
            sec = passes[name] / 1e3
            tc[name] = {"ms": passes[name],
                        "fp32_equiv_tflops": 8.0 * cmacs / sec / 1e12,
                        "tf32_issued_tflops": 24.0 * cmacs / sec / 1e12,
                        "tf32_peak_tflops": tf32_peak,
                        "frac_of_tf32_peak": 24.0 * cmacs / sec / 1e12 / tf32_peak}
    t.free()
    return {"workload": f"5D N={N} uniform, Gaussian eps=1.5, depth 2, L=4, M={M} "
                        f"(far-kernel error {err_k:.2e}), {nrhs} columns",
            "single_column_ms": ms1, "single_column_points_per_s": N / (ms1 / 1e3),
            "single_column_rel_err_vs_direct_2048": err1,
            "block_ms": msb, "block_points_x_rhs_per_s": N * nrhs / (msb / 1e3),
            "speedup_vs_columns": ms1 * nrhs / msb,
            "block_vs_single_rel_diff": max(diffs), "block_passes_ms": passes,
            "tensor_core_passes": tc,
            "tf32_peak_source": "measured bf16 burst x 1.1/2.25 (nominal TF32/BF16 ratio)"}


def _oracle_sample(X, lam, p):
    """Centres of the level-1 box at the origin (about N/8), same tree and parameters."""
    k = np.floor(X * 2).astype(np.int64)
    sel = np.all(k == 0, axis=1)
    return X[sel], lam[sel]


def cpu_baseline(X, lam, p, budget_s=60.0):
    import oracle as O
    Xs, ls = _oracle_sample(X, lam, p)
    t0 = time.perf_counter()
    T = O.tree(Xs, np.zeros(3), 1.0, p["depth"])
    wc = O.coeffs_sampled(p["kernel"], p["eps"], 3, p["M"], p["L"], p["alpha"], 1.0)
    t1 = time.perf_counter()
    O.fmm(T, ls, p["kernel"], p["eps"], wc, p["M"], p["L"])
    t2 = time.perf_counter()
    return {"value": len(Xs) / (t2 - t1), "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle MLFMM product on the {len(Xs)} centres of the level-1 box at "
                      f"the origin (same root cube, depth 5, M=32, L=4, alpha=4.5); "
                      f"setup {t1 - t0:.1f} s not timed, product {t2 - t1:.1f} s"}


def _box_sample(X, level, pick=None):
    """Indices of the centres in one level-`level` box of the unit cube: the box at the
    origin, or the most populated one (pick='max')."""
    k = np.minimum(np.floor(X * (1 << level)).astype(np.int64), (1 << level) - 1)
    code = np.zeros(len(X), dtype=np.int64)
    for t in range(X.shape[1]):
        code = code * (1 << level) + k[:, t]
    if pick == "max":
        target = np.bincount(code).argmax()
    else:
        target = 0
    return np.flatnonzero(code == target)


def _timed_oracle(fn, threads):
    import oracle as O
    O.set_num_threads(threads)
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def cpu_baseline_suite(solve_iters=None):
    """The oracle on the host cores, on all of them and on one, for the configurations
    of the measurement plan: c1 in full (product and direct sum), c2 on the centres of
    one level-2 box (same tree and expansion), the c5 direct sum on sampled targets, and
    c3 as the product on its most populated level-1 box, scaled to the whole workload and
    multiplied by the GPU solve's iteration count (an estimate: the oracle solve itself
    would take hours)."""
    import oracle as O
    import workloads
    allc = O.num_threads()
    out = {"cores_all": allc}
    # c1: d=2, N=4096, Gaussian eps=4, depth 3, M=32, L=2.5
    X1, lam1, p1 = workloads.config1()
    T1 = O.tree(X1, np.zeros(2), 1.0, p1["depth"])
    wc1 = O.coeffs_sampled(p1["kernel"], p1["eps"], 2, p1["M"], p1["L"], p1["alpha"], 1.0)
    c1 = {}
    for tag, th in (("all_cores", allc), ("one_core", 1)):
        sec = _timed_oracle(lambda: O.fmm(T1, lam1, p1["kernel"], p1["eps"], wc1, p1["M"],
                                          p1["L"]), th)
        c1[tag] = {"points_per_s": len(X1) / sec, "seconds": sec}
    sec = _timed_oracle(lambda: O.direct(X1, lam1, p1["kernel"], p1["eps"]), allc)
    c1["direct_all_cores"] = {"points_per_s": len(X1) / sec, "seconds": sec}
    out["c1"] = dict(c1, sample="all 4096 centres")
    # c2: centres of the level-2 box at the origin, depth 5, M=32, L=4, alpha=4.5
    X2, lam2, _, p2 = workloads.config2()
    sel = _box_sample(X2, 2)
    Xs, ls = X2[sel], lam2[sel]
    T2 = O.tree(Xs, np.zeros(3), 1.0, p2["depth"])
    wc2 = O.coeffs_sampled(p2["kernel"], p2["eps"], 3, p2["M"], p2["L"], p2["alpha"], 1.0)
    c2 = {}
    for tag, th in (("all_cores", allc), ("one_core", 1)):
        sec = _timed_oracle(lambda: O.fmm(T2, ls, p2["kernel"], p2["eps"], wc2, p2["M"], p2["L"]), th)
        c2[tag] = {"points_per_s": len(Xs) / sec, "seconds": sec}
    out["c2"] = dict(c2, sample="%d centres of the level-2 box at the origin" % len(Xs))
    # c5: direct sum over all 2^19 centres at sampled targets (the oracle FMM's per-level
    # coupling is out of reach in 5-D)
    X5, lam5, _, tg5, p5 = workloads.config5()
    c5 = {}
    for tag, th, nt in (("all_cores", allc, 1024), ("one_core", 1, 64)):
        sec = _timed_oracle(lambda: O.direct(X5, lam5, p5["kernel"], p5["eps"], tg5[:nt]), th)
        c5[tag] = {"targets_per_s": nt / sec, "pairs_per_s": nt * len(X5) / sec, "seconds": sec}
    out["c5"] = dict(c5, sample="direct sum over %d centres at 1024 / 64 targets" % len(X5))
    # c3: product on the most populated level-1 box (depth 6, M=24, L=3), scaled
    X3, u3, p3 = workloads.config3()
    sel = _box_sample(X3, 1, pick="max")
    lam3 = np.random.default_rng(5).standard_normal(len(sel))
    T3 = O.tree(X3[sel], np.zeros(3), 1.0, 6)
    wc3 = O.coeffs_sampled(p3["kernel"], p3["eps"], 3, p3["M"], p3["L"], p3["alpha"], 1.0)
    sec = _timed_oracle(lambda: O.fmm(T3, lam3, p3["kernel"], p3["eps"], wc3, p3["M"], p3["L"]), allc)
    per = sec * len(X3) / len(sel)
    out["c3"] = {"sample": "%d centres of the most populated level-1 box" % len(sel),
                 "sample_seconds": sec, "per_product_estimate_s": per,
                 "iterations": solve_iters,
                 "solve_estimate_s": per * solve_iters if solve_iters else None}
    O.set_num_threads(allc)
    return out


def run_reference(args):
    """The oracle (the paper ships no code) as the reference arm: W untimed and K timed
    steps, each the oracle's FP64 multilevel FMM product on a bounded sample of workload
    (2) with the same root cube, depth and expansion (the centres of the level-1 box at the
    origin, about 5 s a step on 16 cores; of the level-2 box when K > 12, so that the run
    stays within a few minutes); value = sample points / median step time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle as O
    import workloads
    X, lam, _, p = workloads.config2()
    level = 1 if args.steps <= 12 else 2
    sel = _box_sample(X, level)
    Xs, ls = X[sel], lam[sel]
    t0 = time.perf_counter()
    T = O.tree(Xs, np.zeros(3), 1.0, p["depth"])
    wc = O.coeffs_sampled(p["kernel"], p["eps"], 3, p["M"], p["L"], p["alpha"], 1.0)
    setup_s = time.perf_counter() - t0
    step = lambda: O.fmm(T, ls, p["kernel"], p["eps"], wc, p["M"], p["L"])
    for _ in range(max(args.warmup, 0)):
        step()
    secs = []
    for _ in range(max(args.steps, 1)):
        t1 = time.perf_counter()
        step()
        secs.append(time.perf_counter() - t1)
    med = float(np.median(secs))
    v = len(Xs) / med
    cb = {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
          "sample": f"FP64 oracle MLFMM product on the {len(Xs)} centres of the level-{level} box "
                    f"at the origin (same root cube, depth 5, M=32, L=4, alpha=4.5); setup "
                    f"{setup_s:.1f} s not timed; median of {len(secs)} steps {med:.2f} s"}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": len(secs), "warmup": args.warmup, "ms_per_step": med * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uniform centres, N(0,1) coefficients)",
            "config": {"workload": "3D N=2^20 uniform, IMQ eps=2, depth 5, M=32, L=4, alpha=4.5",
                       "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=60.0)
    ap.add_argument("--pg-timeout", type=float, default=600.0,
                    help="seconds before a collective waiting on a lost rank raises (N > 1)")
    ap.add_argument("--n", type=int, default=0, help="override the number of centres (profiling)")
    ap.add_argument("--peaks", type=int, default=1,
                    help="measure the unit peaks first (0: skip, for profiler runs)")
    ap.add_argument("--batch", type=int, default=1, help="also time the 256-problem batch")
    ap.add_argument("--nested", type=int, default=1, help="also time the nested-grid product")
    ap.add_argument("--evaluate", type=int, default=1,
                    help="also time the evaluation at 2^20 new points")
    ap.add_argument("--kernels", type=int, default=1,
                    help="also run the IMQ / MQ / Wendland error-vs-M sweep")
    ap.add_argument("--solve", type=int, default=1, help="also run the solve comparison")
    ap.add_argument("--solve-big", type=int, default=1,
                    help="include the N=2^20 solve leg (about a minute)")
    ap.add_argument("--mrhs", type=int, default=1,
                    help="also time the 5D 16-column product on the tensor cores")
    ap.add_argument("--mrhs-n", type=int, default=1 << 19, help="centres of the 5D product")
    ap.add_argument("--mrhs-M", type=int, default=0, help="modes per dimension (0: error target)")
    ap.add_argument("--mrhs-cols", type=int, default=16, help="columns of the 5D block")
    args = ap.parse_args()
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
