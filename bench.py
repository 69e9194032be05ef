"""Benchmark: MG setup (iCSVD) + Galerkin coarse build + solve to 1e-10 on one GB300.

A step is one pass of the whole hot path on the 16^3 x 32 near-critical isotropic
workload: Philox test vectors smoothed by GMRES (Eq. 2), chiral split and streaming
SVD into P (Algorithm 3), Galerkin coarse operator (Eq. 5), and the K-cycle FGMRES
solve of D x = b (Eq. 1) to a true relative residual of 1e-10, in the mixed-precision
form (FP32 setup smoother and inner solve, FP64 SVD / coarse assembly / refinement).
The plain FP64 form of the same step is timed beside it.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_16^3x32_near_critical"
METRIC = "MG setup+solve seconds to 1e-10 residual (mixed precision); Dslash GB/s"
# The timed step's K-cycle post-smoother runs its 8 GMRES steps on the even-odd Schur system
# (even-odd preconditioning, Sec. 1), in both the mixed and the FP64 form; the same step with
# the smoother on the full system is timed beside it.
SCHUR_SMOOTHER = True


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self.rows
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[2 + i]
                          and "Not" not in r[2 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


class L2Flush:
    """Evicts L2 between timed launches: writes a 256 MB buffer (larger than the 129 MB L2)
    and then reads a second 256 MB buffer, so the lines left in L2 are clean and the next
    kernel is not charged for writing the flush data back to HBM."""

    def __init__(self, dev):
        import torch
        n = 256 * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device=dev)
        self.r = torch.ones(n, dtype=torch.float32, device=dev)
        self.s = torch.empty((), dtype=torch.float32, device=dev)

    def zero_(self):
        import torch
        self.w.zero_()
        torch.sum(self.r, dim=0, out=self.s)


def max_over_ranks(t, device=None):
    """Replicas only: the job's step time is the slowest rank's (no data-path collective)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# DRAM bytes per launch (read + write, dram__bytes_read.sum + dram__bytes_write.sum averaged
# over the launches of one warm-up and one timed step) from one ncu capture of this bench
# command on its workload, reported as roofline.traffic for that kernel; an entry is removed
# whenever its kernel changes, until it is captured again.
NCU_TRAFFIC = {("galerkin_tc", "c2_16^3x32_near_critical"): 1.9608e9,
               ("dslash_proj", "c2_16^3x32_near_critical"): 516.9e6}


def kernel_bound(name, alu, peaks, peak_kind):
    """(bound, peak, unit, source) of a library kernel, by the arithmetic it runs on."""
    if name.startswith("svd_jacobi") or name in ("coarse_gmres", "cgs_givens"):
        # data-dependent sweep / iteration counts and grid barriers: no fixed algorithmic
        # flop or byte count per launch, so no roofline fraction
        return "latency", None, "TFLOP/s", "none"
    if name.endswith("_df64"):
        # double-float: one real multiply-add (2 FP64-equivalent flops) costs 12 FP32
        # instructions (1 mul, 3 fma, 8 add/sub), so the peak is the FP32 FMA rate / 12
        return "alu", alu["fp32"] / 12.0, "TFLOP/s", "measured FP32 FMA rate / 12"
    if name.endswith("_tc"):
        # the method's FP64-equivalent flops; the exact bf16 digit-plane products it issues on
        # the tensor pipe are reported beside them.  Its time is set by the double-float staging
        # (colour transport, digit split) on the FP32 units, so that is the peak it is set against
        return "alu", alu["fp32"] / 12.0, "TFLOP/s", "measured FP32 FMA rate / 12 (staging)"
    if name.endswith("_fp64") or name.startswith("galerkin") or name == "dslash_c128":
        # the FP64 stencil runs at the FP64 FMA rate (1/74 of FP32 on this part), not at HBM
        return "alu", alu["fp64"], "TFLOP/s", "measured FP64 FMA rate"
    return "hbm", peaks["hbm_gbs"], "GB/s", peak_kind


def kernel_table(kern, alu, peaks, peak_kind):
    """Per-kernel table of the timed steps and the roofline of the dominant kernel.

    kern: {name: {"launches", "ms", "bytes", "flops"}} per step, from the library's per-launch
    CUDA events.  Each kernel is set against the peak of the unit that bounds it; kernels
    bound by latency (barriers, data-dependent sweeps) get no fraction.  The dominant kernel
    is the one with the largest summed time among those with a peak.  Returns (kernels, roof);
    roof is None when no kernel was timed.
    """
    kernels, roof = {}, None
    if not kern:
        return kernels, roof
    tot = sum(v["ms"] for v in kern.values())
    for name, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms"]):
        ent = {"launches_per_step": v["launches"], "ms_per_step": v["ms"],
               "share": v["ms"] / tot if tot > 0 else 0.0}
        if v["ms"] > 0:
            ent["GBps"] = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            ent["TFLOPs"] = v["flops"] / (v["ms"] * 1e-3) / 1e12
            bound, pk, unit, src = kernel_bound(name, alu, peaks, peak_kind)
            ach = ent["TFLOPs"] if unit == "TFLOP/s" else ent["GBps"]
            ent.update({"bound": bound, "frac": ach / pk if pk else None})
            if v.get("issued_flops"):
                tis = v["issued_flops"] / (v["ms"] * 1e-3) / 1e12
                ent["tensor_issued_TFLOPs"] = tis
                ent["tensor_issued_frac_of_bf16"] = tis / peaks["bf16_tflops"]
        kernels[name] = ent
    ranked = [kv for kv in kern.items()
              if kv[1]["ms"] > 0 and kernel_bound(kv[0], alu, peaks, peak_kind)[1]]
    if not ranked:
        return kernels, roof
    name, v = max(ranked, key=lambda kv: kv[1]["ms"])
    per_launch_s = v["ms"] * 1e-3 / max(v["launches"], 1e-9)
    bound, pk, unit, src = kernel_bound(name, alu, peaks, peak_kind)
    if unit == "TFLOP/s":
        ach = v["flops"] / max(v["launches"], 1e-9) / per_launch_s / 1e12
        roof = {"kernel": name, "bound": bound, "achieved": ach, "peak": pk,
                "unit": unit, "frac": ach / pk, "peak_source": src,
                "traffic": NCU_TRAFFIC.get((name, WORKLOAD)),
                "avg_launch_us": per_launch_s * 1e6,
                "algorithmic_flops_per_launch": v["flops"] / max(v["launches"], 1e-9),
                "algorithmic_bytes_per_launch": v["bytes"] / max(v["launches"], 1e-9)}
    else:
        ach = v["bytes"] / max(v["launches"], 1e-9) / per_launch_s / 1e9
        roof = {"kernel": name, "bound": bound, "achieved": ach, "peak": pk,
                "unit": unit, "frac": ach / pk, "peak_source": src,
                "traffic": NCU_TRAFFIC.get((name, WORKLOAD)),
                "avg_launch_us": per_launch_s * 1e6,
                "algorithmic_bytes_per_launch": v["bytes"] / max(v["launches"], 1e-9)}
    return kernels, roof


def anisotropic_leg(api, synthetic, dev, step, reps=2):
    """Setup + solve seconds on the anisotropic 16^3 x 64 lattice (2x2x2x4 aggregates, k = 24,
    64 test vectors in 4 streams) with the post-smoother in FP16 / BF16 storage, and in FP64."""
    import torch
    cfg = dict(synthetic.WORKLOADS["c3_16^3x64_aniso"])
    cfg["kappa"] = synthetic.kappa_of(cfg)
    U = torch.from_numpy(synthetic.make_links(cfg)).to(dev)
    b = torch.from_numpy(synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])).to(dev)
    out = {"dims": list(cfg["dims"]), "kappa": cfg["kappa"], "k": cfg["k"], "r": cfg["r"],
           "n_s": cfg["n_s"]}
    for tag, setup, solve in (("f16", "c64", "f16"), ("bf16", "c64", "bf16"),
                              ("fp32", "c64", "c64"), ("fp64", "c128", "c128")):
        p = api.params(cfg["dims"], cfg["block"], cfg["kappa"], cfg["k"], cfg["r"], cfg["n_s"],
                       cfg["sweeps"], cfg["tv_seed"], cfg["hop_weight"], cfg["bc"],
                       setup_dtype=setup, solve_dtype=solve)
        step(p, U, b)   # warm-up
        ts = []
        for _ in range(reps if tag != "fp64" else 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = step(p, U, b)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        out[tag] = {"seconds": float(np.mean(ts)), "outer": info["outer"],
                    "refinements": info["refinements"], "residual": info["residual"]}
    out["f16_over_fp64_speedup"] = out["fp64"]["seconds"] / out["f16"]["seconds"]
    out["galerkin_k24"] = galerkin_k24(api, U, cfg, dev)
    return out


def galerkin_k24(api, U, cfg, dev, reps=3):
    """Double-float Galerkin build (Eq. 5) of the k = 24 hierarchy: the tensor-pipe digit
    contraction on the setup's own orthonormal prolongator, and the FP32-unit double-float
    kernel that the build runs instead on Gaussian tiles of the same shape (entries outside
    the fixed-point range).  Per-launch times from CUDA events around each kernel."""
    import torch
    from paper_2505_14399_gb300 import _lib
    p = api.params(cfg["dims"], cfg["block"], cfg["kappa"], cfg["k"], cfg["r"], cfg["n_s"],
                   cfg["sweeps"], cfg["tv_seed"], cfg["hop_weight"], cfg["bc"],
                   setup_dtype="c64", solve_dtype="c64")
    h = api.Hierarchy(U, p)

    def build():
        h.coarse_build()
        torch.cuda.synchronize()
        _lib.check(_lib.lib().mg_profile_enable(1, 1000), "mg_profile_enable")
        try:
            for _ in range(reps):
                h.coarse_build()
            torch.cuda.synchronize()
            kern = json.loads(_lib.lib().mg_profile_report().decode())
        finally:
            _lib.lib().mg_profile_enable(0, 0)
        return kern

    kt = build()
    g = torch.Generator(device="cpu").manual_seed(11)
    shape = (h.d, 2, h.k, 6 * h.nd)
    G = torch.complex(torch.randn(shape, generator=g, dtype=torch.float64),
                      torch.randn(shape, generator=g, dtype=torch.float64)).to(dev)
    h.set_prolongator(G)
    kf = build()
    h.close()
    tc, fb = kt["galerkin_tc"], kf.get("galerkin_tc_range_fallback")
    out = {"k": cfg["k"], "sites": int(np.prod(cfg["dims"])), "block": list(cfg["block"]),
           "tensor_ms": tc["ms"] / reps, "method_gflop": tc["flops"] / reps / 1e9,
           "tensor_method_TFLOPs": tc["flops"] / (tc["ms"] * 1e-3) / 1e12,
           "tensor_issued_TFLOPs": tc.get("issued_flops", 0.0) / (tc["ms"] * 1e-3) / 1e12,
           "fallback_on_gaussian_tiles": fb is not None}
    if fb is not None:
        out["fp32_unit_ms"] = fb["ms"] / reps
        out["tensor_speedup"] = fb["ms"] / tc["ms"]
    return out


def dslash_32(api, synthetic, dev, flush, peaks, peak_kind, reps=20):
    """The solver's FP32 stencil (lane-contiguous links) on a 32^3 x 64 lattice, one launch
    per timing with the L2 flushed before it: 1.007 GB of algorithmic traffic per apply
    (24 + 24 spinor reals and 72 link reals per site).  Timed with the links stored as two
    rows (the third rebuilt; 96 reals cross HBM per site) and as three rows (120 reals)."""
    import torch
    from paper_2505_14399_gb300 import _lib
    dims = (32, 32, 32, 64)
    V = int(np.prod(dims))
    U = torch.from_numpy(synthetic.smooth_links(dims, 1003)).to(dev)
    psi = torch.from_numpy(synthetic.gaussian_rhs(dims, 9)).to(torch.complex64).to(dev)
    out = torch.empty_like(psi)
    res = {}
    for compress in (1, 0):
        p = api.params(dims, (4, 4, 4, 4), 0.13, 24, 24, 2, link_compress=compress)
        h = api.Hierarchy(U, p, setup=False)
        rows = _lib.lib().mg_link_rows(h._h)
        ev = []
        for i in range(reps + 3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            h.apply_fine(psi, out=out)
            e1.record()
            torch.cuda.synchronize()
            if i >= 3:
                ev.append(e0.elapsed_time(e1) / 1e3)
        h.close()
        t = float(np.mean(ev))
        moved = V * 4.0 * (48 + 4 * 6 * rows)
        res[rows] = {"avg_launch_us": t * 1e6, "achieved": V * 480.0 / t / 1e9,
                     "bytes_moved_per_apply": moved, "moved_GBps": moved / t / 1e9}
    del U
    best = res[2]
    gbs = best["achieved"]
    return {"kernel": "dslash_c64, lane-contiguous two-row links (32^3x64, L2 flushed)",
            "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"], "peak_source": peak_kind,
            "avg_launch_us": best["avg_launch_us"], "algorithmic_bytes": V * 480.0,
            "bytes_moved": best["bytes_moved_per_apply"],
            "moved_frac": best["moved_GBps"] / peaks["hbm_gbs"],
            "three_row_links": dict(res[3], frac=res[3]["achieved"] / peaks["hbm_gbs"])}


def bench_config(cfg, world):
    """The `config` object of the JSON line (both arms): the workload and its parameters."""
    return {"workload": WORKLOAD, "dims": list(cfg["dims"]), "block": list(cfg["block"]),
            "k": cfg["k"], "r": cfg["r"], "n_s": cfg["n_s"], "sweeps": cfg["sweeps"],
            "kappa": cfg["kappa"], "tol": 1e-10, "nrhs": 1,
            "post_smoother": ("8 GMRES steps on the even-odd Schur system" if SCHUR_SMOOTHER
                              else "8 GMRES steps on D"),
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "256 MB buffer written, then a second 256 MB buffer read, before every timed step"}


def workload():
    from paper_2505_14399_gb300 import synthetic
    cfg = dict(synthetic.WORKLOADS[WORKLOAD])
    cfg["kappa"] = synthetic.kappa_of(cfg)
    return cfg


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_14399_gb300 import _lib, api, synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    cfg = workload()
    dims = cfg["dims"]
    V = int(np.prod(dims))
    U = synthetic.make_links(cfg)
    b = synthetic.gaussian_rhs(dims, cfg["rhs_seed"] + rank)
    Ud = torch.from_numpy(U).to(dev)
    bd = torch.from_numpy(b).to(dev)
    flush = L2Flush(dev)

    def make_params(mixed, schur=SCHUR_SMOOTHER):
        return api.params(dims, cfg["block"], cfg["kappa"], cfg["k"], cfg["r"], cfg["n_s"],
                          cfg["sweeps"], cfg["tv_seed"], cfg["hop_weight"], cfg["bc"],
                          setup_dtype="c64" if mixed else "c128",
                          solve_dtype="c64" if mixed else "c128", schur_smoother=int(schur))

    def step(p, links, rhs, levels=()):
        h = api.Hierarchy(links, p)
        h.coarse_build()
        for blk, kl, rl, nsl, tl in levels:
            h.add_level(blk, kl, rl, nsl, tl)
        x, info = h.solve(rhs, tol=1e-10, maxiter=4000)
        if levels:
            info = dict(info, level_iterations=h.level_iterations())
        h.close()
        return x, info

    def timed(p, links, rhs, K, W, kernel_events=False):
        for _ in range(W):
            step(p, links, rhs)
        torch.cuda.synchronize()
        times, infos = [], []
        if kernel_events:
            # every library launch in the timed steps is bracketed by CUDA events on its stream
            _lib.check(_lib.lib().mg_profile_enable(1, 400000), "mg_profile_enable")
        n0 = _lib.lib().mg_kernel_launches()
        for _ in range(K):
            flush.zero_()
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("timed_step")
            e0.record()
            x, info = step(p, links, rhs)
            e1.record()
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            infos.append(info)
        launches = _lib.lib().mg_kernel_launches() - n0
        kern = None
        if kernel_events:
            kern = json.loads(_lib.lib().mg_profile_report().decode())
            _lib.lib().mg_profile_enable(0, 0)
            for v in kern.values():
                for key in ("launches", "ms"):
                    v[key] = v[key] / K
                v["bytes"] /= K
                v["flops"] /= K
                if "issued_flops" in v:
                    v["issued_flops"] /= K
        t = max_over_ranks(float(np.mean(times)), dev if world > 1 else None)
        return t, infos[-1], launches // max(K, 1), x, kern

    # measured arithmetic peaks (FMA chains on every SM) for the ALU-bound kernels
    alu = {}
    for key, dt in (("fp64", _lib.MG_C128), ("fp32", _lib.MG_C64)):
        tf = ctypes.c_double(0)
        _lib.check(_lib.lib().mg_probe_fma_peak(dt, ctypes.byref(tf), None), "mg_probe_fma_peak")
        alu[key] = tf.value

    pm, p64 = make_params(True), make_params(False)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.nvtx.range_push("mixed")
    t_mixed, info_m, launches, x, _ = timed(pm, Ud, bd, args.steps, args.warmup)
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    # the same steps again with every library launch bracketed by CUDA events (per-kernel
    # times for the roofline); the events cost host time, so `value` comes from the pass above
    torch.cuda.nvtx.range_push("profiled")
    t_prof, _, _, _, kern = timed(pm, Ud, bd, args.steps, 1, kernel_events=True)
    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("fp64")
    t_fp64, info_64, _, _, _ = timed(p64, Ud, bd, max(1, min(args.steps, 2)), 1)
    torch.cuda.nvtx.range_pop()
    # the same steps with the post-smoother on the full system
    t_plain, info_plain, _, _, _ = timed(make_params(True, False), Ud, bd, args.steps, 1)
    t_plain64, info_plain64, _, _, _ = timed(make_params(False, False), Ud, bd,
                                             max(1, min(args.steps, 2)), 1)

    # end to end through the C ABI with host buffers (links, b on the host; x back to host)
    Uh = torch.from_numpy(U).pin_memory()
    bh = torch.from_numpy(b).pin_memory()
    e2e = []
    for i in range(args.steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xh, _ = step(pm, Uh, bh)
        torch.cuda.synchronize()
        if i > 0:
            e2e.append(time.perf_counter() - t0)

    # Dslash roofline: FP32 full operator on the workload lattice, L2 flushed between launches
    nd = 20
    psi = torch.from_numpy(synthetic.gaussian_rhs(dims, 7)).to(torch.complex64).to(dev)
    U32 = Ud.to(torch.complex64)
    out = torch.empty_like(psi)
    ev = []
    for i in range(nd + 3):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        api.dslash(psi, U32, dims, cfg["kappa"], out=out)
        e1.record()
        torch.cuda.synchronize()
        if i >= 3:
            ev.append(e0.elapsed_time(e1) / 1e3)
    t_d = float(np.mean(ev))
    bytes_d = V * 480.0   # 24 reals in + 24 out + 72 link reals per site, FP32
    peaks, peak_kind = load_peaks()
    gbs = bytes_d / t_d / 1e9

    kernels, roof = kernel_table(kern, alu, peaks, peak_kind)
    if roof is None:
        roof = {"kernel": "dslash_c64 (16^3x32, L2 flushed)", "bound": "hbm", "achieved": gbs,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                "peak_source": peak_kind, "traffic": None, "avg_launch_us": t_d * 1e6,
                "algorithmic_bytes_per_launch": bytes_d}

    # The comparison of Table 2 on the synthetic near-critical lattice: fine-level outer
    # iterations of Regular (k test vectors, one stream) and iCSVD (streams of r = 8, n_s = 4
    # and 8), together with the setup + solve seconds of the mixed and the plain FP64 form on
    # the same configuration, at the timed smoothing (5 GMRES steps per test vector) and at 20,
    # on two levels and on four (level 2: 2^4 aggregates of the level-1 lattice, k = 16;
    # level 3: the rest, k = 16; level tolerances 0.03 / 0.06 / 0.6 as at the critical mass in
    # Sec. 4.5).
    def timed_once(p, levels=()):
        step(p, Ud, bd, levels)            # warm-up (autotuner, allocation cache)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, inf = step(p, Ud, bd, levels)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, inf

    fine = {}
    lc = [dims[m] // cfg["block"][m] for m in range(4)]
    depths = (2, 4) if args.extras else ()
    def four(reg):
        return (((2, 2, 2, 2), 16, 16 if reg else 8, 1 if reg else 4, 0.06),
                ((lc[0] // 2, lc[1] // 2, lc[2] // 2, lc[3] // 2), 16, 16 if reg else 8,
                 1 if reg else 4, 0.6))
    for depth in depths:
        for sw in (cfg["sweeps"], 20):
            row = {}
            for tag, r, ns in (("regular_ns1", cfg["k"], 1), ("icsvd_ns4", cfg["r"], 4),
                               ("icsvd_ns8", cfg["r"], 8)):
                levels = four(tag == "regular_ns1") if depth == 4 else ()
                ent = {"test_vectors": r * ns}
                for form, sd in (("fp64", "c128"), ("mixed", "c64")):
                    pf = api.params(dims, cfg["block"], cfg["kappa"], cfg["k"], r, ns, sw,
                                    cfg["tv_seed"], cfg["hop_weight"], cfg["bc"], setup_dtype=sd,
                                    solve_dtype=sd)
                    t, inf = timed_once(pf, levels)
                    ent[form] = {"seconds": t, "outer": inf["outer"], "coarse": inf["coarse"]}
                    if "level_iterations" in inf:
                        ent[form]["level_iterations"] = inf["level_iterations"]
                ent["mixed_over_fp64_speedup"] = ent["fp64"]["seconds"] / ent["mixed"]["seconds"]
                row[tag] = ent
            for t in ("icsvd_ns4", "icsvd_ns8"):
                row["reduction_regular_over_" + t] = (row["regular_ns1"]["fp64"]["outer"]
                                                      / max(row[t]["fp64"]["outer"], 1))
            fine["levels_%d_sweeps_%d" % (depth, sw)] = row

    # the next rows on the timed workload: the Schur-form post-smoother (even-odd
    # preconditioning, Sec. 1), the Wilson-clover operator (c_sw = 1.7, at kappa = 0.125 since
    # the clover term moves the critical point) and the Eq. 9 prolongator (one stream of 32
    # test vectors, weights 10^(-i/31)): setup + Galerkin + solve seconds and iterations,
    # mixed and FP64
    variants = {}
    if args.extras:
        m32 = cfg["r"] * cfg["n_s"]
        omega = [10.0 ** (-i / (m32 - 1)) for i in range(m32)]
        for tag, extra, kap in (("schur_smoother", dict(schur_smoother=1), cfg["kappa"]),
                                ("clover_csw1.7", dict(csw=1.7), 0.125),
                                ("wilson_kappa0.125", {}, 0.125),
                                ("ls_interpolation", dict(n_s=1, r=m32), cfg["kappa"])):
            ent = {}
            for form, sd in (("fp64", "c128"), ("mixed", "c64")):
                args_p = dict(dims=dims, block=cfg["block"], kappa=kap, k=cfg["k"], r=cfg["r"],
                              n_s=cfg["n_s"], sweeps=cfg["sweeps"], seed=cfg["tv_seed"],
                              hop_weight=cfg["hop_weight"], bc=cfg["bc"], setup_dtype=sd,
                              solve_dtype=sd)
                args_p.update(extra)
                pv = api.params(**args_p)
                ls = omega if tag == "ls_interpolation" else None

                def run_v():
                    h = api.Hierarchy(Ud, pv, ls_omega=ls)
                    h.coarse_build()
                    x, inf = h.solve(bd, tol=1e-10, maxiter=4000)
                    h.close()
                    return inf
                run_v()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                inf = run_v()
                e1.record()
                torch.cuda.synchronize()
                ent[form] = {"seconds": e0.elapsed_time(e1) / 1e3, "outer": inf["outer"],
                             "coarse": inf["coarse"], "residual": inf["residual"]}
            variants[tag] = ent

    # anisotropic 16^3 x 64 (w_t = 1/3.5): FP16 and BF16 smoother storage vs plain FP64
    aniso = anisotropic_leg(api, synthetic, dev, step) if args.aniso else None

    d32 = dslash_32(api, synthetic, dev, flush, peaks, peak_kind) if args.extras else None

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": t_mixed,
            "solves_per_s_all_ranks": world / t_mixed,
            "unit": "s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_mixed * 1e3,
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "c64+f64",
            "data": "synthetic",
            "config": bench_config(cfg, world),
            "fp64_seconds": t_fp64,
            "mixed_over_fp64_speedup": t_fp64 / t_mixed,
            "full_system_smoother": {"mixed_seconds": t_plain, "fp64_seconds": t_plain64,
                                     "solve_info_mixed": info_plain,
                                     "solve_info_fp64": info_plain64},
            "profiled_step_seconds": t_prof,
            "solve_info_mixed": info_m,
            "solve_info_fp64": info_64,
            "dslash_fp32_gbs": gbs,
            "e2e": {"value": float(np.mean(e2e)), "unit": "s",
                    "h2d_bytes_per_step": int(U.nbytes + b.nbytes),
                    "d2h_bytes_per_step": int(b.nbytes)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": roof,
            "kernels": kernels,
            "alu_peaks_tflops": alu,
            "autotune": json.loads(_lib.lib().mg_autotune_report().decode()),
            "fine_iterations": fine,
            "next_rows_16^3x32": variants,
            "anisotropic_16^3x64": aniso,
            "dslash_roofline_32^3x64": d32,
            "dslash_roofline": {"kernel": "dslash_c64 (16^3x32, L2 flushed, standalone)",
                                "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                                "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                                "avg_launch_us": t_d * 1e6, "algorithmic_bytes": bytes_d},
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg, U, b, info_64["outer"])[0]
            line["cpu_baseline"]["full_steps_small"] = small_full_steps(api, synthetic, dev, step)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def host_info():
    """CPU model and the cores this process may run on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part"):
                    model = line.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    import platform
    return {"cpu": model or platform.processor() or platform.machine(),
            "arch": platform.machine(), "available_cores": len(os.sched_getaffinity(0))}


FULL_STEP_RECORD = os.path.join(ROOT, "oracle", "records",
                                "full_step_c2_16x16x16x32%s.json" % ("_schur" if SCHUR_SMOOTHER else ""))


def oracle_outer_iterations(cfg, fallback):
    """Outer FGMRES iterations of the oracle's own full step on this workload (written by the
    oracle's full-step script), else `fallback` (the FP64 GPU solve of the same run, whose
    iteration counts the parity tests hold equal to the oracle's within one)."""
    try:
        with open(FULL_STEP_RECORD) as f:
            rec = json.load(f)
        if (rec.get("workload") == WORKLOAD and abs(rec["kappa"] - cfg["kappa"]) < 1e-12
                and bool(rec.get("schur_smoother", False)) == SCHUR_SMOOTHER):
            return int(rec["info"]["outer"]), "oracle full step (recorded)", rec
    except Exception:
        pass
    return int(fallback), "FP64 GPU solve of this run", None


def cpu_baseline(cfg, U, b, outer_fallback):
    """The FP64 oracle, as it stands, timed on the host cores on a bounded sample of one step.

    The sample runs every part of the step with the oracle's own functions (test vectors,
    streaming SVD over all aggregates, Galerkin product, K-cycle FGMRES iteration), units the
    method treats independently spread over one process per available core; each part's time
    is scaled by its share of one whole step (oracle.full_step.SampledStep).
    """
    from oracle import full_step
    workers = len(os.sched_getaffinity(0))
    outer, src, rec = oracle_outer_iterations(cfg, outer_fallback)
    s = full_step.SampledStep(U, b[0], cfg, cfg["kappa"], workers, outer, schur=SCHUR_SMOOTHER)
    t0 = time.perf_counter()
    s.run_all()
    out = {"value": s.estimate(), "unit": "s", "cores": workers, "kind": "oracle",
           "sample": s.describe() + "; outer iterations from the " + src,
           "sample_wall_s": time.perf_counter() - t0, "host": host_info(),
           "parts_run_s": dict(s.run_s), "parts_scaled_s": dict(s.scaled_s)}
    if rec:
        out["recorded_full_step"] = {"seconds": rec["seconds"], "workers": rec["workers"],
                                     "host_cores": rec["host_cores"], "info": rec["info"],
                                     "parts_s": rec["parts_s"]}
    return out, s


def small_full_steps(api, synthetic, dev, step):
    """The two small workloads (4^4 and 8^4) end to end on both sides: the GPU's mixed step
    (setup + Galerkin + solve, the timed configuration's smoother) and the FP64 oracle's whole
    step (oracle.full_step, one process per available core), each with its own iteration
    counts."""
    import torch
    from oracle import full_step
    workers = len(os.sched_getaffinity(0))
    out = {"cores": workers}
    for name in ("c1_4^4_haar", "c5_8^4_autograd"):
        c = dict(synthetic.WORKLOADS[name])
        c["kappa"] = synthetic.kappa_of(c)
        Uc = synthetic.make_links(c)
        bc_ = synthetic.gaussian_rhs(c["dims"], c["rhs_seed"])
        p = api.params(c["dims"], c["block"], c["kappa"], c["k"], c["r"], c["n_s"], c["sweeps"],
                       c["tv_seed"], c["hop_weight"], c["bc"], setup_dtype="c64",
                       solve_dtype="c64", schur_smoother=int(SCHUR_SMOOTHER))
        Ud = torch.from_numpy(Uc).to(dev)
        bd = torch.from_numpy(bc_).to(dev)
        step(p, Ud, bd)   # warm-up
        ts = []
        for _ in range(5):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = step(p, Ud, bd)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        info_o, parts = full_step.full_step(Uc, bc_[0], c, c["kappa"], workers,
                                            schur=SCHUR_SMOOTHER)
        t_o = float(sum(parts.values()))
        out[name] = {"gpu_mixed_seconds": float(np.median(ts)), "gpu_outer": info["outer"],
                     "oracle_seconds": t_o, "oracle_parts_s": parts,
                     "oracle_outer": info_o["outer"],
                     "oracle_over_gpu": t_o / float(np.median(ts))}
    return out


def reference_arm(args):
    """The oracle as the reference arm.  The warm-up measures every part of one sampled step
    (oracle.full_step.SampledStep); each timed step then re-measures one part, in turn, and
    reports the estimate of one whole step from the latest measurement of every part:
    `value` is that estimate in seconds, `ms_per_step` the wall time a timed step took."""
    rank, world, local = _dist()
    if rank != 0:
        return
    from paper_2505_14399_gb300 import synthetic
    cfg = workload()
    U = synthetic.make_links(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    r, s = cpu_baseline(cfg, U, b, outer_fallback=15 if SCHUR_SMOOTHER else 30)
    vals, walls = [], []
    for i in range(args.steps):
        part = s.PARTS[i % len(s.PARTS)]
        t0 = time.perf_counter()
        s.run(part)
        walls.append(time.perf_counter() - t0)
        vals.append(s.estimate())
    v = float(np.mean(vals)) if vals else r["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(walls)) * 1e3 if walls else None,
            "ms_per_step_meaning": "wall time of one timed step (one part of the sampled step "
                                   "re-measured); value is the estimate of one whole step",
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(cfg, world),
            "cpu_baseline": {"value": v, "unit": "s", "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"], "host": r["host"],
                             "warmup_sample_wall_s": r["sample_wall_s"],
                             "parts_scaled_s": dict(s.scaled_s),
                             "recorded_full_step": r.get("recorded_full_step")},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-aniso", dest="aniso", action="store_false",
                    help="skip the anisotropic 16^3 x 64 half-storage leg")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the legs outside the timed step (Regular vs iCSVD iterations, "
                         "32^3 x 64 stencil)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
