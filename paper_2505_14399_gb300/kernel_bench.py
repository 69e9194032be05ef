"""Per-kernel microbenchmarks (CUDA-event timing; also the driver for ncu captures).

    python -m paper_2505_14399_gb300.kernel_bench dslash --dims 24 24 24 48 --dtype c64
    python -m paper_2505_14399_gb300.kernel_bench step --workload c2_16^3x32_near_critical
    python -m paper_2505_14399_gb300.kernel_bench coarse --workload c2_16^3x32_near_critical
    python -m paper_2505_14399_gb300.kernel_bench scan --sweeps 20

Inputs come from the seeded generators in ``synthetic``; L2 is flushed (a 256 MB write and
a 256 MB read, leaving clean lines) before every timed launch.  Prints one JSON line per measurement.
"""
import argparse
import json

import numpy as np
import torch

from . import api, synthetic

BYTES_PER_SITE = {"c128": 960.0, "c64": 480.0, "f16": 240.0, "bf16": 240.0}
TORCH_DT = {"c128": torch.complex128, "c64": torch.complex64, "f16": torch.float16,
            "bf16": torch.bfloat16}


def _field(x, dt, dev):
    if dt in ("c128", "c64"):
        return torch.from_numpy(x).to(TORCH_DT[dt]).to(dev)
    return torch.from_numpy(np.stack([x.real, x.imag], axis=-1)).to(TORCH_DT[dt]).to(dev)


class L2Flush:
    """Evicts L2 between timed launches: writes a 256 MB buffer (larger than the 129 MB L2)
    and then reads a second 256 MB buffer, so the lines left in L2 are clean and the next
    kernel is not charged for writing the flush data back to HBM."""

    def __init__(self, dev):
        n = 256 * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device=dev)
        self.r = torch.ones(n, dtype=torch.float32, device=dev)
        self.s = torch.empty((), dtype=torch.float32, device=dev)

    def zero_(self):
        self.w.zero_()
        torch.sum(self.r, dim=0, out=self.s)


def _timeit(fn, reps, flush):
    ts = []
    for i in range(reps + 2):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            ts.append(e0.elapsed_time(e1) / 1e3)
    return float(np.mean(ts)), float(np.min(ts))


def bench_dslash(a, dev, flush):
    dims = tuple(a.dims)
    V = int(np.prod(dims))
    U = synthetic.smooth_links(dims, 1)
    psi = synthetic.gaussian_rhs(dims, 2, a.nrhs)
    if a.parity >= 0:
        psi = psi[:, : V // 2]
    pt = _field(np.ascontiguousarray(psi), a.dtype, dev)
    out = torch.empty_like(pt)
    if a.layout == "lanes":
        # the solver's stencil: the hierarchy's lane-contiguous link copy
        if a.parity >= 0 or a.dtype not in ("c128", "c64"):
            raise SystemExit("lane-contiguous links: full operator, c128/c64 only")
        p = api.params(dims, (2, 2, 2, 2), 0.12, 4, 4, 1)
        h = api.Hierarchy(torch.from_numpy(U).to(dev), p, setup=False)
        fn = lambda: h.apply_fine(pt, out=out)
    else:
        Ut = _field(U, a.dtype, dev)
        fn = lambda: api.dslash(pt, Ut, dims, 0.12, parity=a.parity, out=out)
    t, tmin = _timeit(fn, a.reps, flush)
    sites = V if a.parity < 0 else V // 2
    eb = BYTES_PER_SITE[a.dtype] / 120.0
    byts = sites * (48 * a.nrhs + 72) * eb if a.parity < 0 else sites * (48 * a.nrhs + 144) * eb
    return {"kernel": "dslash", "layout": a.layout, "dims": dims, "dtype": a.dtype, "nrhs": a.nrhs,
            "parity": a.parity, "us": t * 1e6, "us_min": tmin * 1e6,
            "algorithmic_bytes": byts, "GBps": byts / t / 1e9}


def _workload(name, kappa=None):
    cfg = dict(synthetic.WORKLOADS[name])
    cfg["kappa"] = kappa if kappa is not None else synthetic.kappa_of(cfg)
    return cfg


def _params(cfg, mixed=True):
    return api.params(cfg["dims"], cfg["block"], cfg["kappa"], cfg["k"], cfg["r"], cfg["n_s"],
                      cfg["sweeps"], cfg["tv_seed"], cfg["hop_weight"], cfg["bc"],
                      setup_dtype="c64" if mixed else "c128",
                      solve_dtype="c64" if mixed else "c128")


def bench_step(a, dev, flush):
    cfg = _workload(a.workload, a.kappa)
    U = torch.from_numpy(synthetic.make_links(cfg)).to(dev)
    b = torch.from_numpy(synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])).to(dev)
    p = _params(cfg, not a.fp64)
    out = {}

    def run():
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        h = api.Hierarchy(U, p)
        e[1].record()
        h.coarse_build()
        e[2].record()
        x, info = h.solve(b, tol=1e-10, maxiter=4000)
        e[3].record()
        torch.cuda.synchronize()
        h.close()
        out.update(setup_s=e[0].elapsed_time(e[1]) / 1e3, coarse_s=e[1].elapsed_time(e[2]) / 1e3,
                   solve_s=e[2].elapsed_time(e[3]) / 1e3, info=info)

    for _ in range(a.reps):
        flush.zero_()
        run()
    out.update(kernel="step", workload=a.workload, fp64=a.fp64, kappa=cfg["kappa"])
    return out


def bench_coarse(a, dev, flush):
    cfg = _workload(a.workload, a.kappa)
    U = torch.from_numpy(synthetic.make_links(cfg)).to(dev)
    h = api.Hierarchy(U, _params(cfg))
    t, _ = _timeit(h.coarse_build, a.reps, flush)
    d = h.d
    k = h.k
    vc = torch.randn((1, d, 2, k), dtype=torch.complex64, device=dev)
    tc, _ = _timeit(lambda: h.coarse_apply(vc), a.reps, flush)
    V = h.V
    flops = 8.0 * V * (8 * 6 * (2 * k) ** 2)
    h.close()
    return {"kernel": "coarse", "workload": a.workload, "coarse_build_s": t,
            "galerkin_fp64_tflops": flops / t / 1e12, "coarse_apply_us": tc * 1e6,
            "coarse_apply_GBps": d * 9 * (2 * k) ** 2 * 8 / tc / 1e9}


def bench_scan(a, dev, flush):
    """The paper's parameter studies on the synthetic near-critical lattice (one JSON line
    per point): fine-level FGMRES iterations of the FP64 solve and seconds of the mixed
    setup + solve, against the number of sampled test vectors m = n_s r (streams of r = 8,
    k = 12; Fig. 1 / Table 2), the truncation rank k at m = 64 (Fig. 3), and the smoother
    iterations that make each test vector (Figs. 4-5), each with the Regular setup (k test
    vectors, no truncation) beside it."""
    cfg = _workload(a.workload, a.kappa)
    U = torch.from_numpy(synthetic.make_links(cfg)).to(dev)
    b = torch.from_numpy(synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])).to(dev)

    def point(study, k, r, n_s, sweeps):
        res = {"study": study, "k": k, "r": r, "n_s": n_s, "m": r * n_s, "sweeps": sweeps}
        for tag, mixed in (("fp64", False), ("mixed", True)):
            p = api.params(cfg["dims"], cfg["block"], cfg["kappa"], k, r, n_s, sweeps,
                           cfg["tv_seed"], cfg["hop_weight"], cfg["bc"],
                           setup_dtype="c64" if mixed else "c128",
                           solve_dtype="c64" if mixed else "c128")
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            h = api.Hierarchy(U, p)
            h.coarse_build()
            _, info = h.solve(b, tol=1e-10, maxiter=4000)
            e1.record()
            torch.cuda.synchronize()
            h.close()
            res[tag] = {"outer": info["outer"], "coarse": info["coarse"],
                        "seconds": e0.elapsed_time(e1) / 1e3}
        print(json.dumps(res), flush=True)

    sw = a.sweeps
    for n_s in (2, 4, 8, 12, 16):                         # m = 16 ... 128
        point("m", 12, 8, n_s, sw)
    point("m", 12, 12, 1, sw)                              # Regular
    for k in (8, 12, 16, 24):                              # truncation at m = 64
        point("k", k, 16, 4, sw)
        point("k", k, k, 1, sw)                            # Regular with k vectors
    for s in (2, 5, 10, 20, 30):                           # smoother iterations
        point("sweeps", 12, 8, 4, s)
        point("sweeps", 12, 12, 1, s)
    return {"kernel": "scan", "workload": a.workload, "kappa": cfg["kappa"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["dslash", "step", "coarse", "scan"])
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--dtype", default="c64", choices=list(BYTES_PER_SITE))
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--parity", type=int, default=-1)
    ap.add_argument("--layout", default="abi", choices=["abi", "lanes"],
                    help="links in the ABI layout or the solver's lane-contiguous copy")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--workload", default="c2_16^3x32_near_critical")
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--kappa", type=float, default=None, help="override the workload's kappa")
    ap.add_argument("--sweeps", type=int, default=20,
                    help="scan: smoother iterations per test vector for the m and k studies")
    a = ap.parse_args()
    dev = torch.device("cuda:0")
    flush = L2Flush(dev)
    fn = {"dslash": bench_dslash, "step": bench_step, "coarse": bench_coarse,
          "scan": bench_scan}[a.what]
    print(json.dumps(fn(a, dev, flush)), flush=True)


if __name__ == "__main__":
    main()
