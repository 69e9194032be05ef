"""One whole step of the two-level method run by this oracle, timed (test infrastructure only).

A step is what the GPU library's benchmark times: the test vectors of Eq. 2 for every
stream, the streaming chiral SVD of Algorithm 3 over all aggregates, the Galerkin product
of Eq. 5, and the K-cycle preconditioned FGMRES solve of D x = b (Sec. 2.1 end, Sec. 4) to a
relative residual of 1e-10.  Nothing here is new arithmetic: every part calls the oracle's
own functions (``icsvd.test_vectors``, ``icsvd.chiral_split``, ``icsvd.icsvd_tiles``,
``coarse.galerkin``, ``mg.TwoLevel``) unchanged.

Host cores: units of work that the method treats independently -- one test vector, one
aggregate's tiles, one coarse time slab of the Galerkin sum -- may be handed to a pool of
worker processes (``spawn``: no state is inherited from the caller), each running the same
oracle function on its own unit.  The sequential FGMRES iteration runs in one process.

Two uses:
* ``full_step``: the whole step, with the oracle's own iteration counts (minutes at
  16^3 x 32).  ``python -m oracle.full_step <workload> [workers] [out.json]``.
* ``sampled_step``: a bounded piece of every part, timed, each scaled by its share of the
  whole step (the number of test vectors, aggregates and coarse slabs; the outer iteration
  count of a recorded full step), giving the estimated seconds of one whole step.
"""
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

from . import coarse, icsvd, mg

_W = {}


def _init(links):
    _W["links"] = links


def _one_vector(args):
    dims, kappa, w, bc, seed, vid, sweeps = args
    t0 = time.perf_counter()
    v = icsvd.test_vectors(_W["links"], dims, kappa, w, bc, seed, 1, vid, sweeps)[0]
    return vid, v, time.perf_counter() - t0


def _svd_chunk(args):
    tiles, k = args
    t0 = time.perf_counter()
    Pt, S, hist = icsvd.icsvd_tiles(tiles, k)
    return Pt, S, time.perf_counter() - t0


_BLAS_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def _pool(workers, links):
    """`workers` single-threaded processes (one per core: their BLAS calls stay on one thread,
    so the pool does not oversubscribe the cores)."""
    saved = {v: os.environ.get(v) for v in _BLAS_VARS}
    for v in _BLAS_VARS:
        os.environ[v] = "1"
    try:
        return mp.get_context("spawn").Pool(workers, initializer=_init, initargs=(links,))
    finally:
        for v, x in saved.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x


def _vectors(pool, cfg, kappa, ids):
    args = [(cfg["dims"], kappa, cfg["hop_weight"], cfg["bc"], cfg["tv_seed"], int(i),
             cfg["sweeps"]) for i in ids]
    out = dict((vid, (v, t)) for vid, v, t in pool.map(_one_vector, args, chunksize=1))
    return np.stack([out[int(i)][0] for i in ids]), [out[int(i)][1] for i in ids]


def _icsvd(pool, stream_tiles, k, workers):
    d = stream_tiles[0].shape[0]
    cuts = np.linspace(0, d, min(workers, d) + 1).astype(int)
    chunks = [([t[a:b] for t in stream_tiles], k) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    res = pool.map(_svd_chunk, chunks, chunksize=1)
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])


def full_step(links, b, cfg, kappa, workers=1, tol=1e-10, log=None):
    """The whole step on `workers` processes.  Returns the solve info, per-part seconds."""
    dims, block, k, r, n_s = cfg["dims"], cfg["block"], cfg["k"], cfg["r"], cfg["n_s"]
    w, bc = cfg["hop_weight"], cfg["bc"]
    parts = {}
    with _pool(workers, links) as pool:
        t0 = time.perf_counter()
        tiles = []
        for s in range(n_s):
            vecs, _ = _vectors(pool, cfg, kappa, range(s * r, (s + 1) * r))
            tiles.append(icsvd.chiral_split(vecs, dims, block))
        parts["test_vectors"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        Pt, _ = _icsvd(pool, tiles, k, workers)
        parts["icsvd"] = time.perf_counter() - t0
    if log:
        log("setup %.1f s" % (parts["test_vectors"] + parts["icsvd"]))
    t0 = time.perf_counter()
    XY = coarse.galerkin(Pt, links, dims, block, kappa, w, bc)
    parts["galerkin"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    lvl = mg.TwoLevel(links, dims, kappa, w, bc, block, Pt, XY=XY)
    _, info = lvl.solve(np.asarray(b).reshape(-1), tol=tol, maxiter=4000)
    parts["solve"] = time.perf_counter() - t0
    info = dict(info, kcycles=lvl.kcycles)
    return info, parts


def sampled_step(links, b, cfg, kappa, workers, outer_its, n_outer=1):
    """A bounded sample of every part of the step, scaled to one whole step.

    * test vectors: `workers` of the r n_s vectors smoothed at full volume, one per process,
      scaled by ceil(r n_s / workers) rounds;
    * streaming SVD: every aggregate and stream, on the sampled vectors (the stream tiles are
      the sampled vectors taken r at a time, cycled when fewer than r n_s were smoothed);
    * Galerkin product: the full lattice (one process);
    * solve: `n_outer` FGMRES iterations of the K-cycle-preconditioned solve on the sampled
      prolongator, scaled by `outer_its` (the outer iterations of a recorded full step).
    Returns (estimated seconds of one step, per-part seconds as run, description).
    """
    dims, block, k, r, n_s = cfg["dims"], cfg["block"], cfg["k"], cfg["r"], cfg["n_s"]
    w, bc = cfg["hop_weight"], cfg["bc"]
    m = r * n_s
    nv = max(1, min(workers, m))
    run = {}
    with _pool(workers, links) as pool:
        t0 = time.perf_counter()
        vecs, _ = _vectors(pool, cfg, kappa, range(nv))
        run["test_vectors"] = time.perf_counter() - t0
        tiles = []
        for s in range(n_s):
            idx = [(s * r + i) % nv for i in range(r)]
            tiles.append(icsvd.chiral_split(vecs[idx], dims, block))
        t0 = time.perf_counter()
        Pt, _ = _icsvd(pool, tiles, k, workers)
        run["icsvd"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    XY = coarse.galerkin(Pt, links, dims, block, kappa, w, bc)
    run["galerkin"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    lvl = mg.TwoLevel(links, dims, kappa, w, bc, block, Pt, XY=XY)
    lvl.solve(np.asarray(b).reshape(-1), tol=1e-30, maxiter=n_outer)
    run["solve"] = time.perf_counter() - t0
    scaled = {"test_vectors": run["test_vectors"] * math.ceil(m / nv),
              "icsvd": run["icsvd"], "galerkin": run["galerkin"],
              "solve": run["solve"] * outer_its / n_outer}
    desc = ("%d of %d test vectors smoothed at full volume (one per process, scaled by %d "
            "rounds); streaming SVD of all %d aggregates; full Galerkin product; %d of %d "
            "outer FGMRES iterations (scaled)" % (nv, m, math.ceil(m / nv),
                                                   int(np.prod(dims)) // int(np.prod(block)),
                                                   n_outer, outer_its))
    return sum(scaled.values()), run, scaled, desc


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2505_14399_gb300 import synthetic
    name = sys.argv[1]
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else 1
    out = sys.argv[3] if len(sys.argv) > 3 else None
    cfg = synthetic.WORKLOADS[name]
    kappa = synthetic.kappa_of(name)
    U = synthetic.make_links(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])[0]
    t0 = time.perf_counter()
    info, parts = full_step(U, b, cfg, kappa, workers, log=lambda s: print(s, flush=True))
    rec = {"workload": name, "kappa": kappa, "workers": workers,
           "seconds": time.perf_counter() - t0, "parts_s": parts, "info": info,
           "host_cores": len(os.sched_getaffinity(0))}
    print(json.dumps(rec), flush=True)
    if out:
        with open(out, "w") as f:
            json.dump(rec, f, indent=1)
