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
  16^3 x 32).  ``python -m oracle.full_step <workload> [workers] [out.json] [schur]``
  (``schur``: the Schur-form post-smoother).
* ``SampledStep``: a bounded piece of every part, timed, each scaled by its share of the
  whole step (the number of test vectors and coarse slabs; the outer iteration count of a
  recorded full step), giving the estimated seconds of one whole step.
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


def full_step(links, b, cfg, kappa, workers=1, tol=1e-10, log=None, schur=False):
    """The whole step on `workers` processes (schur: the K-cycle's post-smoother on the
    even-odd Schur system).  Returns the solve info, per-part seconds."""
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
    lvl = mg.TwoLevel(links, dims, kappa, w, bc, block, Pt, XY=XY, schur=schur)
    _, info = lvl.solve(np.asarray(b).reshape(-1), tol=tol, maxiter=4000)
    parts["solve"] = time.perf_counter() - t0
    info = dict(info, kcycles=lvl.kcycles)
    return info, parts


class SampledStep:
    """A bounded sample of every part of the step, each part timed and scaled to its share of
    one whole step on `workers` host cores:

    * ``vectors``: `workers` of the r n_s test vectors smoothed at full volume (Eq. 2), one per
      process; scaled by ceil(r n_s / workers) rounds;
    * ``svd``: the streaming SVD of all aggregates and streams (Algorithm 3) on the sampled
      vectors (stream tiles take them r at a time, cycled), aggregates spread over the pool;
    * ``galerkin``: the Galerkin product (Eq. 5) of one coarse time slab, computed as a
      periodic lattice of that slab's extent (the same work per site as the whole lattice);
      scaled by ceil(slabs / workers), the slabs being independent units;
    * ``solve``: one outer FGMRES iteration of the K-cycle preconditioned solve on the full
      lattice with the sampled prolongator (its coarse operator: the slab's, repeated over the
      slabs); scaled by `outer_its`, the outer iterations of a recorded full step.

    `run(part)` measures one part; `estimate()` sums the latest scaled measurement of every
    part (None until each part has been measured once).
    """
    PARTS = ("vectors", "svd", "galerkin", "solve")

    def __init__(self, links, b, cfg, kappa, workers, outer_its, schur=False):
        self.links, self.b, self.cfg, self.kappa = links, np.asarray(b).reshape(-1), cfg, kappa
        self.workers, self.outer_its, self.schur = workers, outer_its, schur
        dims, block = cfg["dims"], cfg["block"]
        self.m = cfg["r"] * cfg["n_s"]
        self.nv = max(1, min(workers, self.m))
        self.nslab = dims[3] // block[3]
        self.run_s, self.scaled_s = {}, {}
        self.vecs = self.Pt = self.XY = None

    def _slab(self):
        dims, block = self.cfg["dims"], self.cfg["block"]
        sub = (dims[0], dims[1], dims[2], block[3])
        vs = int(np.prod(sub))
        nb = vs // int(np.prod(block))
        return sub, np.ascontiguousarray(self.links[:, :vs]), nb

    def run(self, part, pool=None):
        cfg, dims, block, k, r = (self.cfg, self.cfg["dims"], self.cfg["block"], self.cfg["k"],
                                  self.cfg["r"])
        w, bc = cfg["hop_weight"], cfg["bc"]
        own = pool is None and part in ("vectors", "svd")
        if own:
            pool = _pool(self.workers, self.links)
        try:
            t0 = time.perf_counter()
            if part == "vectors":
                self.vecs, _ = _vectors(pool, cfg, self.kappa, range(self.nv))
                t = time.perf_counter() - t0
                scaled = t * math.ceil(self.m / self.nv)
            elif part == "svd":
                tiles = []
                for s in range(cfg["n_s"]):
                    idx = [(s * r + i) % self.nv for i in range(r)]
                    tiles.append(icsvd.chiral_split(self.vecs[idx], dims, block))
                t0 = time.perf_counter()
                self.Pt, _ = _icsvd(pool, tiles, k, self.workers)
                t = scaled = time.perf_counter() - t0
            elif part == "galerkin":
                sub, Ls, nb = self._slab()
                X, Y = coarse.galerkin(self.Pt[:nb], Ls, sub, block, self.kappa, w, bc)
                t = time.perf_counter() - t0
                scaled = t * math.ceil(self.nslab / self.workers)
                self.XY = (np.concatenate([X] * self.nslab, axis=0),
                           np.concatenate([Y] * self.nslab, axis=1))
            else:
                lvl = mg.TwoLevel(self.links, dims, self.kappa, w, bc, block, self.Pt, XY=self.XY,
                                  schur=self.schur)
                t0 = time.perf_counter()
                lvl.solve(self.b, tol=1e-30, maxiter=1)
                t = time.perf_counter() - t0
                scaled = t * self.outer_its
        finally:
            if own:
                pool.close()
                pool.join()
        self.run_s[part], self.scaled_s[part] = t, scaled
        return t

    def run_all(self):
        with _pool(self.workers, self.links) as pool:
            self.run("vectors", pool)
            self.run("svd", pool)
        self.run("galerkin")
        self.run("solve")

    def estimate(self):
        if any(p not in self.scaled_s for p in self.PARTS):
            return None
        return sum(self.scaled_s.values())

    def describe(self):
        dims, block = self.cfg["dims"], self.cfg["block"]
        return ("%d of %d test vectors smoothed at full volume on %d processes (x%d rounds); "
                "streaming SVD of all %d aggregates; Galerkin product of 1 of %d coarse time "
                "slabs (x%d); 1 outer FGMRES iteration (x%d)"
                % (self.nv, self.m, self.workers, math.ceil(self.m / self.nv),
                   int(np.prod(dims)) // int(np.prod(block)), self.nslab,
                   math.ceil(self.nslab / self.workers), self.outer_its))


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2505_14399_gb300 import synthetic
    name = sys.argv[1]
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else 1
    out = sys.argv[3] if len(sys.argv) > 3 else None
    schur = len(sys.argv) > 4 and sys.argv[4] == "schur"
    cfg = synthetic.WORKLOADS[name]
    kappa = synthetic.kappa_of(name)
    U = synthetic.make_links(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])[0]
    t0 = time.perf_counter()
    info, parts = full_step(U, b, cfg, kappa, workers, log=lambda s: print(s, flush=True),
                            schur=schur)
    rec = {"workload": name, "kappa": kappa, "workers": workers, "schur_smoother": schur,
           "seconds": time.perf_counter() - t0, "parts_s": parts, "info": info,
           "host_cores": len(os.sched_getaffinity(0))}
    print(json.dumps(rec), flush=True)
    if out:
        with open(out, "w") as f:
            json.dump(rec, f, indent=1)
