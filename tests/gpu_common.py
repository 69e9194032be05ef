"""Shared helpers of the GPU parity tests (inputs from the seeded generators only)."""
import numpy as np
import torch

from paper_2505_14399_gb300 import api, synthetic

DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).reshape(-1)) / max(np.linalg.norm(b.reshape(-1)), 1e-300))


def to_dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def half_pair(x, dtype):
    """complex numpy -> real torch tensor (..., 2) of dtype on the device."""
    t = torch.from_numpy(np.stack([x.real, x.imag], axis=-1))
    return t.to(dtype).to(DEV)


def from_half_pair(t):
    a = t.float().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def random_tiles(d, nd, k, seed):
    """Seeded complex-Gaussian prolongator tiles (d, 2, k, 6 n_d) -- an input, not an SVD."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((d, 2, k, 6 * nd)) + 1j * rng.standard_normal((d, 2, k, 6 * nd))


def orthonormal_tiles(d, nd, k, seed):
    """Seeded tiles (d, 2, k, 6 n_d) whose k rows are orthonormal (QR of complex Gaussians), so
    every entry has modulus at most 1, as for the iCSVD prolongator -- an input, not an SVD."""
    g = random_tiles(d, nd, k, seed)
    out = np.empty_like(g)
    for j in range(d):
        for a in range(2):
            q, _ = np.linalg.qr(g[j, a].T)
            out[j, a] = q.T
    return out


def params_for(cfg, **kw):
    args = dict(dims=cfg["dims"], block=cfg["block"], kappa=cfg["kappa"], k=cfg["k"], r=cfg["r"],
                n_s=cfg["n_s"], sweeps=cfg["sweeps"], seed=cfg["tv_seed"],
                hop_weight=cfg["hop_weight"], bc=cfg["bc"])
    args.update(kw)
    return api.params(**args)


def links_for(cfg):
    return synthetic.make_links(cfg)


def record(name, **values):
    """Append measured errors and their bounds to the JSON-lines file named by
    WMG_PARITY_LOG (nothing when it is unset)."""
    import json
    import os
    path = os.environ.get("WMG_PARITY_LOG")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps(dict(test=name, **{k: float(v) for k, v in values.items()})) + "\n")
