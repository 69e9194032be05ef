"""Philox4x32-10 and the complex-Gaussian map, FP64 oracle (test infrastructure only).

The random initial guesses phi_i of Eq. (2) (Sec. 2.1; Algorithm 3, first inner loop)
are drawn from a counter-based generator so that the GPU library and this oracle can
produce the same numbers independently.  The paper does not fix a distribution; the
library documents complex Gaussian entries (real and imaginary parts N(0, 1)).

Philox4x32-10 follows its published definition (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
a 4 x 32-bit counter and a 2 x 32-bit key; each of 10 rounds multiplies counter
words 0 and 2 by fixed odd constants, splits the 64-bit products into hi/lo halves,
and permutes/xors them with the key; the key is bumped by the Weyl constants
between rounds.

Gaussian map (library convention): for test vector v (global index over streams),
site s and component c = 3*spin + colour, counter = (s, c, v, 0) and
key = (seed mod 2^32, seed >> 32).  The four output words give two 53-bit uniforms
u_a = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53 and u_b likewise from (w2, w3); then
Box-Muller: rho = sqrt(-2 ln(1 - u_a)), Re = rho cos(2 pi u_b), Im = rho sin(2 pi u_b).
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10. ctr: (..., 4) uint, key: (2,) ints. Returns (..., 4) uint64."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.uint64(int(key[0]) & MASK)
    k1 = np.uint64(int(key[1]) & MASK)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    mask = np.uint64(MASK)
    s32 = np.uint64(32)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + W0) & MASK)
            k1 = np.uint64((int(k1) + W1) & MASK)
        p0 = m0 * c[0]          # < 2^64: exact in uint64
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def gaussian_field(seed, vec_ids, nsites, ncomp, word3=0):
    """Complex Gaussian fields, shape (len(vec_ids), nsites, ncomp), complex128.

    Counter (site, component, vector id, word3), key (seed mod 2^32, seed >> 32), then the
    53-bit uniforms and Box-Muller of the module header.  word3 = 0 for the fine-level
    spinors; a coarse level of the hierarchy uses its level index, so its fields are
    independent of the fine ones drawn with the same seed and vector ids.
    """
    vec_ids = np.asarray(vec_ids, dtype=np.uint64)
    nv = len(vec_ids)
    s = np.arange(nsites, dtype=np.uint64)
    c = np.arange(ncomp, dtype=np.uint64)
    ctr = np.zeros((nv, nsites, ncomp, 4), dtype=np.uint64)
    ctr[..., 0] = s[None, :, None]
    ctr[..., 1] = c[None, None, :]
    ctr[..., 2] = vec_ids[:, None, None]
    ctr[..., 3] = np.uint64(word3)
    key = (seed & MASK, (seed >> 32) & MASK)
    w = philox4x32_10(ctr, key)
    two26 = np.float64(67108864.0)
    scale = np.float64(2.0 ** -53)
    ua = ((w[..., 0] >> np.uint64(5)).astype(np.float64) * two26
          + (w[..., 1] >> np.uint64(6)).astype(np.float64)) * scale
    ub = ((w[..., 2] >> np.uint64(5)).astype(np.float64) * two26
          + (w[..., 3] >> np.uint64(6)).astype(np.float64)) * scale
    rho = np.sqrt(-2.0 * np.log(1.0 - ua))
    th = 2.0 * np.pi * ub
    return rho * np.cos(th) + 1j * (rho * np.sin(th))


def gaussian_vectors(seed, vec_ids, volume):
    """Complex Gaussian spinor fields, shape (len(vec_ids), volume, 4, 3), complex128
    (component c = 3 * spin + colour, counter word 3 = 0)."""
    return gaussian_field(seed, vec_ids, volume, 12, 0).reshape(len(vec_ids), volume, 4, 3)
