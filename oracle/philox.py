"""Counter-based Gaussian probe for the Monte-Carlo divergence (Eq. MC_SURE).

Section 4.3 estimates the denoiser divergence with one Gaussian probe
b ~ N(0, I) per iteration (K = 1).  So that the oracle and the CUDA library
draw the same probe without passing it between them, each side implements,
separately, the Philox4x32-10 generator of Salmon, Moraes, Dror and Shaw
("Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller
transform:

* multipliers 0xD2511F53 and 0xCD9E8D57, Weyl key increments 0x9E3779B9 and
  0xBB67AE85, ten rounds; one round maps counter (c0, c1, c2, c3) and key
  (k0, k1) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
  the key is bumped between rounds;
* probe element i of iteration t for slice ``slice`` and seed ``seed`` comes
  from block counter (i // 4, t, slice, 0) with key (seed mod 2^32,
  seed // 2^32), output word i % 4;
* a word x becomes the uniform u = (x + 0.5) / 2^32 in (0, 1); words (0, 1)
  and (2, 3) of a block form Box-Muller pairs:
  r = sqrt(-2 ln u_a), n_a = r cos(2 pi u_b), n_b = r sin(2 pi u_b).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint32 arrays; returns four uint32 arrays."""
    c = [np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [(hi1 ^ c[1] ^ k0) & MASK, lo1, (hi0 ^ c[3] ^ k1) & MASK, lo0]
        if rnd < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return [v.astype(np.uint32) for v in c]


def probe_words(n: int, seed: int, t: int, slice_id: int) -> np.ndarray:
    """The first ``n`` raw 32-bit words of the probe stream."""
    nb = (n + 3) // 4
    g = np.arange(nb, dtype=np.uint64)
    out = philox4x32_10(g, np.full(nb, t), np.full(nb, slice_id), np.zeros(nb),
                        seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return np.stack(out, axis=1).reshape(-1)[:n]


def probe_normals(n: int, seed: int, t: int, slice_id: int) -> np.ndarray:
    """b ~ N(0, I) of length n (fp64) for iteration t."""
    nb = (n + 3) // 4
    words = probe_words(4 * nb, seed, t, slice_id).reshape(nb, 4).astype(np.float64)
    u = (words + 0.5) / 4294967296.0
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    a01 = 2.0 * np.pi * u[:, 1]
    a23 = 2.0 * np.pi * u[:, 3]
    out = np.stack([r01 * np.cos(a01), r01 * np.sin(a01),
                    r23 * np.cos(a23), r23 * np.sin(a23)], axis=1)
    return out.reshape(-1)[:n]
