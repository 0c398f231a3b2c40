"""Counter-based Gaussian draws for the RSVD test matrix Omega (oracle side).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import this module.

The paper draws Omega with i.i.d. N(0,1) entries (Sec. 3.5, step S.1) and names
no generator.  Both the oracle and the CUDA library therefore implement the
same published counter-based generator, each in its own code:

* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a 10-round Feistel-like bijection of a 256-bit counter
  under a 128-bit key.  Each round multiplies two of the four 64-bit words by
  fixed odd constants, keeps the high and low halves of the 128-bit products,
  and mixes the high halves with the other two words and the round key; the
  key is advanced by two Weyl constants between rounds.
* Box-Muller (Box and Muller, 1958) turns each pair of uniforms into a pair of
  independent standard normals.

Element (j, c) of the S x q matrix Omega drawn at update step t has linear
index e = j*q + c.  Block b = e // 4 is produced by one Philox call with
counter (b, t, 0, 0) and key (seed, 0x47524553 "GRES"); word e % 4 of the
block feeds Box-Muller: words (0,1) give normals 0 and 1, words (2,3) give
normals 2 and 3.  A uniform in (0,1] is (x >> 11 + 1) * 2**-53 and one in
[0,1) is (x >> 11) * 2**-53.
"""
import numpy as np

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B
KEY_TAG = 0x47524553  # "GRES"


def philox4x64_10(ctr, key):
    """One Philox4x64-10 block: four 64-bit outputs for a 4-word counter, 2-word key."""
    x0, x1, x2, x3 = (int(v) & MASK64 for v in ctr)
    k0, k1 = (int(v) & MASK64 for v in key)
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


def _u_open0(x):
    return ((x >> 11) + 1) * 2.0 ** -53


def _u_closed0(x):
    return (x >> 11) * 2.0 ** -53


def box_muller(a, b):
    """Two standard normals from two 64-bit words (first word -> radius)."""
    r = np.sqrt(-2.0 * np.log(_u_open0(a)))
    ang = 2.0 * np.pi * _u_closed0(b)
    return r * np.cos(ang), r * np.sin(ang)


def gaussian_block(seed, step, block):
    w = philox4x64_10((block, step, 0, 0), (seed, KEY_TAG))
    z0, z1 = box_muller(w[0], w[1])
    z2, z3 = box_muller(w[2], w[3])
    return (z0, z1, z2, z3)


def gaussian_matrix(seed, step, rows, cols):
    """The rows x cols matrix Omega of step `step` (row-major linear index)."""
    total = rows * cols
    out = np.empty(total, dtype=np.float64)
    nblk = (total + 3) // 4
    for b in range(nblk):
        z = gaussian_block(seed, step, b)
        for t in range(4):
            e = 4 * b + t
            if e < total:
                out[e] = z[t]
    return out.reshape(rows, cols)
