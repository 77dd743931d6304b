"""Philox4x32-10 counter-based generator and the Box-Muller normals the oracle draws.

TEST INFRASTRUCTURE ONLY.  This module belongs to the FP64 CPU oracle.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference legs
of ``bench.py`` may import it; the CUDA library never does, and it shares no code
with the CUDA path.

Philox4x32-10 is written from its published definition (Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.3 and
Table 2): a 4-word counter and a 2-word key, ten rounds, each round multiplying
words 0 and 2 by two fixed constants (full 64-bit products), mixing the high
halves with the other two words and the key, and bumping the key by two Weyl
constants between rounds.

The stochastic stress of the method (Sec. III.B.2, the flux Sigma^n built from
i.i.d. unit normals W^n drawn afresh each step) needs 6 normals per cell and
step.  Counter layout (a reading; the paper names no generator):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (cell_linear_index, step, call, 0), call in {0, 1}
  call 0: words (0,1) -> Z_xx, Z_yy ; words (2,3) -> Z_zz, Z_xy
  call 1: words (0,1) -> Z_xz, Z_yz ; words 2,3 unused
Each word x maps to a uniform u = (x + 0.5) * 2**-32 in (0, 1); a pair (u1, u2)
gives sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2)  (Box and Muller, 1958).
"""
import numpy as np

# Round multipliers and key increments of Philox4x32 (SC'11, Table 2).
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(counter, key, rounds=10):
    """Philox4x32-R on arrays.

    counter: sequence of 4 integer arrays (broadcastable), each word < 2**32.
    key:     pair of python ints < 2**32.
    Returns a tuple of 4 uint32 arrays.
    """
    c = [np.asarray(w, dtype=np.uint64) & _MASK32 for w in counter]
    c = list(np.broadcast_arrays(*c))
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for rnd in range(rounds):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = PHILOX_M0 * c[0]          # exact: both factors < 2**32
        p1 = PHILOX_M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return tuple(w.astype(np.uint32) for w in c)


def uniform_from_word(x):
    """Map 32-bit words to uniforms in (0, 1): (x + 1/2) 2^-32, in FP64."""
    return (np.asarray(x, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(x1, x2):
    """Two words -> two independent unit normals (cos branch, sin branch), FP64."""
    u1 = uniform_from_word(x1)
    u2 = uniform_from_word(x2)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def stress_normals(seed, step, ncell, plane):
    """The 6 unit normals of every cell for one step.

    Returns an array (6, ncell) ordered (Z_xx, Z_yy, Z_zz, Z_xy, Z_xz, Z_yz),
    cell index = i + Nx (j + Ny k); plane = Nx Ny cells per z plane.

    Counter layout (key = the seed's two 32-bit halves, counter word 1 = the step):
    call 0 at (cell, step, 0, 0) gives (Z_xx, Z_yy) from words 0-1 and (Z_zz, Z_xy)
    from words 2-3.  Call 1 at (cell of plane 2m, step, 1, 0) serves the two planes
    2m and 2m + 1: words 0-1 give (Z_xz, Z_yz) of the cell in plane 2m, words 2-3 those
    of the cell above it.  Every normal comes from its own pair of words, so all of
    them are independent (Sec. III.B: W holds independent unit normals per cell and
    step; which counter draws which entry is a free choice).
    """
    seed = int(seed)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    lin = np.arange(ncell, dtype=np.int64)
    odd = (lin // int(plane)) % 2 == 1
    below = (lin - np.where(odd, int(plane), 0)).astype(np.uint64)
    n = np.uint64(int(step) & 0xFFFFFFFF)
    a0, a1, a2, a3 = philox4x32((lin.astype(np.uint64), n, np.uint64(0), np.uint64(0)), key)
    b0, b1, b2, b3 = philox4x32((below, n, np.uint64(1), np.uint64(0)), key)
    zxx, zyy = box_muller(a0, a1)
    zzz, zxy = box_muller(a2, a3)
    zxz, zyz = box_muller(np.where(odd, b2, b0), np.where(odd, b3, b1))
    return np.stack([zxx, zyy, zzz, zxy, zxz, zyz])
