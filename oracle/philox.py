"""Philox4x64-10 and the Z4 volume sources.

The paper draws its stochastic sources with RANLUX on the host and plans to
move generation to the GPU (Sec. 2, Sec. 2.4).  Here both sides implement
one counter-based generator from its published definition -- Philox4x64 with
10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11) -- so that the device and this oracle draw identical noise.

Round function on the counter (X0, X1, X2, X3) with key (K0, K1):

    (H0, L0) = hi/lo(0xD2E7470EE14C6C93 * X0)
    (H1, L1) = hi/lo(0xCA5A826395121157 * X2)
    X' = (H1 ^ X1 ^ K0, L1, H0 ^ X3 ^ K1, L0)

with the key bumped by (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B) between
rounds.  64x64 -> 128-bit products are formed from 32-bit limbs.

Z4 source (proposed reading; the paper does not fix the noise): component
k = 3*spin + colour of site i of source r takes bits 2k, 2k+1 of word X'0 of
Philox(counter = (i, 0, 0, 0), key = (noise_seed, r)); the two-bit value z
maps to eta = i**z, i.e. 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i.
"""
import numpy as np

from . import lattice

_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)
_MUL0 = np.uint64(0xD2E7470EE14C6C93)
_MUL1 = np.uint64(0xCA5A826395121157)
_WEYL0 = np.uint64(0x9E3779B97F4A7C15)
_WEYL1 = np.uint64(0xBB67AE8584CAA73B)


def mulhilo64(a, b):
    """High and low 64-bit words of the 128-bit product a*b (uint64 arrays)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _M32, a >> _S32
    b_lo, b_hi = b & _M32, b >> _S32
    ll, lh, hl, hh = a_lo * b_lo, a_lo * b_hi, a_hi * b_lo, a_hi * b_hi
    mid = (ll >> _S32) + (lh & _M32) + (hl & _M32)
    lo = (ll & _M32) | ((mid & _M32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(ctr, key):
    """ctr: four uint64 arrays (broadcastable); key: two uint64 arrays."""
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) for k in key)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd:
                k0 = k0 + _WEYL0
                k1 = k1 + _WEYL1
            h0, l0 = mulhilo64(_MUL0, x0)
            h1, l1 = mulhilo64(_MUL1, x2)
            x0, x1, x2, x3 = h1 ^ x1 ^ k0, l1, h0 ^ x3 ^ k1, l0
    return x0, x1, x2, x3


Z4_VALUES = np.array([1.0, 1.0j, -1.0, -1.0j], dtype=np.complex128)


def z4_source(dims, noise_seed, source_id):
    """One Z4 volume source, shape (t, z, y, x, 4, 3), complex128."""
    v = lattice.volume(dims)
    site = np.arange(v, dtype=np.uint64)
    zero = np.zeros(v, dtype=np.uint64)
    w0, _, _, _ = philox4x64_10(
        (site, zero, zero, zero),
        (np.uint64(noise_seed), np.uint64(source_id)))
    k = np.arange(12, dtype=np.uint64)
    z = (w0[:, None] >> (np.uint64(2) * k[None, :])) & np.uint64(3)
    eta = Z4_VALUES[z.astype(np.int64)]
    return eta.reshape(lattice.shape(dims) + (4, 3))
