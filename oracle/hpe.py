"""Hopping parameter expansion (HPE) of the standard estimator.  TEST
INFRASTRUCTURE ONLY.

The paper cites the HPE as one of its variance reductions (Sec. 2.3) and
prints no formula.  The reading used here: with the operator split as
M = A0 - kappa H (A0 = 1 + i mu' g5 site-local, H the hopping term of
``dirac.hop`` with sign -1) and Y = A0^{-1} kappa H,

    G = sum_{k < 4} Y^k A0^{-1} + Y^4 G,

so for an insertion X the trace Tr[X G](x) is the exact diagonal of the
first four terms plus Tr[X Y^4 G](x), whose standard estimator is
eta(x)^dag X (Y^4 s)(x) with s = G eta.  It is applied to the 16 ultra-local
insertions of both flavours (d through g5-hermiticity as in ``tdil``); the
derivative insertions keep the plain standard estimator.  Per source, the
exact part is added on the timeslices the source covers.
"""
import numpy as np

from . import dirac, lattice, tdil
from .gamma import GAMMA5, INSERTIONS

ORDER = 4


def apply_a0inv(psi, kappa, mu):
    """A0^{-1} psi = (1 - i mu' g5) psi / (1 + mu'^2)."""
    mup = 2.0 * kappa * mu
    return (psi - 1j * mup * dirac.gamma5(psi)) / (1.0 + mup * mup)


def apply_y(u, psi, kappa, mu):
    """Y psi = A0^{-1} kappa H psi."""
    return apply_a0inv(kappa * dirac.hop(u, psi, -1.0), kappa, mu)


def remainder(u, s, kappa, mu, order=ORDER):
    """Y^order s."""
    for _ in range(order):
        s = apply_y(u, s, kappa, mu)
    return s


def exact_blocks(u, dims, kappa, mu, order=ORDER):
    """The 12x12 diagonal blocks [sum_{k < order} Y^k A0^{-1}](x, x) at every
    site, from the series applied to the 12 unit vectors of each site:
    complex128 (t, z, y, x, 12, 12), index 3 spin + colour."""
    shp = lattice.shape(dims) + (4, 3)
    n = int(np.prod(shp))
    out = np.zeros(lattice.shape(dims) + (12, 12), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        v = apply_a0inv(e.reshape(shp), kappa, mu)
        acc = v.copy()
        for _ in range(order - 1):
            v = apply_y(u, v, kappa, mu)
            acc += v
        site, a = divmod(j, 12)
        idx = np.unravel_index(site, lattice.shape(dims))
        out[idx + (slice(None), a)] = acc[idx].reshape(12)
    return out


def exact_ultralocal(blocks):
    """Per-site exact traces (flavour u, 16 Gamma): Tr[(Gamma x 1_colour) B(x)]."""
    out = np.zeros((16,) + blocks.shape[:-2], dtype=np.complex128)
    for g in range(16):
        k = np.kron(INSERTIONS[g], np.eye(3))
        out[g] = np.einsum("ab,...ba->...", k, blocks)
    return out


def _gd_index(g):
    """k and sign with g5 Gamma_g^dag g5 = sign * Gamma_k."""
    gd = GAMMA5 @ INSERTIONS[g].conj().T @ GAMMA5
    for k in range(16):
        for sign in (1.0, -1.0):
            if np.allclose(INSERTIONS[k], sign * gd):
                return k, sign
    raise AssertionError("g5 Gamma^dag g5 is not a Gamma")


def exact_densities(exact_u):
    """Exact HPE part of the 160 per-site densities: ultra-local u - d and
    u + d with Tr[X G_d] = conj(Tr[g5 X^dag g5 G_u]); zero for the
    derivative insertions."""
    out = np.zeros((160,) + exact_u.shape[1:], dtype=np.complex128)
    for g in range(16):
        k, sign = _gd_index(g)
        du, dd = exact_u[g], np.conj(sign * exact_u[k])
        out[g] = du - dd
        out[80 + g] = du + dd
    return out


def hpe_densities(u, eta, s, kappa, mu, exact_u=None, support=None, ultralocal_only=False):
    """Per-site densities of the 160 insertions for one source eta and its
    solution s (leading batch axes allowed): the ultra-local ones from the
    remainder estimator eta^dag X Y^4 s (both flavours), the derivative ones
    plain.  With exact_u (output of ``exact_ultralocal``) the exact part is
    added on the timeslices in `support` (all when None) -- once per noise
    source, since E[eta eta^dag] = 1 holds per source."""
    if ultralocal_only:
        out = np.zeros((160,) + eta.shape[:-2], dtype=np.complex128)
    else:
        out = tdil.standard_densities(u, eta, s)
    rem = remainder(u, s, kappa, mu)
    for g in range(16):
        gm = INSERTIONS[g]
        gd = GAMMA5 @ gm.conj().T @ GAMMA5
        du = tdil._bilinear(eta, gm, rem)
        dd = np.conj(tdil._bilinear(eta, gd, rem))
        out[g] = du - dd
        out[80 + g] = du + dd
    if exact_u is not None:
        ex = exact_densities(exact_u)
        if support is not None:
            keep = np.zeros(ex.shape[1], dtype=bool)
            keep[list(support)] = True
            ex = ex * keep[None, :, None, None, None]
        out = out + ex
    return out


def exact_ultralocal_constant(dims, kappa, mu):
    """The closed form of ``exact_ultralocal`` for lattices with every extent
    >= 4, broadcast to every site: orders 0 and 2 of the expansion (pinned
    against the series by the tests)."""
    from .gamma import GAMMA
    if min(dims) < 4:
        raise ValueError("the closed form needs every extent >= 4")
    mup = 2 * kappa * mu
    one = np.eye(4)
    a0i = (one - 1j * mup * GAMMA5) / (1 + mup * mup)
    inner = a0i.copy()
    for m in range(4):
        pm, pp = one - GAMMA[m], one + GAMMA[m]
        inner = inner + kappa ** 2 * (a0i @ pm @ a0i @ pp @ a0i + a0i @ pp @ a0i @ pm @ a0i)
    c = np.array([3 * np.trace(INSERTIONS[g] @ inner) for g in range(16)])
    return np.broadcast_to(c[:, None, None, None, None], (16,) + lattice.shape(dims)).copy()
