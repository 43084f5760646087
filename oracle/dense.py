"""Dense matrices and exact loop traces on small lattices.

Used to pin the stochastic estimators: with G = M^{-1} formed explicitly
(numpy's LU-based inverse as the library step) the exact traces
Tr[X (G_u -/+ G_d)] of every insertion operator X are read off the matrix
entries directly.  The vector index is 12*site + 3*spin + colour, with the
site index x + Lx*(y + Ly*(z + Lz*t)).

Bilinear convention (same reading as ``contract``): psibar(y) K psi(z) has
the value Tr[K G(z, y)], with K a 12x12 spin-colour matrix.
"""
import numpy as np

from . import dirac, lattice
from .gamma import INSERTIONS

N_INSERTIONS = 160


def operator_matrix(apply, dims):
    """Dense matrix of a linear map on spinor fields, built column by column."""
    shp = lattice.shape(dims) + (4, 3)
    n = int(np.prod(shp))
    mat = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        mat[:, j] = apply(e.reshape(shp)).ravel()
        e[j] = 0.0
    return mat


def m_matrix(u, dims, kappa, mu):
    return operator_matrix(lambda f: dirac.apply_M(u, f, kappa, mu), dims)


def propagators(u, dims, kappa, mu):
    """(G_u, G_d) = (M(mu)^{-1}, M(-mu)^{-1}) as dense matrices."""
    g_u = np.linalg.inv(m_matrix(u, dims, kappa, mu))
    g_d = np.linalg.inv(m_matrix(u, dims, kappa, -mu))
    return g_u, g_d


def _site(dims, x, y, z, t):
    lx, ly, lz, lt = dims
    return (x % lx) + lx * ((y % ly) + ly * ((z % lz) + lz * (t % lt)))


def _shift(c, mu, d):
    c = list(c)
    c[mu] += d
    return tuple(c)


def _bilinear_trace(g, dims, y, z, k):
    """Tr[K G(z, y)] for sites y, z given as coordinate tuples."""
    iy, iz = _site(dims, *y), _site(dims, *z)
    blk = g[12 * iz:12 * iz + 12, 12 * iy:12 * iy + 12]
    return np.trace(k @ blk)


def exact_densities(g, u, dims):
    """Per-site exact traces of the 80 insertion operators (no flavour factor).

    g is a dense propagator; returns complex128 (80, t, z, y, x) where index
    g_idx is ultra-local Gamma_g and 16 + 16 mu + g_idx the derivative.
    """
    lx, ly, lz, lt = dims
    one = np.eye(3, dtype=np.complex128)
    out = np.zeros((80, lt, lz, ly, lx), dtype=np.complex128)
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    c = (x, y, z, t)
                    for gi in range(16):
                        out[gi, t, z, y, x] = _bilinear_trace(
                            g, dims, c, c, np.kron(INSERTIONS[gi], one))
                    for m in range(4):
                        cp, cm = _shift(c, m, 1), _shift(c, m, -1)
                        ux = u[t, z, y, x, m]
                        xm, ym, zm, tm = cm[0] % lx, cm[1] % ly, cm[2] % lz, cm[3] % lt
                        ub = u[tm, zm, ym, xm, m]
                        for gi in range(16):
                            gm = INSERTIONS[gi]
                            t1 = _bilinear_trace(g, dims, c, cp, np.kron(gm, ux))
                            t2 = _bilinear_trace(g, dims, cp, c, np.kron(gm, ux.conj().T))
                            t3 = _bilinear_trace(g, dims, cm, c, np.kron(gm, ub))
                            t4 = _bilinear_trace(g, dims, c, cm, np.kron(gm, ub.conj().T))
                            out[16 + 16 * m + gi, t, z, y, x] = 0.25 * (t1 - t2 + t3 - t4)
    return out


def exact_flavour_densities(u, dims, kappa, mu):
    """Exact per-site traces for all 160 insertions: (160, t, z, y, x).

    Insertions 0..79 carry Tr[X (G_u - G_d)] (with tau_3), 80..159 carry
    Tr[X (G_u + G_d)] (without).
    """
    g_u, g_d = propagators(u, dims, kappa, mu)
    du = exact_densities(g_u, u, dims)
    dd = exact_densities(g_d, u, dims)
    return np.concatenate([du - dd, du + dd])
