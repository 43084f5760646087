"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only makes inputs.

* Gauge links U_mu(x) = exp(i eps H), H = sum_a h_a lambda_a / 2 with
  h_a ~ N(0, 1) i.i.d. and lambda_a the Gell-Mann matrices -- a stand-in for
  the paper's twisted-mass ensembles (Sec. 2.1.1 mentions 32^3 x 64
  configurations), which are not available.  The exponential is taken through
  the eigen-decomposition of the Hermitian 3x3 H, in FP64, giving an SU(3)
  matrix to rounding.
* Gaussian test spinors and random gauge transformations.

Layout: links are complex128 arrays (T, Lz, Ly, Lx, 4, 3, 3), i.e. the
row-major host layout [V][4][3][3] with site x + Lx*(y + Ly*(z + Lz*t));
spinors are (T, Lz, Ly, Lx, 4, 3).  dims = (Lx, Ly, Lz, T).
"""
import numpy as np


def _gell_mann():
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


GELL_MANN = _gell_mann()


def field_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def su3_from_hermitian(h, eps):
    """exp(i eps H) for a batch of Hermitian 3x3 matrices (..., 3, 3)."""
    w, vec = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.matmul(vec * ph[..., None, :], np.conj(np.swapaxes(vec, -1, -2)))


def gauge_links(dims, eps, seed):
    """Seeded SU(3) links U = exp(i eps H) on every site and direction."""
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal(field_shape(dims) + (4, 8))
    h = np.einsum("...a,aij->...ij", coef, GELL_MANN) * 0.5
    return su3_from_hermitian(h, eps)


def unit_links(dims):
    u = np.zeros(field_shape(dims) + (4, 3, 3), dtype=np.complex128)
    u[..., :, :] = np.eye(3)
    return u


def gaussian_spinor(dims, seed, nrhs=None):
    """Complex Gaussian spinor(s) with unit variance per real component."""
    rng = np.random.default_rng(seed)
    shp = field_shape(dims) + (4, 3)
    if nrhs is not None:
        shp = (nrhs,) + shp
    return rng.standard_normal(shp) + 1j * rng.standard_normal(shp)


def gauge_transform(dims, seed, eps=1.0):
    """Random SU(3) matrix g(x) per site, shape (T, Lz, Ly, Lx, 3, 3)."""
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal(field_shape(dims) + (8,))
    h = np.einsum("...a,aij->...ij", coef, GELL_MANN) * 0.5
    return su3_from_hermitian(h, eps)
