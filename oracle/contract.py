"""One-end-trick loop densities for the 160 insertions and their projection.

Sec. 2.1.1 computes, with the one-end trick for twisted mass, "all ultra-local
and one-derivative insertions ... with and without a flavor tau_3 matrix, that
is, 160 insertions", projected to momenta with p^2 <= 9 per timeslice
(Sec. 2.2: volume indices kept open for the Fourier transform; the result
carries a timeslice index).  The paper prints no estimator formula; the
readings used here (derived from gamma_5-hermiticity and
M^dag M = A^dag A + mu'^2) are, for an operator X and s_r = M^{-1} eta_r:

    with tau_3 (flavour u - d):  Tr[X (G_u - G_d)] ~ -2 i mu' <s_r^dag g5 X s_r>
    without (flavour u + d):     Tr[X (G_u + G_d)] ~  2      <s_r^dag g5 X g5 A s_r>

where G_u = M(mu)^{-1}, G_d = M(-mu)^{-1}, <.> is the average over sources
and A = M(mu = 0).  With phi = g5 s, chi_0 = s and chi_1 = v = g5 A s both are
bilinears phi^dag X chi.  The bilinear of psibar(y) K psi(z) is the trace
Tr[K G(z, y)], i.e. phi(y)^dag K chi(z) (no fermion-loop sign).

Insertions (index ins = 80 f + (g if ultra-local else 16 + 16 mu + g)):

    ultra-local  X = psibar(x) Gamma_g psi(x)
    derivative   X = 1/4 [ psibar(x) Gamma U_mu(x) psi(x+mu)
                         - psibar(x+mu) Gamma U_mu(x)^dag psi(x)
                         + psibar(x-mu) Gamma U_mu(x-mu) psi(x)
                         - psibar(x) Gamma U_mu(x-mu)^dag psi(x-mu) ]

assigned to site x.  Each density is written out here literally, insertion by
insertion -- not through the open-Dirac 4x4 route of Sec. 2.2.

Projection: L(n, t) = sum over the spatial sites of
L(x, t) exp(-2 pi i (nx x / Lx + ny y / Ly + nz z / Lz)), the sign of a
forward FFT (Sec. 2.3 uses cuFFT), written as a direct sum.
"""
import numpy as np

from . import dirac, lattice
from .gamma import INSERTIONS

N_INSERTIONS = 160


def insertion_index(flavour, derivative, direction, g):
    """flavour 0 = with tau_3, 1 = without; derivative False = ultra-local."""
    return 80 * flavour + ((16 + 16 * direction + g) if derivative else g)


def bilinear(a, g, b):
    """sum_{s, r, c} conj(a_{s c}) G_{s r} b_{r c} at every site."""
    return np.einsum("...sc,sr,...rc->...", np.conj(a), g, b)


def loop_densities_pair(u, a, b, kappa, mu, prefactor_derivative=False, only=None, chi1=None):
    """The sesquilinear form behind the loop densities: phi = g5 a on the left,
    chi_0 = b and chi_1 = g5 A b on the right, so loop_densities(s) is the
    pair (s, s).  With prefactor_derivative the flavour prefactors are
    replaced by their mu-derivatives (-2 i mu' -> -4 i kappa, 2 -> 0).
    ``only`` (a collection of insertion indices) skips every other insertion,
    leaving it zero: the same formulas, evaluated for a subset (large
    lattices).  ``chi1``, if given, is g5 A b computed beforehand (the same
    field, so that several subsets of one source share it)."""
    mu_p = 2.0 * kappa * mu
    want = (lambda i: True) if only is None else (lambda i: i in only)
    phi = dirac.gamma5(a)
    v = dirac.gamma5(dirac.apply_A(u, b, kappa)) if chi1 is None else chi1
    prefs = (-4j * kappa, 0.0) if prefactor_derivative else (-2j * mu_p, 2.0)
    out = np.zeros((N_INSERTIONS,) + a.shape[:-2], dtype=np.complex128)
    for flavour, (chi, pref) in enumerate(((b, prefs[0]), (v, prefs[1]))):
        if pref == 0.0:
            continue
        for g in range(16):
            if want(insertion_index(flavour, False, 0, g)):
                out[insertion_index(flavour, False, 0, g)] = pref * bilinear(phi, INSERTIONS[g], chi)
        for m in range(4):
            um = u[..., m, :, :]
            ub = lattice.bwd(um, m)
            for g in range(16):
                if not want(insertion_index(flavour, True, m, g)):
                    continue
                gm = INSERTIONS[g]
                t1 = bilinear(phi, gm, dirac.colour_mul(um, lattice.fwd(chi, m)))
                t2 = bilinear(lattice.fwd(phi, m), gm, dirac.colour_mul_dag(um, chi))
                t3 = bilinear(lattice.bwd(phi, m), gm, dirac.colour_mul(ub, chi))
                t4 = bilinear(phi, gm, dirac.colour_mul_dag(ub, lattice.bwd(chi, m)))
                out[insertion_index(flavour, True, m, g)] = pref * 0.25 * (t1 - t2 + t3 - t4)
    return out


def loop_densities(u, s, kappa, mu, only=None):
    """Per-site densities of all 160 insertions for one solved source s.

    ``u`` are effective links; ``s`` may carry leading batch axes (several
    sources).  Returns complex128 (160, ..., t, z, y, x); with ``only``, the
    insertions not listed are left zero.
    """
    return loop_densities_pair(u, s, s, kappa, mu, only=only)


def phases(dims, moms):
    """exp(-2 pi i n.x / L) for every momentum, shape (n_mom, z, y, x)."""
    lx, ly, lz, _ = dims
    x, y, z, _ = lattice.coords((lx, ly, lz, 1))
    x, y, z = x[0], y[0], z[0]
    out = np.empty((len(moms),) + x.shape, dtype=np.complex128)
    for k, (nx, ny, nz) in enumerate(moms):
        out[k] = np.exp(-2j * np.pi * (nx * x / lx + ny * y / ly + nz * z / lz))
    return out


def project(dens, dims, moms):
    """Direct sum over space: (..., t, z, y, x) -> (..., n_mom, t)."""
    return np.einsum("...tzyx,kzyx->...kt", dens, phases(dims, moms))


def one_end_loops(u, sources, kappa, mu, dims, moms):
    """Average over the given solved sources of the projected densities.

    Returns complex128 (160, n_mom, T).
    """
    acc = None
    for s in sources:
        d = project(loop_densities(u, s, kappa, mu), dims, moms)
        acc = d if acc is None else acc + d
    return acc / len(sources)
