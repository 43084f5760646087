"""Time-diluted sources and the standard loop estimator.  TEST INFRASTRUCTURE ONLY.

Sec. 2.2 also works with time dilution, with GPU kernels that contract a
single time slice and return an array with a timeslice index; the one-end
trick needs volume sources, so time-diluted sources go with the standard
estimator.  The paper prints no formula; the readings used here:

* source: the Z4 volume source of (noise_seed, source_id) kept on timeslice
  t0 and zero elsewhere, so the T diluted sources of one noise vector sum to
  the volume source;
* solve: s = M(mu)^{-1} eta_t0 (the u flavour only);
* the bilinear psibar(y) K psi(z), whose value is Tr[K G(z, y)] (same reading
  as ``contract``), is estimated for the u flavour by eta(y)^dag K s(z), since
  E[eta eta^dag] is the identity on the source's support;
* the d flavour comes from the same solve through g5-hermiticity,
  G_d = g5 G_u^dag g5:  Tr[K G_d(z, y)] = conj(Tr[g5 K^dag g5 G_u(y, z)]),
  estimated by conj(eta(z)^dag g5 K^dag g5 s(y));
* insertions, derivative form and index as in ``contract``: flavour 0 is
  u - d (with tau_3), flavour 1 is u + d.

Every density is written out term by term here.
"""
import numpy as np

from . import dirac, lattice, philox
from .gamma import GAMMA5, INSERTIONS

N_INSERTIONS = 160


def diluted_source(dims, noise_seed, source_id, t0):
    """The Z4 volume source of (noise_seed, source_id) on timeslice t0 only."""
    eta = philox.z4_source(dims, noise_seed, source_id)
    keep = np.zeros(lattice.shape(dims)[0], dtype=bool)
    keep[t0] = True
    return eta * keep[:, None, None, None, None, None]


def _bilinear(a, g, b):
    """sum_{s, r, c} conj(a_{s c}) G_{s r} b_{r c} at every site."""
    return np.einsum("...sc,sr,...rc->...", np.conj(a), g, b)


def standard_densities(u, eta, s, only=None):
    """Per-site densities of the 160 insertions from one source eta and its
    solution s = M(mu)^{-1} eta: complex128 (160, t, z, y, x).  ``only`` (a
    collection of insertion indices) evaluates the same formulas for those
    insertions (both flavour combinations of each listed Gamma and direction)
    and leaves the others zero."""
    out = np.zeros((N_INSERTIONS,) + eta.shape[:-2], dtype=np.complex128)
    want = (lambda i: True) if only is None else (lambda i: (i % 80) in {k % 80 for k in only})
    for g in range(16):
        if not want(g):
            continue
        gm = INSERTIONS[g]
        gd = GAMMA5 @ gm.conj().T @ GAMMA5
        du = _bilinear(eta, gm, s)
        dd = np.conj(_bilinear(eta, gd, s))
        out[g] = du - dd
        out[80 + g] = du + dd
    for m in range(4):
        um = u[..., m, :, :]
        ub = lattice.bwd(um, m)
        ef, eb = lattice.fwd(eta, m), lattice.bwd(eta, m)
        sf, sb = lattice.fwd(s, m), lattice.bwd(s, m)
        for g in range(16):
            if not want(16 + 16 * m + g):
                continue
            gm = INSERTIONS[g]
            gd = GAMMA5 @ gm.conj().T @ GAMMA5
            # u: psibar(y) K psi(z) -> eta(y)^dag K s(z)
            u1 = _bilinear(eta, gm, dirac.colour_mul(um, sf))       # psibar(x) G U(x) psi(x+mu)
            u2 = _bilinear(ef, gm, dirac.colour_mul_dag(um, s))     # psibar(x+mu) G U(x)^dag psi(x)
            u3 = _bilinear(eb, gm, dirac.colour_mul(ub, s))         # psibar(x-mu) G U(x-mu) psi(x)
            u4 = _bilinear(eta, gm, dirac.colour_mul_dag(ub, sb))   # psibar(x) G U(x-mu)^dag psi(x-mu)
            # d: psibar(y) K psi(z) -> conj(eta(z)^dag g5 K^dag g5 s(y))
            d1 = np.conj(_bilinear(ef, gd, dirac.colour_mul_dag(um, s)))
            d2 = np.conj(_bilinear(eta, gd, dirac.colour_mul(um, sf)))
            d3 = np.conj(_bilinear(eta, gd, dirac.colour_mul_dag(ub, sb)))
            d4 = np.conj(_bilinear(eb, gd, dirac.colour_mul(ub, s)))
            du = 0.25 * (u1 - u2 + u3 - u4)
            dd = 0.25 * (d1 - d2 + d3 - d4)
            out[16 + 16 * m + g] = du - dd
            out[80 + 16 + 16 * m + g] = du + dd
    return out


def tdil_loops(u, dims, kappa, mu, noise_seed, source_ids, moms, rho=1e-12):
    """Time-diluted standard-estimator loops: for every noise vector and every
    timeslice t0, solve with the diluted source, form the densities and
    project; averaged over the noise vectors.  Returns (160, n_mom, T)."""
    from . import contract, solver
    acc = 0
    for sid in source_ids:
        for t0 in range(dims[3]):
            eta = diluted_source(dims, noise_seed, sid, t0)
            s, _, _ = solver.solve(u, eta, kappa, mu, rho)
            acc = acc + contract.project(standard_densities(u, eta, s), dims, moms)
    return acc / len(source_ids)
