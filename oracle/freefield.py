"""Unit-gauge (free field) closed forms, used only to pin the oracle.

With U = 1 a plane wave exp(i p.x) u is an eigenfunction of the hopping term,
so the twisted-mass operator is the 4x4 matrix

    M(p) = a(p) + i 2 kappa (sum_mu gamma_mu sin p_mu + mu gamma_5),
    a(p) = 1 - 2 kappa sum_mu cos p_mu,

with p_k = 2 pi n_k / L_k in space and p_4 = (2 n + theta) pi / T in time
(theta = 0 periodic, 1 antiperiodic).  Its inverse is
(a - i 2 kappa (sum gamma sin p + mu gamma_5)) / (a^2 + 4 kappa^2 (sum sin^2 p + mu^2)).
Translation invariance then gives, per timeslice and at zero momentum,

    ultra-local:  sum_x Tr[Gamma G(x, x)]              = (3 / T) sum_p tr[Gamma G(p)]
    derivative:   1/4 [T1 - T2 + T3 - T4] summed        = (3 / T) sum_p i sin p_mu tr[Gamma G(p)]

and zero at every non-zero spatial momentum.
"""
import numpy as np

from .gamma import GAMMA, GAMMA5, INSERTIONS


def momentum_grid(dims, t_bc):
    lx, ly, lz, lt = dims
    theta = 0.0 if t_bc > 0 else 1.0
    px = 2 * np.pi * np.arange(lx) / lx
    py = 2 * np.pi * np.arange(ly) / ly
    pz = 2 * np.pi * np.arange(lz) / lz
    pt = (2 * np.arange(lt) + theta) * np.pi / lt
    return np.meshgrid(px, py, pz, pt, indexing="ij")


def propagator_p(p, kappa, mu):
    """G(p) for arrays p = (px, py, pz, pt); returns (..., 4, 4)."""
    a = 1.0 - 2.0 * kappa * sum(np.cos(q) for q in p)
    s = [np.sin(q) for q in p]
    den = a * a + 4.0 * kappa * kappa * (sum(q * q for q in s) + mu * mu)
    num = a[..., None, None] * np.eye(4)
    for m in range(4):
        num = num - 2j * kappa * s[m][..., None, None] * GAMMA[m]
    num = num - 2j * kappa * mu * np.ones_like(a)[..., None, None] * GAMMA5
    return num / den[..., None, None]


def zero_momentum_loops(dims, t_bc, kappa, mu):
    """Closed-form loops of all 160 insertions at n = 0, one value per timeslice.

    Returns complex128 (160,); the value is the same on every timeslice.
    Flavour order as in ``contract``: 0..79 with tau_3 (G_u - G_d),
    80..159 without (G_u + G_d).
    """
    lt = dims[3]
    p = momentum_grid(dims, t_bc)
    out = np.zeros(160, dtype=np.complex128)
    for flavour, sgn in ((0, -1.0), (1, 1.0)):
        g = propagator_p(p, kappa, mu) + sgn * propagator_p(p, kappa, -mu)
        for gi in range(16):
            tr = np.einsum("ab,...ba->...", INSERTIONS[gi], g)
            out[80 * flavour + gi] = 3.0 / lt * tr.sum()
            for m in range(4):
                out[80 * flavour + 16 + 16 * m + gi] = 3.0 / lt * (1j * np.sin(p[m]) * tr).sum()
    return out
