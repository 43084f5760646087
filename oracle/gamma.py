"""Euclidean Dirac matrices and the 16 ultra-local insertion matrices.

The paper (Sec. 2.1.1) computes "all ultra-local ... insertions": the 16
independent Dirac matrices.  It fixes no basis; traces do not depend on it.
This oracle uses a chiral basis in which gamma_5 is diagonal:

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   k = 1, 2, 3  (x, y, z)
    gamma_4 = [[0, 1], [1, 0]]                                   (t)

with 2x2 blocks and Pauli matrices sigma_k.  All four are Hermitian and
satisfy {gamma_mu, gamma_nu} = 2 delta_{mu nu}; gamma_5 = g1 g2 g3 g4.

Insertion order: Gamma_g = g1^{b0} g2^{b1} g3^{b2} g4^{b3}, where b_j is bit j
of g (so Gamma_0 = 1, Gamma_8 = gamma_4, Gamma_15 = gamma_5).
"""
import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
PAULI = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


def gammas():
    """Return an array g[mu] (mu = 0..3 for x, y, z, t) of 4x4 matrices."""
    out = np.zeros((4, 4, 4), dtype=np.complex128)
    for k in range(3):
        out[k] = _block(_Z2, -1j * PAULI[k], 1j * PAULI[k], _Z2)
    out[3] = _block(_Z2, _I2, _I2, _Z2)
    return out


GAMMA = gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def insertion(g):
    """Gamma_g = product over set bits j of g, in increasing j, of gamma_{j+1}."""
    m = np.eye(4, dtype=np.complex128)
    for j in range(4):
        if (g >> j) & 1:
            m = m @ GAMMA[j]
    return m


INSERTIONS = np.stack([insertion(g) for g in range(16)])
