"""Lattice geometry for the oracle.

Fields are numpy arrays whose lattice axes are (t, z, y, x), followed by
exactly two internal axes (spin, colour) or (colour, colour); any leading axes
are batch axes.  The flat site index of C order is i = x + Lx*(y + Ly*(z + Lz*t)).  ``dims`` is always
(Lx, Ly, Lz, T).  Direction mu = 0, 1, 2, 3 means x, y, z, t.

Boundary conditions: periodic in space; in time the link U_t(x) on the last
timeslice (t = T-1, hopping to t = 0) carries the factor ``t_bc`` (+1
periodic, -1 antiperiodic).  This sign is applied to a copy of the links
("effective links") that every other module then uses with plain periodic
shifts -- so the hopping term and the derivative insertions see the same sign.
"""
import numpy as np

AXIS = (-3, -4, -5, -6)  # direction mu -> axis of a (..., t, z, y, x, i, j) field


def shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def volume(dims):
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


def fwd(f, mu):
    """f(x + mu_hat) stored at x (periodic shift)."""
    return np.roll(f, -1, axis=AXIS[mu])


def bwd(f, mu):
    """f(x - mu_hat) stored at x (periodic shift)."""
    return np.roll(f, 1, axis=AXIS[mu])


def effective_links(links, t_bc):
    """Copy of links (t, z, y, x, mu, a, b) with U_t on t = T-1 times t_bc."""
    u = np.array(links, dtype=np.complex128, copy=True)
    u[-1, :, :, :, 3] *= t_bc
    return u


def coords(dims):
    """Integer coordinate arrays x, y, z, t of the field shape."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing="ij")
    return x, y, z, t
