"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks one oracle function against a closed form, a numpy library
routine, an algebraic identity or brute force, chosen so that a plausible
slip (a dropped term, a wrong sign or index, a transposed operand) fails.
"""
import numpy as np
import pytest

from oracle import contract, dense, dirac, freefield, gamma, lattice, momenta, philox, solver, tsm
from paper_1401_6750_gb300 import synth

RNG_DIMS = (2, 2, 2, 4)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


# --------------------------------------------------------------------------- gammas
def test_gamma_clifford_and_hermitian():
    g = gamma.GAMMA
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2.0 * (m == n) * np.eye(4), atol=0)


def test_gamma5_diagonal_chiral():
    assert np.allclose(gamma.GAMMA5, np.diag([1, 1, -1, -1]), atol=0)
    for m in range(4):
        assert np.allclose(gamma.GAMMA5 @ gamma.GAMMA[m], -gamma.GAMMA[m] @ gamma.GAMMA5)


def test_insertion_basis_orthogonal_and_ordered():
    ins = gamma.INSERTIONS
    gram = np.einsum("aij,bij->ab", ins.conj(), ins)  # Tr[Gamma_a^dag Gamma_b]
    assert np.allclose(gram, 4 * np.eye(16))
    assert np.allclose(ins[0], np.eye(4))
    for j in range(4):
        assert np.allclose(ins[1 << j], gamma.GAMMA[j])
    assert np.allclose(ins[15], gamma.GAMMA5)
    assert np.allclose(ins[3], gamma.GAMMA[0] @ gamma.GAMMA[1])


# --------------------------------------------------------------------------- RNG
def _counter_before(ctr):
    """numpy's Philox (Philox4x64-10) advances its 256-bit counter before each
    block, so a generator started at c - 1 first returns block c."""
    c = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    c = (c - 1) % 2**256
    return np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)


@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((5, 7, 9, 11), (123, 456)),
    ((2**64 - 2, 3, 4, 5), (2**63, 17)),
    ((1234567, 0, 0, 0), (1003, 42)),
])
def test_philox_matches_numpy(ctr, key):
    ref = np.random.Philox(counter=_counter_before(ctr),
                           key=np.array(key, dtype=np.uint64)).random_raw(4)
    got = philox.philox4x64_10([np.uint64(c) for c in ctr], [np.uint64(k) for k in key])
    assert [int(v) for v in got] == [int(v) for v in ref]


def test_z4_source_values_and_statistics():
    dims = (4, 4, 4, 8)
    eta = philox.z4_source(dims, 1001, 3)
    vals = eta.ravel()
    assert set(np.round(vals, 12).tolist()) <= {1, 1j, -1, -1j}
    counts = [np.sum(vals == z) for z in (1, 1j, -1, -1j)]
    n = vals.size
    for c in counts:  # each value has probability 1/4; 5 sigma band
        assert abs(c - n / 4) < 5 * np.sqrt(n * 3 / 16)
    other = philox.z4_source(dims, 1001, 4)
    assert np.mean(other == eta) < 0.4  # different source ids are different draws
    # E[eta eta^dag] = 1: off-diagonal average is small
    flat = eta.reshape(-1, 12)
    corr = flat.conj().T @ flat / flat.shape[0]
    assert np.allclose(np.diag(corr), 1.0)
    assert np.max(np.abs(corr - np.eye(12))) < 5 / np.sqrt(flat.shape[0])


def test_z4_bits_from_word0():
    # site 0 of source r uses bits (2k, 2k+1) of Philox word 0 for component k
    dims = (2, 2, 2, 2)
    eta = philox.z4_source(dims, 77, 5).reshape(-1, 12)
    w0 = int(np.random.Philox(counter=_counter_before((0, 0, 0, 0)),
                              key=np.array([77, 5], dtype=np.uint64)).random_raw(1)[0])
    want = [(1, 1j, -1, -1j)[(w0 >> (2 * k)) & 3] for k in range(12)]
    assert np.allclose(eta[0], want)


# --------------------------------------------------------------------------- momenta
def test_momentum_counts_lattice_points_in_ball():
    # number of integer points with n^2 <= R^2 (sum of r_3(k) for k <= R^2)
    expected = {0: 1, 1: 7, 2: 19, 3: 27, 4: 33, 5: 57, 6: 81, 7: 81, 8: 93, 9: 123}
    for p2, cnt in expected.items():
        assert len(momenta.momentum_list(p2)) == cnt


def test_momentum_order_and_symmetry():
    moms = momenta.momentum_list(9)
    assert moms[0] == (0, 0, 0)
    n2 = [a * a + b * b + c * c for a, b, c in moms]
    assert n2 == sorted(n2)
    assert len(set(moms)) == len(moms)
    assert set(moms) == {(-a, -b, -c) for a, b, c in moms}
    for i in range(len(moms) - 1):
        if n2[i] == n2[i + 1]:
            assert moms[i] < moms[i + 1]


# --------------------------------------------------------------------------- operator
@pytest.mark.parametrize("t_bc", [1, -1])
def test_free_field_plane_wave(t_bc):
    dims = (4, 2, 6, 8)
    kappa, mu = 0.137, 0.043
    u = lattice.effective_links(synth.unit_links(dims), t_bc)
    x, y, z, t = lattice.coords(dims)
    rng = np.random.default_rng(0)
    theta = 0.0 if t_bc > 0 else 1.0
    for trial in range(3):
        n = [rng.integers(0, L) for L in dims]
        p = [2 * np.pi * n[0] / dims[0], 2 * np.pi * n[1] / dims[1],
             2 * np.pi * n[2] / dims[2], (2 * n[3] + theta) * np.pi / dims[3]]
        spin = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        col = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        wave = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = wave[..., None, None] * np.outer(spin, col)
        # closed form M(p) = a + i 2 kappa (sum gamma sin p + mu gamma5)
        a = 1 - 2 * kappa * sum(np.cos(q) for q in p)
        mp = a * np.eye(4) + 2j * kappa * (sum(gamma.GAMMA[m] * np.sin(p[m]) for m in range(4))
                                          + mu * gamma.GAMMA5)
        want = wave[..., None, None] * np.outer(mp @ spin, col)
        assert rel(dirac.apply_M(u, psi, kappa, mu), want) < 1e-13
        mdag = mp.conj().T
        want = wave[..., None, None] * np.outer(mdag @ spin, col)
        assert rel(dirac.apply_Mdag(u, psi, kappa, mu), want) < 1e-13


def _gauge_rotate(u, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    out = np.empty_like(u)
    for m in range(4):
        gp = lattice.fwd(g, m)
        out[..., m, :, :] = g @ u[..., m, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    return out


def test_gauge_covariance():
    dims = (2, 4, 2, 4)
    u0 = synth.gauge_links(dims, 0.7, 11)
    g = synth.gauge_transform(dims, 12)
    psi = synth.gaussian_spinor(dims, 13)
    kappa, mu = 0.11, 0.2
    u = lattice.effective_links(u0, -1)
    ug = lattice.effective_links(_gauge_rotate(u0, g), -1)
    gpsi = np.matmul(psi, np.swapaxes(g, -1, -2))  # (g psi)_{s a} = g_ab psi_sb
    for op in (dirac.apply_M, dirac.apply_Mdag):
        lhs = op(ug, gpsi, kappa, mu)
        rhs = np.matmul(op(u, psi, kappa, mu), np.swapaxes(g, -1, -2))
        assert rel(lhs, rhs) < 1e-13


def test_adjoint_pair():
    dims = (2, 2, 4, 4)
    u = lattice.effective_links(synth.gauge_links(dims, 0.5, 3), -1)
    a = synth.gaussian_spinor(dims, 4)
    b = synth.gaussian_spinor(dims, 5)
    kappa, mu = 0.13, 0.07
    lhs = np.vdot(a.ravel(), dirac.apply_M(u, b, kappa, mu).ravel())
    rhs = np.vdot(dirac.apply_Mdag(u, a, kappa, mu).ravel(), b.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gamma5_hermiticity_dense():
    dims = RNG_DIMS
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 6), -1)
    kappa, mu = 0.125, 0.01
    m_plus = dense.m_matrix(u, dims, kappa, mu)
    m_minus = dense.m_matrix(u, dims, kappa, -mu)
    g5 = np.kron(np.eye(lattice.volume(dims)), np.kron(gamma.GAMMA5, np.eye(3)))
    assert np.allclose(g5 @ m_plus @ g5, m_minus.conj().T, atol=1e-14)
    mdag = dense.operator_matrix(lambda f: dirac.apply_Mdag(u, f, kappa, mu), dims)
    assert np.allclose(mdag, m_plus.conj().T, atol=1e-14)


def test_normal_operator_is_flavour_blind():
    dims = (2, 2, 2, 4)
    u = lattice.effective_links(synth.gauge_links(dims, 0.5, 7), -1)
    psi = synth.gaussian_spinor(dims, 8)
    kappa, mu = 0.12, 0.3
    lhs = dirac.apply_MdagM(u, psi, kappa, mu)
    rhs = dirac.apply_Adag(u, dirac.apply_A(u, psi, kappa), kappa) + (2 * kappa * mu) ** 2 * psi
    assert rel(lhs, rhs) < 1e-14


# --------------------------------------------------------------------------- solver
def test_cg_matches_dense_solve():
    dims = RNG_DIMS
    u = lattice.effective_links(synth.gauge_links(dims, 0.3, 1), -1)
    kappa, mu = 0.125, 0.01
    eta = philox.z4_source(dims, 1001, 0)
    s, iters, res = solver.solve(u, eta, kappa, mu, rho=1e-13)
    assert res <= 1e-13 and iters > 5
    m = dense.m_matrix(u, dims, kappa, mu)
    want = np.linalg.solve(m, eta.ravel()).reshape(eta.shape)
    assert rel(s, want) < 1e-9


def test_cg_stopping_rule():
    dims = RNG_DIMS
    u = lattice.effective_links(synth.gauge_links(dims, 0.3, 1), -1)
    eta = philox.z4_source(dims, 1001, 1)
    b = dirac.apply_Mdag(u, eta, 0.125, 0.01)
    for rho in (1e-2, 1e-5, 1e-8):
        x, iters, res = solver.cg_normal(u, b, 0.125, 0.01, rho, 10000)
        true = np.linalg.norm((b - dirac.apply_MdagM(u, x, 0.125, 0.01)).ravel()) / np.linalg.norm(b.ravel())
        assert abs(true - res) <= 1e-12 * max(1.0, res) and res <= rho


# --------------------------------------------------------------------------- traces and estimators
@pytest.mark.parametrize("dims,t_bc", [((2, 2, 2, 4), -1), ((3, 2, 4, 4), 1)])
def test_dense_traces_free_field_closed_form(dims, t_bc):
    kappa, mu = 0.12, 0.05
    u = lattice.effective_links(synth.unit_links(dims), t_bc)
    moms = momenta.momentum_list(2)
    ex = contract.project(dense.exact_flavour_densities(u, dims, kappa, mu), dims, moms)
    cf = freefield.zero_momentum_loops(dims, t_bc, kappa, mu)
    scale = np.max(np.abs(cf))
    for t in range(dims[3]):
        assert np.max(np.abs(ex[:, 0, t] - cf)) < 1e-12 * scale
    assert np.max(np.abs(ex[:, 1:, :])) < 1e-12 * scale
    # the check has teeth: tau3-gamma5, the u+d scalar and the u+d gamma_4
    # t-derivative are non-zero in the free field (and gamma_mu mu-derivatives
    # for every direction whose extent is above 2)
    for ins in (15, 80, 80 + 16 + 16 * 3 + 8):
        assert abs(cf[ins]) > 1e-3 * scale
    assert np.sum(np.abs(cf) > 1e-3 * scale) == 3 + sum(L > 2 for L in dims[:3])


@pytest.mark.parametrize("mu", [0.05, 0.0])
def test_one_end_identity_unit_sources(mu):
    """Summed over all 12V unit-vector sources the estimators are exact.  At
    mu = 0 (G_u = G_d = A^-1) the tau_3 estimator vanishes identically and
    the other gives 2 Tr[X A^-1] (g5-hermiticity of A)."""
    dims = RNG_DIMS
    kappa = 0.12
    u = lattice.effective_links(synth.gauge_links(dims, 0.5, 21), -1)
    g_u, _ = dense.propagators(u, dims, kappa, mu)
    n = g_u.shape[0]
    cols = g_u.T.reshape((n,) + lattice.shape(dims) + (4, 3))  # s_j = G_u e_j
    est = contract.loop_densities(u, cols, kappa, mu).sum(axis=1)
    exact = dense.exact_flavour_densities(u, dims, kappa, mu)
    assert rel(est, exact) < 1e-11
    for ins in range(160):
        scale = np.max(np.abs(exact[ins]))
        assert np.max(np.abs(est[ins] - exact[ins])) <= 1e-10 * max(scale, 1e-12)


def test_loop_densities_gauge_invariant():
    dims = (2, 4, 2, 4)
    kappa, mu = 0.13, 0.02
    u0 = synth.gauge_links(dims, 0.6, 31)
    g = synth.gauge_transform(dims, 32)
    s = synth.gaussian_spinor(dims, 33)
    d0 = contract.loop_densities(lattice.effective_links(u0, -1), s, kappa, mu)
    gs = np.matmul(s, np.swapaxes(g, -1, -2))
    d1 = contract.loop_densities(lattice.effective_links(_gauge_rotate(u0, g), -1), gs, kappa, mu)
    assert rel(d1, d0) < 1e-13


def test_projection_matches_numpy_fft():
    dims = (6, 4, 5, 3)
    rng = np.random.default_rng(5)
    dens = rng.standard_normal((7,) + lattice.shape(dims)) + 1j * rng.standard_normal((7,) + lattice.shape(dims))
    moms = momenta.momentum_list(9)
    got = contract.project(dens, dims, moms)
    fft = np.fft.fftn(dens, axes=(-3, -2, -1))  # sum f e^{-2 pi i k n / N} over (z, y, x)
    lx, ly, lz, _ = dims
    for k, (nx, ny, nz) in enumerate(moms):
        want = fft[:, :, nz % lz, ny % ly, nx % lx]
        assert np.allclose(got[:, k, :], want, atol=1e-11)


def test_reality_of_hermitian_insertions():
    """phi^dag X chi0 with phi = g5 s: real per site when g5 X is Hermitian."""
    dims = (2, 2, 2, 4)
    u = lattice.effective_links(synth.gauge_links(dims, 0.5, 41), -1)
    s = synth.gaussian_spinor(dims, 42)
    kappa, mu = 0.12, 0.05
    d = contract.loop_densities(u, s, kappa, mu)
    mu_p = 2 * kappa * mu
    for g in range(16):
        h = gamma.GAMMA5 @ gamma.INSERTIONS[g]
        raw = d[g] / (-2j * mu_p)
        if np.allclose(h, h.conj().T):
            assert np.max(np.abs(raw.imag)) < 1e-12 * np.max(np.abs(raw))
        else:  # anti-Hermitian: purely imaginary
            assert np.allclose(h, -h.conj().T)
            assert np.max(np.abs(raw.real)) < 1e-12 * np.max(np.abs(raw))


# --------------------------------------------------------------------------- TSM
def test_tsm_correction_vanishes_when_maps_agree():
    dims = RNG_DIMS
    kappa, mu = 0.125, 0.01
    u = lattice.effective_links(synth.gauge_links(dims, 0.3, 1), -1)
    moms = momenta.momentum_list(1)
    est, (bulk, hp, lpc) = tsm.tsm_loops(u, dims, kappa, mu, 1001, 3, 2, 1e-6, 1e-6, moms)
    assert np.array_equal(hp, lpc)
    assert np.allclose(est, bulk / 3, rtol=0, atol=0)


def test_tsm_unbiased_against_exact():
    """The TSM estimate of p = 0 loops is consistent with the exact traces.

    The low-precision map here is deliberately crude (rho = 0.3, so LP-only
    averages are biased); 4 sigma from a jackknife over correction sources.
    """
    dims = RNG_DIMS
    kappa, mu = 0.12, 0.1
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 51), -1)
    moms = [(0, 0, 0)]
    exact = contract.project(dense.exact_flavour_densities(u, dims, kappa, mu), dims, moms)
    n_lp, n_hp = 60, 30
    lp = [tsm.source_loops(u, dims, kappa, mu, 7, r, 0.3, moms)[0] for r in range(n_lp + n_hp)]
    hp = [tsm.source_loops(u, dims, kappa, mu, 7, r, 1e-10, moms)[0] for r in range(n_lp, n_lp + n_hp)]
    lp, hp = np.array(lp), np.array(hp)
    est = tsm.combine(lp[:n_lp].sum(0), n_lp, hp.sum(0), lp[n_lp:].sum(0), n_hp)
    # per-sample TSM contributions -> standard error
    corr = hp - lp[n_lp:]
    def var(a):  # component-wise variance of the mean (real, imaginary)
        return a.real.var(0, ddof=1) + 1j * a.imag.var(0, ddof=1)
    v = var(lp[:n_lp]) / n_lp + var(corr) / n_hp
    sig = np.sqrt(v.real) + 1j * np.sqrt(v.imag)
    for ins in (0, 15, 80, 95):  # scalar and gamma5, both flavour structures
        for t in range(dims[3]):
            d = est[ins, 0, t] - exact[ins, 0, t]
            assert abs(d.real) <= 4 * sig[ins, 0, t].real + 1e-12
            assert abs(d.imag) <= 4 * sig[ins, 0, t].imag + 1e-12


def test_density_subset_equals_full():
    """loop_densities(only=...) evaluates the same formulas for the listed
    insertions and leaves the rest zero."""
    dims = (2, 2, 2, 4)
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 61), -1)
    s = synth.gaussian_spinor(dims, 62)
    full = contract.loop_densities(u, s, 0.12, 0.05)
    sel = {0, 15, 17, 95, 152}
    part = contract.loop_densities(u, s, 0.12, 0.05, only=sel)
    for i in range(contract.N_INSERTIONS):
        if i in sel:
            assert np.array_equal(part[i], full[i])
        else:
            assert not np.any(part[i])


def test_density_given_chi1_equals_full():
    """Passing g5 A s beforehand changes nothing."""
    dims = (2, 2, 2, 4)
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 63), -1)
    s = synth.gaussian_spinor(dims, 64)
    v = dirac.gamma5(dirac.apply_A(u, s, 0.12))
    full = contract.loop_densities(u, s, 0.12, 0.05)
    assert np.array_equal(contract.loop_densities_pair(u, s, s, 0.12, 0.05, chi1=v), full)
