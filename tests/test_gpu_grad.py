"""Autograd backward of the loops (adjoint M^dag solve) against the oracle.

* dl/dmu for a random complex weighting G of all 160 insertions and several
  momenta, against the oracle's forward-mode derivative Re sum conj(G) dL/dmu
  (FP64 path 1e-8; FP32 contraction with FP32/FP64-reliable solves 2e-5);
* dl/deta against the oracle's directional derivative in a random direction;
* torch.autograd.gradcheck on a scalar loss at 2^4 (FP64);
* 16^3 x 32 (eps 0.3, seed 2, kappa 0.125, mu 0.01), FP32: d/dmu of the scalar
  and gamma_5 loops (both flavour structures) against central differences
  (dmu = 1e-4) of the forward.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import gauge, to_device
from oracle import grad as ograd
from oracle import lattice, momenta, philox
from paper_1401_6750_gb300 import abi, api, synth

pytestmark = pytest.mark.gpu


def _weights(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("prec,solver,rho,tol", [
    (abi.TSM_F64, abi.TSM_SOLVER_F64, 1e-12, 1e-8),
    (abi.TSM_F32, abi.TSM_SOLVER_F32_RELIABLE, 1e-10, 2e-5),
])
def test_backward_matches_oracle(ctx, prec, solver, rho, tol):
    dims = (4, 4, 2, 6)
    kappa, mu = 0.125, 0.05
    g, links = gauge(ctx, dims, 0.4, 81, -1)
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(1)
    nsrc = 2
    etas = np.stack([philox.z4_source(dims, 9, r) for r in range(nsrc)])
    G = _weights((160, len(moms), dims[3]), 82)
    mu_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    eta_t = torch.from_numpy(etas).to("cuda").requires_grad_(True)
    L = api.one_end_loops(mu_t, eta_t, g, kappa, moms, solver, rho, prec)
    loss = (torch.conj(torch.from_numpy(G).to("cuda")) * L).real.sum()
    loss.backward()
    _, dL = ograd.loops_and_mu_derivative(u, list(etas), kappa, mu, dims, moms, rho=1e-13)
    want = float(np.real(np.sum(np.conj(G) * dL)))
    assert abs(mu_t.grad.item() - want) <= tol * abs(want), (mu_t.grad.item(), want)
    d = synth.gaussian_spinor(dims, 83, nrhs=nsrc)
    dLd = ograd.loops_eta_directional(u, list(etas), list(d), kappa, mu, dims, moms, rho=1e-13)
    want_d = float(np.real(np.sum(np.conj(G) * dLd)))
    got_d = float(np.real(np.sum(np.conj(eta_t.grad.cpu().numpy()) * d)))
    assert abs(got_d - want_d) <= tol * abs(want_d), (got_d, want_d)
    g.close()


def test_gradcheck_small_fp64(ctx):
    dims = (2, 2, 2, 4)
    kappa = 0.12
    g, _ = gauge(ctx, dims, 0.5, 84, -1, precs=(abi.TSM_F64,))
    moms = [(0, 0, 0), (1, 0, 0)]
    W = torch.from_numpy(_weights((160, 2, 4), 85)).to("cuda")
    eta = torch.from_numpy(synth.gaussian_spinor(dims, 86, nrhs=1)).to("cuda").requires_grad_(True)
    mu = torch.tensor(0.07, dtype=torch.float64, requires_grad=True)

    def f(m, e):
        L = api.one_end_loops(m, e, g, kappa, moms, abi.TSM_SOLVER_F64, 1e-13, abi.TSM_F64)
        return (torch.conj(W) * L).real.sum()

    assert torch.autograd.gradcheck(f, (mu, eta), eps=1e-6, atol=1e-7, rtol=1e-5, fast_mode=True)
    g.close()


def test_mu_derivative_16x16x16x32_fp32_finite_difference(ctx):
    """The differentiation configuration: 16^3 x 32 (eps 0.3, seed 2, kappa
    0.125, mu 0.01), d/dmu of the scalar and g5 loops of both flavour
    structures over 100 Z4 sources by the adjoint backward (FP32 solves with
    float-float reliable updates, even-odd), against central finite
    differences with delta mu = 1e-4."""
    dims = (16, 16, 16, 32)
    kappa, mu, h = 0.125, 0.01, 1e-4
    g, _ = gauge(ctx, dims, 0.3, 2, -1)
    moms = [(0, 0, 0)]
    nsrc = 100
    etas = torch.stack([to_device(philox.z4_source(dims, 1005, r)) for r in range(nsrc)])
    sel = [0, 15, 80, 95]  # scalar and gamma_5, with and without tau_3
    W = torch.zeros((160, 1, dims[3]), dtype=torch.complex128, device="cuda")
    W[sel] = 1.0 + 0.5j

    def loss(m):
        L = api.one_end_loops(m, etas, g, kappa, moms, abi.TSM_SOLVER_F32_RELIABLE | abi.TSM_SOLVER_EO, 1e-10,
                              abi.TSM_F32)
        return (torch.conj(W) * L).real.sum()

    mu_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    loss(mu_t).backward()
    with torch.no_grad():
        fd = (loss(torch.tensor(mu + h, dtype=torch.float64)) - loss(torch.tensor(mu - h, dtype=torch.float64))) / (2 * h)
    assert abs(mu_t.grad.item() - fd.item()) <= 2e-3 * abs(fd.item()), (mu_t.grad.item(), fd.item())
    g.close()
