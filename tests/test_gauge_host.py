"""The library's host gauge generator (tsm_generate_gauge_host), no GPU:
the documented normals (Philox4x64-10 words, Box-Muller pairs) rebuilt here
with the oracle's Philox give H, and scipy's matrix exponential of i eps H
must equal the returned link; SU(3) properties; determinism."""
import os
import shutil

import numpy as np
import pytest

from oracle import philox
from paper_1401_6750_gb300 import build, synth

scipy_linalg = pytest.importorskip("scipy.linalg")
pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="CUDA toolkit needed to build the library")


@pytest.fixture(scope="module")
def api_mod():
    build.build()
    from paper_1401_6750_gb300 import api
    return api


def _normals(n_links, seed):
    ctr = np.arange(n_links, dtype=np.uint64)
    zero = np.zeros(n_links, dtype=np.uint64)
    words = philox.philox4x64_10((ctr, zero, zero, zero), (np.uint64(seed), np.uint64(0x67617567)))
    u = np.empty((n_links, 8))
    for k, w in enumerate(words):
        u[:, 2 * k] = ((w & np.uint64(0xFFFFFFFF)).astype(np.float64) + 0.5) * 2.0 ** -32
        u[:, 2 * k + 1] = ((w >> np.uint64(32)).astype(np.float64) + 0.5) * 2.0 ** -32
    h = np.empty((n_links, 8))
    r = np.sqrt(-2.0 * np.log(u[:, 0::2]))
    ph = 2.0 * np.pi * u[:, 1::2]
    h[:, 0::2] = r * np.cos(ph)
    h[:, 1::2] = r * np.sin(ph)
    return h


def test_links_are_exp_of_documented_generator(api_mod):
    dims, eps, seed = (4, 2, 2, 4), 0.3, 11
    u = api_mod.generate_gauge_host(dims, eps, seed).reshape(-1, 3, 3)
    h = _normals(u.shape[0], seed)
    H = np.einsum("na,aij->nij", h, synth.GELL_MANN) * 0.5
    for n in range(u.shape[0]):
        want = scipy_linalg.expm(1j * eps * H[n])
        assert np.max(np.abs(u[n] - want)) < 1e-13, n


def test_su3_and_determinism(api_mod):
    dims = (6, 4, 4, 8)
    a = api_mod.generate_gauge_host(dims, 0.5, 3)
    b = api_mod.generate_gauge_host(dims, 0.5, 3)
    c = api_mod.generate_gauge_host(dims, 0.5, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    m = a.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.max(np.abs(np.matmul(m, np.conj(np.swapaxes(m, -1, -2))) - eye)) < 1e-13
    assert np.max(np.abs(np.linalg.det(m) - 1.0)) < 1e-13


def test_same_distribution_as_synth(api_mod):
    """E[Re tr U / 3] and its spread agree with synth.gauge_links (another
    stream of the same distribution) within statistical error."""
    dims, eps = (8, 8, 8, 8), 0.4
    a = np.real(np.trace(api_mod.generate_gauge_host(dims, eps, 21), axis1=-2, axis2=-1)).ravel() / 3
    b = np.real(np.trace(synth.gauge_links(dims, eps, 21), axis1=-2, axis2=-1)).ravel() / 3
    se = np.sqrt(a.var() / a.size + b.var() / b.size)
    assert abs(a.mean() - b.mean()) < 5 * se
    assert abs(a.std() - b.std()) < 0.05 * b.std()
