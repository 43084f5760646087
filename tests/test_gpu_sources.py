"""Z4 volume sources: device Philox4x64-10 against the oracle's, bit for bit."""
import numpy as np
import pytest

from gpu_helpers import gauge
from oracle import philox
from paper_1401_6750_gb300 import abi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (5, 3, 2, 7), (24, 24, 24, 48)])
@pytest.mark.parametrize("prec", [abi.TSM_F64, abi.TSM_F32, abi.TSM_F16, abi.TSM_BF16])
def test_sources_bit_exact(ctx, dims, prec):
    g, _ = gauge(ctx, dims, 0.3, 1, -1, precs=(prec,))
    seed, first, n = 1003, 7, 3
    nat = g.sources(seed, first, n, prec)
    got = g.unpack(nat, prec, n).cpu().numpy()
    for k in range(n if np.prod(dims) < 10**5 else 1):
        want = philox.z4_source(dims, seed, first + k)
        assert np.array_equal(got[k], want)
    g.close()


def test_large_seed_and_source_ids(ctx):
    dims = (4, 2, 2, 4)
    g, _ = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    seed, first = 2**63 + 12345, 2**40 + 3
    got = g.unpack(g.sources(seed, first, 2, abi.TSM_F64), abi.TSM_F64, 2).cpu().numpy()
    for k in range(2):
        assert np.array_equal(got[k], philox.z4_source(dims, seed, first + k))
    g.close()
