"""The oracle reproduces the counts and thresholds the paper prints."""
import os

from oracle import contract, gamma, momenta

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = v
    return out


def test_insertion_count():
    g = _golden()
    assert contract.N_INSERTIONS == int(g["n_insertions"])
    assert len(gamma.INSERTIONS) == int(g["n_ultralocal_gamma"])
    n_ul, n_dir = int(g["n_ultralocal_gamma"]), int(g["n_derivative_dirs"])
    assert 2 * (n_ul + n_dir * n_ul) == int(g["n_insertions"])
    idx = {contract.insertion_index(f, d, m, gi)
           for f in (0, 1) for gi in range(16)
           for d, ms in ((False, [0]), (True, range(4))) for m in ms}
    assert idx == set(range(160))


def test_momentum_cut_and_fig2_example():
    g = _golden()
    moms = momenta.momentum_list(int(g["p2_max"]))
    assert max(a * a + b * b + c * c for a, b, c in moms) == int(g["p2_max"])
    mask = [int(b) for b in g["fig2_mask"].split(",")]
    assert sum(m << k for k, m in enumerate(mask)) == int(g["fig2_sources"])
    assert float(g["rho_lp"]) > float(g["rho_hp"])
