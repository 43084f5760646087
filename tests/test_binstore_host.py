"""Binary-weight storage (Sec. 2.1.1, Fig. 2), host side, against the
oracle's definition: block ranges, any-N means (bit-exact: same additions in
the same order), resume after an interruption, and refusal of damaged files.
Only host calls of the library run here (no GPU)."""
import os
import shutil

import numpy as np
import pytest

from oracle import binstore as obs
from paper_1401_6750_gb300 import abi, build

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="CUDA toolkit needed to build the library")


@pytest.fixture(scope="module")
def api_mod():
    build.build()
    from paper_1401_6750_gb300 import api
    return api


def _blocks(n_values, k_max, seed=5):
    rng = np.random.default_rng(seed)
    per_source = rng.standard_normal((2 ** k_max - 1, n_values))
    sums = {k: per_source[obs.block_range(k)[0]:sum(obs.block_range(k))].sum(axis=0) for k in range(k_max)}
    return per_source, sums


def test_block_ranges_match_definition(api_mod):
    for k in range(12):
        assert api_mod.BinStore.block(k) == obs.block_range(k)


def test_any_n_mean_bit_exact(api_mod, tmp_path):
    n_values = 37
    per_source, sums = _blocks(n_values, 6)
    st = api_mod.BinStore(tmp_path / "loops", n_values)
    for k in range(6):
        st.put(k, sums[k])
    assert st.sources == 63
    for n in range(1, 64):
        got = st.mean(n)
        assert np.array_equal(got, obs.mean_from_blocks(sums, n)), n
        assert np.allclose(got, per_source[obs.sources_for(n)].mean(axis=0), rtol=1e-13, atol=1e-13)
    st.close()
    # storage: log2 N files for N sources
    files = [f for f in os.listdir(tmp_path) if f.endswith(".bin")]
    assert len(files) == 6


def test_resume_and_gaps(api_mod, tmp_path):
    n_values = 8
    _, sums = _blocks(n_values, 4, seed=6)
    st = api_mod.BinStore(tmp_path / "run", n_values)
    for k in (0, 1, 3):
        st.put(k, sums[k])
    assert st.sources == 3  # blocks 0 and 1 are contiguous, block 2 missing
    st.close()
    st = api_mod.BinStore(tmp_path / "run", n_values)  # reopen: same state
    assert st.sources == 3
    with pytest.raises(abi.TsmError):
        st.mean(7)  # needs block 2
    assert np.array_equal(st.mean(3), obs.mean_from_blocks(sums, 3))
    assert np.array_equal(st.mean(9), obs.mean_from_blocks(sums, 9))  # blocks 0 and 3
    st.put(2, sums[2])
    assert st.sources == 15
    st.close()


def test_damaged_files_are_refused(api_mod, tmp_path):
    n_values = 16
    _, sums = _blocks(n_values, 3, seed=7)
    st = api_mod.BinStore(tmp_path / "d", n_values)
    for k in range(3):
        st.put(k, sums[k])
    st.close()
    path = str(tmp_path / "d") + ".w4.bin"
    data = bytearray(open(path, "rb").read())
    data[-3] ^= 0x40  # flip one bit of a value
    open(path, "wb").write(bytes(data))
    with pytest.raises(abi.TsmError):
        api_mod.BinStore(tmp_path / "d", n_values)
    open(path, "wb").write(bytes(data[:-8]))  # truncated
    with pytest.raises(abi.TsmError):
        api_mod.BinStore(tmp_path / "d", n_values)
    os.remove(path)
    with pytest.raises(abi.TsmError):
        api_mod.BinStore(tmp_path / "d", n_values + 1)  # blocks of another size
    st = api_mod.BinStore(tmp_path / "d", n_values)
    assert st.sources == 3
    st.close()
