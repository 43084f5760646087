"""Pins of the binary-weight storage definition (Sec. 2.1.1, Fig. 2)."""
import numpy as np

from oracle import binstore


def test_figure_example_13_sources():
    # the paper's example: weights 1 2 4 8 with mask 1 0 1 1 make 13
    assert binstore.blocks_for(13) == [0, 2, 3]
    assert len(binstore.sources_for(13)) == 13


def test_blocks_partition_consecutive_sources():
    seen = []
    for k in range(8):
        first, count = binstore.block_range(k)
        assert first == len(seen) and count == 2 ** k
        seen.extend(range(first, first + count))
    assert seen == list(range(2 ** 8 - 1))


def test_any_n_is_n_distinct_sources():
    for n in range(1, 300):
        ids = binstore.sources_for(n)
        assert len(ids) == n == len(set(ids))
        assert max(ids) < 2 ** n.bit_length() - 1  # within the blocks that must exist
    assert binstore.sources_for(2 ** 10 - 1) == list(range(2 ** 10 - 1))


def test_mean_from_blocks_equals_direct_mean():
    rng = np.random.default_rng(3)
    per_source = rng.standard_normal((255, 5))
    blocks = {k: per_source[binstore.block_range(k)[0]:sum(binstore.block_range(k))].sum(axis=0)
              for k in range(8)}
    for n in (1, 2, 3, 7, 13, 100, 255):
        want = per_source[binstore.sources_for(n)].mean(axis=0)
        assert np.allclose(binstore.mean_from_blocks(blocks, n), want, rtol=1e-14, atol=1e-14)
