"""Binary-weight storage of source sums (Sec. 2.1.1, Fig. 2).  TEST
INFRASTRUCTURE ONLY.

Files are weighted like the bits of a byte: the file of weight 2^k stores
the sum of the contractions of the 2^k sources 2^k .. 2^{k+1} - 1 (counting
sources from 1), so File.1 holds source 1, File.2 sources 2 and 3, File.4
sources 4 to 7.  N sources are recovered from the files whose weights are
the set bits of N (13 = 1 + 4 + 8: files 1, 4, 8); storage grows as log2 N.
Here sources are counted from 0 (source id = 1-based number - 1).
"""


def block_range(k):
    """0-based source ids [first, first + count) summed in the file of weight 2^k."""
    return (1 << k) - 1, 1 << k


def blocks_for(n):
    """The weights' exponents k whose files make up n sources (the set bits of n)."""
    return [k for k in range(n.bit_length()) if (n >> k) & 1]


def sources_for(n):
    """The 0-based source ids those files hold."""
    ids = []
    for k in blocks_for(n):
        first, count = block_range(k)
        ids.extend(range(first, first + count))
    return ids


def mean_from_blocks(block_sums, n):
    """Mean over n sources from per-block sums {k: sum}."""
    acc = 0
    for k in blocks_for(n):
        acc = acc + block_sums[k]
    return acc / n
