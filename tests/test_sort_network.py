"""Host-side check of the warp sort network that the sparsity row kernel runs (fe_sparsity.cu,
warp_bitonic_packed): 32 lanes holding E keys each, every merge of size k opening with a mirror
stage (element i against i ^ (k - 1)) followed by ascending half-cleaners, stages between lanes
exchanging with lane l ^ (stride / E).  The schedule is emulated lane by lane on random inputs,
with duplicates and padding, for every E the kernel instantiates; the result must be the sorted
input.  (A restatement of the index arithmetic, not shared code.)"""
import numpy as np
import pytest


def warp_sort(vals, E, nl=32):
    """The kernel's schedule on nl lanes (32: a warp; 16 or 8: each group of nl lanes of a warp,
    whose exchange masks all stay below nl so that the groups sort independently)."""
    v = vals.reshape(nl, E).copy()
    lanes = np.arange(nl)
    lg = E.bit_length() - 1
    k = 2
    while k <= nl * E:
        if k <= E:  # mirror stage inside a lane
            for h in range(E):
                ph = h ^ (k - 1)
                if h < ph:
                    a, b = v[:, h].copy(), v[:, ph].copy()
                    v[:, h], v[:, ph] = np.minimum(a, b), np.maximum(a, b)
        else:  # mirror stage between lanes: element h meets the partner's element E - 1 - h
            m = (k >> lg) - 1
            lower = (lanes & (k >> (lg + 1))) == 0
            o = v[lanes ^ m][:, ::-1]
            v = np.where(lower[:, None], np.minimum(v, o), np.maximum(v, o))
        j = k >> 2
        while j > 0:
            if j < E:
                for h in range(E):
                    if h & j == 0:
                        a, b = v[:, h].copy(), v[:, h | j].copy()
                        v[:, h], v[:, h | j] = np.minimum(a, b), np.maximum(a, b)
            else:
                m = j >> lg
                lower = (lanes & m) == 0
                o = v[lanes ^ m]
                v = np.where(lower[:, None], np.minimum(v, o), np.maximum(v, o))
            j >>= 1
        k <<= 1
    return v.reshape(-1)


@pytest.mark.parametrize("E", [1, 2, 4, 8, 16])
def test_network_sorts(E):
    rng = np.random.default_rng(E)
    for t in range(200):
        n = 32 * E
        x = rng.integers(0, 40 if t % 3 == 0 else 2**32 - 1, n, dtype=np.uint64)
        ncand = int(rng.integers(1, n + 1))
        x[ncand:] = 0xFFFFFFFF  # padding keys sort last, as in the kernel
        np.testing.assert_array_equal(warp_sort(x, E), np.sort(x))


@pytest.mark.parametrize("nl,Es", [(16, (1, 2, 4)), (8, (2, 4, 8))])
def test_lane_group_network_sorts_each_group(nl, Es):
    """The half-warp and quarter-warp variants (warp_bitonic_packed<E, 16> and <E, 8>: two or four
    rows per warp in the row kernel): run on a whole warp, each group of nl lanes ends sorted on
    its own and nothing crosses between groups."""
    rng = np.random.default_rng(nl)
    ng = 32 // nl
    for E in Es:
        for t in range(100):
            groups = []
            for _ in range(ng):
                x = rng.integers(0, 30 if t % 2 else 2**32 - 1, nl * E, dtype=np.uint64)
                x[int(rng.integers(0, nl * E + 1)):] = 0xFFFFFFFF  # a group may hold no row at all
                groups.append(x)
            lanes = np.concatenate(groups).reshape(32, E)  # lanes nl g .. nl g + nl - 1: row g
            for g, x in enumerate(groups):
                np.testing.assert_array_equal(warp_sort(lanes[nl * g:nl * g + nl].reshape(-1), E, nl=nl), np.sort(x))
        # every exchange mask of the group schedule (mirror stages (k >> lg) - 1, half-cleaners
        # j >> lg) is below nl, so lane l ^ mask stays in l's group
        lg = E.bit_length() - 1
        k = 2
        while k <= nl * E:
            assert k <= E or (k >> lg) - 1 < nl
            j = k >> 2
            while j > 0:
                assert j < E or (j >> lg) < nl
                j >>= 1
            k <<= 1


def test_packed_keys_rank_runs():
    """Packed keys (column << SH | candidate): after the sort, the first key of each run of equal
    columns marks the unique columns in ascending order, and every candidate's rank is the number
    of run starts before it."""
    rng = np.random.default_rng(9)
    E, SH = 8, 8
    for _ in range(50):
        ncand = int(rng.integers(1, 257))
        cols = rng.integers(0, 60, ncand)
        keys = np.full(32 * E, 0xFFFFFFFF, dtype=np.uint64)
        keys[:ncand] = (cols.astype(np.uint64) << SH) | np.arange(ncand, dtype=np.uint64)
        s = warp_sort(keys, E)
        valid = s != 0xFFFFFFFF
        c = s >> SH
        first = valid & np.concatenate([[True], c[1:] != c[:-1]])
        rank = np.cumsum(first) - 1
        uniq = c[first]
        np.testing.assert_array_equal(uniq, np.unique(cols))
        t = (s & ((1 << SH) - 1))[valid].astype(np.int64)
        np.testing.assert_array_equal(uniq[rank[valid]][np.argsort(t)], cols)
