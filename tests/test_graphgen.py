"""The seeded input generators that both the oracle and the GPU path consume:
counter-based streams (a prefix of a stream is the smaller stream, thread
count does not matter), id ranges, and the R-MAT quadrant probabilities of
the recipe (a, b, c, d) = (.57, .19, .19, .05)."""
import numpy as np
import pytest

import graphgen as gg


def test_rmat_prefix_is_the_shorter_stream():
    s, d = gg.rmat(12, 16, 5)
    assert len(s) == 16 << 12
    for k in (1, 1000, 4096, 65535):
        ps, pd = gg.rmat(12, 16, 5, num_edges=k)
        assert np.array_equal(ps, s[:k]) and np.array_equal(pd, d[:k])


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_streams_do_not_depend_on_threads(threads):
    s0, d0 = gg.rmat(13, 16, 9, threads=1)
    s1, d1 = gg.rmat(13, 16, 9, threads=threads)
    assert np.array_equal(s0, s1) and np.array_equal(d0, d1)
    c0 = gg.chunglu(1 << 12, 2.1, 16.0, seed=4, threads=1)
    c1 = gg.chunglu(1 << 12, 2.1, 16.0, seed=4, threads=threads)
    assert np.array_equal(c0[0], c1[0]) and np.array_equal(c0[1], c1[1])


def test_ids_in_range_and_seeds_differ():
    n = 1 << 11
    s, d = gg.rmat(11, 16, 1)
    assert s.min() >= 0 and d.min() >= 0 and s.max() < n and d.max() < n
    s2, _ = gg.rmat(11, 16, 2)
    assert not np.array_equal(s, s2)
    cs, cd = gg.chunglu(3000, 2.5, 8.0, seed=3)
    assert len(cs) == gg.chunglu_num_edges(3000, 8.0)
    assert cs.min() >= 0 and cd.min() >= 0 and cs.max() < 3000 and cd.max() < 3000
    n16, es, ed = gg.er_16k()
    assert n16 == 16384 and len(es) == 262144 and es.max() < n16 and ed.max() < n16


def test_rmat_first_level_quadrants():
    # without the relabelling permutation the top id bit is the first
    # quadrant choice: P(src bit = 0) = a + b, P(dst bit = 0) = a + c
    scale, k = 16, 1 << 18
    s, d = gg.rmat(scale, 16, 11, permute=False, num_edges=k)
    top = 1 << (scale - 1)
    ps = np.mean(s < top)
    pd = np.mean(d < top)
    sd = np.sqrt(0.76 * 0.24 / k)
    assert abs(ps - 0.76) < 6 * sd and abs(pd - 0.76) < 6 * sd
    both = np.mean((s < top) & (d < top))  # quadrant a
    assert abs(both - 0.57) < 6 * np.sqrt(0.57 * 0.43 / k)


def test_batch_recipe():
    nv, ofs, s, d = gg.batch(64, seed=6)
    assert len(nv) == 64 and ofs[0] == 0 and ofs[-1] == len(s) == len(d)
    assert np.all(np.diff(ofs) >= 0)
    assert nv.min() >= 256 and nv.max() <= 65536
    for g in range(64):
        a, b = ofs[g], ofs[g + 1]
        if b > a:
            assert s[a:b].min() >= 0 and s[a:b].max() < nv[g]
            assert d[a:b].min() >= 0 and d[a:b].max() < nv[g]
    nv2, ofs2, s2, d2 = gg.batch(64, seed=6)
    assert np.array_equal(s, s2) and np.array_equal(ofs, ofs2)
