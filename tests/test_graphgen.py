"""The seeded input generators that feed both the oracle and the library.

They hold none of the method's arithmetic; these tests pin their recipes:
the graph model of Section 2 (directed, no self-loops, no multi-arcs,
positive integer weights, rows strictly increasing), exact sizes, the R-MAT
quadrant probabilities, the reciprocal fraction, the tie order of the top
in x out vertices, and determinism in the seed.
"""
import numpy as np
import pytest

import graphgen as gg


def check_model(g):
    t, h = g.arcs()
    assert np.all(t != h), "self-loop"
    for v in range(g.n):
        row = g.cols[g.offsets[v]:g.offsets[v + 1]]
        assert np.all(np.diff(row) > 0), "row not strictly increasing"
    assert g.cols.min(initial=0) >= 0 and g.cols.max(initial=0) < g.n


def same(a, b):
    return np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)


def test_csr_from_arcs_drops_loops_and_repeats():
    g = gg.csr_from_arcs(4, [2, 0, 0, 1, 3, 0, 2], [1, 3, 1, 1, 0, 3, 0])
    assert g.offsets.tolist() == [0, 2, 2, 4, 5]
    assert g.cols.tolist() == [1, 3, 0, 1, 0]


def test_erdos_renyi_exact_size_and_seeded():
    g = gg.erdos_renyi(2000, 16000, 1)
    assert g.n == 2000 and g.m == 16000
    check_model(g)
    assert same(g, gg.erdos_renyi(2000, 16000, 1))
    assert not same(g, gg.erdos_renyi(2000, 16000, 2))
    # uniform pairs: out- and in-degrees near 8 on average, no vertex far above
    assert g.out_degree().max() < 30 and g.in_degree().max() < 30
    with pytest.raises(ValueError):
        gg.erdos_renyi(3, 7, 1)


def test_rmat_quadrants_and_skew():
    scale, ef = 12, 8
    g = gg.rmat(scale, ef, 0.57, 0.19, 0.19, seed=5)
    assert g.n == 1 << scale and g.m <= ef * g.n
    check_model(g)
    assert same(g, gg.rmat(scale, ef, 0.57, 0.19, 0.19, seed=5))
    t, h = g.arcs()
    top = scale - 1
    tb = (t >> top) & 1
    hb = (h >> top) & 1
    # per bit: tail bit set with probability c + d, head bit with b + d, both with d;
    # removing repeats (mostly in the dense low-id corner) shifts these a little
    assert 0.20 < tb.mean() < 0.30
    assert 0.20 < hb.mean() < 0.30
    assert 0.03 < (tb & hb).mean() < 0.08
    # a is the largest quadrant: vertex 0 has the largest out- and in-degree
    assert g.out_degree().argmax() == 0 and g.in_degree().argmax() == 0
    assert g.out_degree().max() > 20 * g.out_degree().mean()


def test_add_reciprocal_fraction():
    g = gg.rmat(11, 8, seed=7)
    g2 = gg.add_reciprocal(g, 0.3, seed=7)
    check_model(g2)
    a1 = set(zip(*(x.tolist() for x in g.arcs())))
    a2 = set(zip(*(x.tolist() for x in g2.arcs())))
    assert a1 <= a2
    assert all((v, u) in a1 for (u, v) in a2 - a1)  # only reversed arcs are added
    recip = sum((v, u) in a2 for (u, v) in a1) / len(a1)
    base = sum((v, u) in a1 for (u, v) in a1) / len(a1)
    # every picked arc gains its reverse: reciprocity rises by about 0.3 of the rest
    want = base + 0.3 * (1 - base)
    assert abs(recip - want) < 0.02, (recip, want)
    assert same(g2, gg.add_reciprocal(g, 0.3, seed=7))


def test_uniform_weights():
    w = gg.uniform_weights(100000, 1, 255, 3)
    assert w.dtype == np.uint32 and w.min() == 1 and w.max() == 255
    assert abs(w.mean() - 128.0) < 1.0
    assert np.array_equal(w, gg.uniform_weights(100000, 1, 255, 3))
    assert not np.array_equal(w, gg.uniform_weights(100000, 1, 255, 4))


def test_random_and_top_vertices():
    r = gg.random_vertices(1000, 500, 103)
    assert r.min() >= 0 and r.max() < 1000
    assert np.array_equal(r, gg.random_vertices(1000, 500, 103))
    g = gg.rmat(10, 4, seed=3)
    top = gg.top_inout_vertices(g, 40).tolist()
    ind, outd = g.in_degree(), g.out_degree()
    brute = sorted(range(g.n), key=lambda v: (-int(ind[v]) * int(outd[v]), v))[:40]
    assert top == brute
    # ties broken by ascending id
    prod = [int(ind[v]) * int(outd[v]) for v in top]
    for i in range(1, len(top)):
        assert prod[i - 1] > prod[i] or (prod[i - 1] == prod[i] and top[i - 1] < top[i])


def test_zipf_vertices():
    z = gg.zipf_vertices(5000, 20000, 1.1, 106)
    assert z.min() >= 0 and z.max() < 5000
    assert np.array_equal(z, gg.zipf_vertices(5000, 20000, 1.1, 106))
    counts = np.bincount(z, minlength=5000)
    perm = gg.rng(106).permutation(5000)
    # rank 1 is the most popular, and rank 1 / rank 2 frequencies follow 2^s
    assert counts.argmax() == perm[0]
    ratio = counts[perm[0]] / counts[perm[1]]
    assert 1.6 < ratio < 2.8, ratio
