"""Pins of the exact CPU oracle against things other than itself.

Paper: SubGraph2Vec (arXiv 2009.11665).  The oracle must give the number of
colourful labelled embeddings of a tree template (Sec. 2.2, Alg. 1).  Each
test below checks it against an independent route to that number: brute
force (C and pure Python), closed forms, invariants the definition implies,
or the exact expectation over all colourings.
"""
import itertools
from fractions import Fraction
from math import comb, factorial, prod

import networkx as nx
import numpy as np
import pytest

import sg2v_inputs as si
import oracle

SMALL_TREES = [
    (-1,),
    (-1, 0),
    (-1, 0, 1),
    (-1, 0, 0),
    (-1, 0, 1, 2),
    (-1, 0, 0, 0),
    (-1, 0, 1, 1),
    (-1, 0, 1, 2, 3),
    (-1, 0, 0, 1, 1),
    (-1, 0, 1, 0, 3),
    (-1, 0, 0, 0, 0),
    (-1, 0, 1, 2, 2, 0),
    (-1, 0, 0, 1, 2, 3),
]


def _run_all(g, parent, root, col, kc=None, weights=None):
    a = oracle.count(g.row_ptr, g.col_idx, parent, root, col, kc, weights, mode="decoupled", cut="last")
    b = oracle.count(g.row_ptr, g.col_idx, parent, root, col, kc, weights, mode="standard", cut="first")
    c = oracle.brute(g.row_ptr, g.col_idx, parent, root, col, kc, weights)
    return a, b, c


@pytest.mark.parametrize("parent", SMALL_TREES)
def test_dp_modes_match_brute_force(parent):
    """Alg. 3 (decoupled) and Alg. 2 (standard) equal enumeration (Sec. 6.7:
    identical in exact arithmetic), for every root and both cut orders."""
    k = len(parent)
    for seed in range(4):
        n = 6 + (seed * 3) % 7  # 6..12 vertices
        g = si.random_small_graph(n, 1, 2, seed)
        for kc in (k, k + 1):
            col = si.colouring(n, kc, seed)
            for root in range(k):
                a, b, c = _run_all(g, parent, root, col, kc)
                assert a.per_vertex == c.per_vertex, (parent, root, seed, kc)
                assert b.per_vertex == c.per_vertex, (parent, root, seed, kc)
                assert a.total == c.total == sum(c.per_vertex)


@pytest.mark.parametrize("parent", [(-1, 0, 1), (-1, 0, 0, 0), (-1, 0, 1, 1), (-1, 0, 1, 2)])
def test_against_pure_python_enumeration(parent):
    """A separately written enumerator over all vertex tuples (Python ints)."""
    k = len(parent)
    for seed in range(3):
        g = si.random_small_graph(6, 2, 3, seed + 10)
        col = si.colouring(6, k, seed)
        for root in range(k):
            per, tot = oracle.py_brute(6, g.edges.tolist(), parent, root, col.tolist())
            r = oracle.count(g.row_ptr, g.col_idx, parent, root, col)
            assert r.per_vertex == per
            assert r.total == tot


def test_weighted_against_pure_python_enumeration():
    """Weighted form: each embedding contributes the product of its edge
    weights (multilinear in the weights); exact dyadic arithmetic."""
    parent = (-1, 0, 1, 1)
    g = si.random_small_graph(6, 2, 3, 5)
    w_edge = si.edge_weights(g, seed=3)
    w_arc = si.arc_weights(g, w_edge)
    wmap = {(int(u), int(v)): Fraction(float(w)) for (u, v), w in zip(g.edges, w_edge)}
    col = si.colouring(6, 4, 7)
    per, tot = oracle.py_brute(6, g.edges.tolist(), parent, 0, col.tolist(), weights=wmap)
    for mode in ("decoupled", "standard"):
        r = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, weights=w_arc, mode=mode)
        assert r.total_value() == tot
        assert r.per_vertex_values() == per
    rb = oracle.brute(g.row_ptr, g.col_idx, parent, 0, col, weights=w_arc)
    assert rb.total_value() == tot


def test_wide_integers_beyond_128_bits():
    """Products of eight weights near 1.5 scaled by 2^24 exceed 2^128: the
    oracle must move to its wider build and stay exact."""
    parent = (-1, 0, 0, 0, 0, 0, 0, 0, 0)  # star with 8 leaves, k = 9
    n = 12
    g = si.complete_graph(n)
    w = np.full(g.nnz, np.float32(1.4999999), dtype=np.float32)
    col = (np.arange(n) % 9).astype(np.int8)
    r = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, weights=w)
    assert r.limbs > 2
    # closed form on K_n: every colourful map uses 8 edges of equal weight
    nc = np.bincount(col, minlength=9)
    colourful = factorial(9) * prod(int(x) for x in nc)
    assert r.total_value() == colourful * Fraction(float(np.float32(1.4999999))) ** 8


def test_star_closed_form():
    """Star with k-1 leaves rooted at its centre: per_vertex[v] equals
    (k-1)! * product over colours c != col(v) of (neighbours of v coloured c)."""
    for k in (3, 4, 5, 7):
        parent = (-1,) + (0,) * (k - 1)
        g = si.erdos_renyi(300, 2400, seed=k)
        col = si.colouring(g.n, k, seed=k)
        r = oracle.count(g.row_ptr, g.col_idx, parent, 0, col)
        for v in range(g.n):
            nb = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
            cnt = np.bincount(col[nb], minlength=k)
            expect = factorial(k - 1) * prod(int(cnt[c]) for c in range(k) if c != col[v])
            assert r.per_vertex[v] == expect


def test_star_expectation_closed_form():
    """Averaged over all colourings, the star's colourful count divided by
    (k-1)! equals sum_v C(deg v, k-1) * k!/k^k (each (k-1)-set of neighbours
    plus the centre is colourful with probability k!/k^k)."""
    k = 3
    parent = (-1, 0, 0)
    g = si.random_small_graph(6, 1, 2, 2)
    acc = Fraction(0)
    for col in itertools.product(range(k), repeat=g.n):
        acc += oracle.count(g.row_ptr, g.col_idx, parent, 0, np.array(col, np.int8)).total
    mean = acc / k ** g.n
    deg = g.degrees()
    expect = sum(comb(int(d), k - 1) for d in deg) * Fraction(factorial(k), k ** k) * factorial(k - 1)
    assert mean == expect


def test_path_on_path_graph_closed_form():
    """Path of k vertices rooted at an end, on a path graph: per_vertex[v] is
    the number of the (at most two) k-vertex windows starting at v whose
    colours are pairwise distinct."""
    for k in (2, 3, 5):
        parent = tuple([-1] + list(range(k - 1)))
        n = 40
        g = si.path_graph(n)
        col = si.colouring(n, k, seed=k)
        r = oracle.count(g.row_ptr, g.col_idx, parent, 0, col)
        for v in range(n):
            expect = 0
            for step in (1, -1):
                idx = [v + step * i for i in range(k)]
                if all(0 <= x < n for x in idx) and len({int(col[x]) for x in idx}) == k:
                    expect += 1
            assert r.per_vertex[v] == expect


@pytest.mark.parametrize("parent", [(-1, 0, 1, 1), (-1, 0, 1, 2, 3), (-1, 0, 0, 1, 1, 2, 2), (-1, 0, 1, 2, 0, 4, 4, 6)])
def test_complete_graph_closed_form(parent):
    """Any tree on K_n: total = k! * prod_c n_c and per_vertex[v] =
    (k-1)! * prod_{c != col v} n_c, with n_c the size of colour class c."""
    k = len(parent)
    g = si.complete_graph(11)
    col = si.colouring(11, k, seed=k)
    nc = np.bincount(col, minlength=k)
    r = oracle.count(g.row_ptr, g.col_idx, parent, 0, col)
    assert r.total == factorial(k) * prod(int(x) for x in nc)
    for v in range(11):
        assert r.per_vertex[v] == factorial(k - 1) * prod(int(nc[c]) for c in range(k) if c != col[v])


def _nx_tree(parent):
    t = nx.Graph()
    t.add_nodes_from(range(len(parent)))
    t.add_edges_from((i, p) for i, p in enumerate(parent) if p >= 0)
    return t


@pytest.mark.parametrize("parent", SMALL_TREES + [si.TREE7.parent, si.TREE8.parent, si.TREE10.parent])
def test_automorphisms_against_networkx(parent):
    """alpha (Alg. 1) against networkx's isomorphism matcher, and against the
    DP on G = T with every vertex a colour of its own (total = alpha)."""
    t = _nx_tree(parent)
    gm = nx.algorithms.isomorphism.GraphMatcher(t, t)
    expect = sum(1 for _ in gm.isomorphisms_iter())
    assert oracle.automorphisms(parent) == expect
    rp, ci = oracle.template_csr(parent)
    col = np.arange(len(parent), dtype=np.int8)
    assert oracle.count(rp, ci, parent, 0, col).total == expect


def test_known_automorphism_counts():
    assert oracle.automorphisms(si.PATH5.parent) == 2
    assert oracle.automorphisms(si.STAR7.parent) == factorial(6)
    assert oracle.automorphisms(si.TREE7.parent) == 8
    assert oracle.automorphisms(si.TREE15.parent) == 4


def _emb_by_edge_subsets(g, parent):
    """emb(T, G) by definition (Sec. 2.2.1): edge subsets of G forming a
    subgraph isomorphic to T."""
    t = _nx_tree(parent)
    k = len(parent)
    cnt = 0
    for es in itertools.combinations([tuple(e) for e in g.edges.tolist()], k - 1):
        h = nx.Graph()
        h.add_edges_from(es)
        if h.number_of_nodes() == k and nx.is_isomorphic(h, t):
            cnt += 1
    return cnt


@pytest.mark.parametrize("parent", [(-1, 0, 1), (-1, 0, 0, 0), (-1, 0, 1, 2), (-1, 0, 1, 1)])
def test_estimator_unbiased_over_all_colourings(parent):
    """Averaging finalCount (Alg. 1) over all kc^n colourings gives exactly
    emb(T, G) (Sec. 2.2.2): the estimator is unbiased."""
    k = len(parent)
    g = si.random_small_graph(6, 1, 2, 11)
    alpha = oracle.automorphisms(parent)
    emb = _emb_by_edge_subsets(g, parent)
    inj = oracle.brute(g.row_ptr, g.col_idx, parent, 0, injective_only=True).total
    assert inj == emb * alpha
    for kc in (k, k + 1):
        acc = Fraction(0)
        for col in itertools.product(range(kc), repeat=g.n):
            tot = oracle.count(g.row_ptr, g.col_idx, parent, 0, np.array(col, np.int8), kc).total
            acc += oracle.estimate(tot, k, alpha, kc)
        assert acc / kc ** g.n == emb


def test_seeded_convergence():
    """The mean of N seeded estimates lies within 4 sigma / sqrt(N) of
    emb(T, G) (sigma estimated from the sample)."""
    parent = (-1, 0, 1, 1)
    g = si.erdos_renyi(14, 30, seed=4)
    alpha = oracle.automorphisms(parent)
    emb = oracle.brute(g.row_ptr, g.col_idx, parent, 0, injective_only=True).total // alpha
    N = 400
    est = [float(oracle.estimate(oracle.count(g.row_ptr, g.col_idx, parent, 0, si.colouring(g.n, 4, 9, b)).total,
                                 4, alpha)) for b in range(N)]
    mean = np.mean(est)
    sd = np.std(est, ddof=1)
    assert abs(mean - emb) <= 4 * sd / np.sqrt(N)


def test_root_and_cut_independence():
    """The total does not depend on the root or the cut order; per-vertex
    counts do not depend on the cut order."""
    parent = si.TREE8.parent
    g = si.erdos_renyi(200, 900, seed=1)
    col = si.colouring(g.n, 8, 1)
    ref = oracle.count(g.row_ptr, g.col_idx, parent, 0, col)
    first = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, cut="first")
    assert first.per_vertex == ref.per_vertex
    for root in range(1, 8):
        assert oracle.count(g.row_ptr, g.col_idx, parent, root, col, per_vertex=False).total == ref.total


def test_affine_in_each_weight():
    """A tree embedding uses an edge at most once, so the weighted count is
    affine in each single weight: F(w_e = 2x) - F(w_e = x) = F(w_e = x) - F(w_e = 0)."""
    parent = (-1, 0, 1, 0)
    g = si.random_small_graph(8, 1, 2, 3)
    w = si.arc_weights(g, si.edge_weights(g, seed=2))
    col = si.colouring(g.n, 4, 3)
    ids = si.arc_edge_ids(g)
    for e in range(min(g.m, 5)):
        vals = []
        for x in (0.0, 0.75, 1.5):
            ww = w.copy()
            ww[ids == e] = np.float32(x)
            vals.append(oracle.count(g.row_ptr, g.col_idx, parent, 0, col, weights=ww).total_value())
        assert vals[2] - vals[1] == vals[1] - vals[0]


def test_isolated_and_empty_inputs():
    """Edge cases: graph without edges, single-vertex template, missing colour."""
    g = si.from_edges(5, [])
    col = np.array([0, 1, 1, 0, 1], np.int8)
    assert oracle.count(g.row_ptr, g.col_idx, (-1, 0), 0, col).total == 0
    r = oracle.count(g.row_ptr, g.col_idx, (-1,), 0, np.zeros(5, np.int8))
    assert r.per_vertex == [1] * 5  # single vertex: every vertex is one embedding
    g = si.complete_graph(6)
    col = np.zeros(6, np.int8)  # one colour used: nothing is colourful
    assert oracle.count(g.row_ptr, g.col_idx, (-1, 0, 1), 0, col).total == 0


def test_rejects_invalid_input():
    g = si.path_graph(4)
    col = np.array([0, 1, 2, 3], np.int8)
    with pytest.raises(ValueError):
        oracle.count(g.row_ptr, g.col_idx, (-1, 0, 1), 0, col)  # colour 3 >= k = 3
    with pytest.raises(ValueError):
        oracle.count(g.row_ptr, g.col_idx, (-1, -1, 1), 0, col % 3)  # two roots
    with pytest.raises(ValueError):
        oracle.count(g.row_ptr, g.col_idx, (1, 2, 0), 0, col % 3)  # a cycle, no root
