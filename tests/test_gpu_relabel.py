"""Vertex relabelling inside sg2v_graph_create is invisible to the caller.

The device copy of a graph numbers its vertices by decreasing degree unless
SG2V_GRAPH_KEEP_ORDER is given.  Counting is invariant under relabelling
(Sec. 2.2: a subgraph count does not depend on vertex names), so a graph in
either order must give the same totals, the same per-vertex counts in the
caller's vertex order, and the same per-arc gradients in the caller's arc
order; weights set later (sg2v_graph_set_weights) must follow their arcs.
"""
import numpy as np
import pytest

import oracle
import sg2v_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as s

    return s


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("parent", [si.TREE10.parent, si.TREE7.parent, si.STAR7.parent, si.PATH5.parent])
def test_counts_in_caller_order(sg, parent):
    g = si.rmat(11, 16000, seed=4)
    k = len(parent)
    cols = si.colourings(g.n, k, 3, seed=2)
    refs = [oracle.count(g.row_ptr, g.col_idx, parent, 0, c) for c in cols]
    plan = sg.Plan(parent)
    out = {}
    for keep in (False, True):
        graph = sg.Graph(g.row_ptr, g.col_idx, keep_order=keep)
        pv, tot, _ = sg.count_batched(graph, [plan], _dev(cols), "fp64", per_vertex=True)
        out[keep] = (pv.cpu().numpy()[0], tot.cpu().numpy()[0])
    for b, ref in enumerate(refs):
        want = np.array(ref.per_vertex, dtype=np.float64)
        if ref.max_bits <= 53:
            assert np.array_equal(out[False][0][b], want)
            assert out[False][1][b] == float(ref.total)
        assert np.array_equal(out[False][0][b], out[True][0][b]) or ref.max_bits > 53
        np.testing.assert_allclose(out[False][0][b], want, rtol=1e-12)


def test_session_and_fp32_in_caller_order(sg):
    g = si.rmat(10, 8000, seed=9)
    cols = si.colourings(g.n, 7, 4, seed=5)
    plans = [sg.Plan(t.parent) for t in (si.TREE7, si.PATH7)]
    import torch

    res = {}
    for keep in (False, True):
        graph = sg.Graph(g.row_ptr, g.col_idx, keep_order=keep)
        ses = sg.Session(graph, plans, 4, "fp32", per_vertex=True)
        tot = torch.empty((2, 4), dtype=torch.float64, device="cuda")
        pv = torch.empty((2, 4, g.n), dtype=torch.float64, device="cuda")
        ses.run(_dev(cols), tot, None, pv)
        ses.sync()
        res[keep] = (tot.cpu().numpy(), pv.cpu().numpy())
        ses.close()
    for i, t in enumerate((si.TREE7, si.PATH7)):
        for b in range(4):
            ref = oracle.count(g.row_ptr, g.col_idx, t.parent, 0, cols[b])
            want = np.array(ref.per_vertex, dtype=np.float64)
            for keep in (False, True):
                got = res[keep][1][i, b]
                nz = want != 0
                assert np.all(got[~nz] == 0)
                assert np.all(np.abs(got[nz] - want[nz]) <= 1e-4 * want[nz])
                assert abs(res[keep][0][i, b] - float(ref.total)) <= 1e-4 * float(ref.total)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradients_in_caller_arc_order(sg, prec):
    import torch

    g = si.chung_lu(800, 4000, 2.3, seed=7)
    w = si.arc_weights(g, si.edge_weights(g, seed=1))
    col = si.colouring(g.n, 8, 3)
    plan = sg.Plan(si.TREE8.parent)
    seedv = np.linspace(0.5, 1.5, g.n)
    grads, tots = {}, {}
    for keep in (False, True):
        graph = sg.Graph(g.row_ptr, g.col_idx, w, keep_order=keep)
        gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        tots[keep] = sg.sg2v_count_backward(graph.handle, plan.handle, _dev(col), sg.PRECISIONS[prec], gw,
                                            _dev(seedv))
        grads[keep] = gw.cpu().numpy()
    rtol = 1e-12 if prec == "fp64" else 1e-4
    np.testing.assert_allclose(grads[False], grads[True], rtol=rtol, atol=rtol * np.abs(grads[True]).max())
    assert abs(tots[False] - tots[True]) <= rtol * abs(tots[True])
    # both arcs of an edge carry the edge's gradient, in the caller's arc order
    rev = np.empty(g.nnz, dtype=np.int64)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    for e in range(g.nnz):
        u, v = src[e], g.col_idx[e]
        lo, hi = g.row_ptr[v], g.row_ptr[v + 1]
        rev[e] = lo + np.searchsorted(g.col_idx[lo:hi], u)
    assert np.array_equal(grads[False], grads[False][rev])


def test_set_weights_follow_their_arcs(sg):
    g = si.chung_lu(600, 3000, 2.3, seed=2)
    w0 = si.arc_weights(g, si.edge_weights(g, seed=0))
    w1 = si.arc_weights(g, si.edge_weights(g, seed=11))
    col = si.colouring(g.n, 6, 1)
    plan = sg.Plan((-1, 0, 1, 1, 0, 4))
    ref = oracle.count(g.row_ptr, g.col_idx, (-1, 0, 1, 1, 0, 4), 0, col, weights=w1)
    graph = sg.Graph(g.row_ptr, g.col_idx, w0)
    sg.sg2v_graph_set_weights(graph.handle, _dev(w1))
    pv, tot, _ = sg.count(graph, plan, _dev(col), "fp64")
    want = np.array([float(x) for x in ref.per_vertex_values()])
    np.testing.assert_allclose(pv.cpu().numpy(), want, rtol=1e-12, atol=0)
    assert abs(tot - float(ref.total_value())) <= 1e-12 * float(ref.total_value())


def _with_isolated(g, extra: int, seed: int):
    """g with `extra` isolated vertices inserted at random places of the
    caller's vertex order (an R-MAT graph has isolated vertices of its own)."""
    rng = np.random.default_rng(seed)
    n2 = g.n + extra
    keep = np.sort(rng.choice(n2, size=g.n, replace=False))  # new id of each old vertex
    deg = np.zeros(n2, dtype=np.int64)
    deg[keep] = np.diff(g.row_ptr)
    rp = np.zeros(n2 + 1, dtype=np.int64)
    rp[1:] = np.cumsum(deg)
    ci = keep[g.col_idx].astype(np.int32)  # rows keep their order; ids stay increasing
    return n2, rp, ci


@pytest.mark.parametrize("prec", ["fp64", "fp32", "u64", "fp32_scaled"])
def test_isolated_vertices_skipped(sg, prec, monkeypatch):
    """Forward counting launches no task for isolated vertices (their table
    rows are neither written nor read) and reports them as zeros: the same
    totals and per-vertex counts as with every row run (SG2V_SKIP_EMPTY=0),
    and the oracle's.  Also with the deferred eMA, whose launch walks rows."""
    g0 = si.rmat(10, 6000, seed=3)
    n, rp, ci = _with_isolated(g0, 700, seed=1)
    assert np.sum(np.diff(rp) == 0) > 700
    cols = si.colourings(n, 10, 2, seed=8)
    plans = [sg.Plan(si.TREE10.parent), sg.Plan((-1,), num_colours=10)]
    graph = sg.Graph(rp, ci)
    res = {}
    for env in ({}, {"SG2V_SKIP_EMPTY": "0"}, {"SG2V_DEFER_EMA": "1"}):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        pv, tot, est = sg.count_batched(graph, plans, _dev(cols), prec, per_vertex=True)
        res[tuple(env)] = (pv.cpu().numpy(), tot.cpu().numpy(), est.cpu().numpy())
        for k in env:
            monkeypatch.delenv(k)
    iso = np.diff(rp) == 0
    for b in range(2):
        ref = oracle.count(rp, ci, si.TREE10.parent, 0, cols[b])
        want = np.array(ref.per_vertex, dtype=np.float64)
        for key, (pv, tot, _) in res.items():
            assert np.all(pv[0, b][iso] == 0), key
            nz = want != 0
            assert np.all(pv[0, b][~nz] == 0), key
            rtol = 1e-12 if prec in ("fp64", "u64") else 1e-4
            assert np.all(np.abs(pv[0, b][nz] - want[nz]) <= rtol * want[nz]), key
            assert abs(tot[0, b] - float(ref.total)) <= rtol * float(ref.total), key
            # a single-vertex template counts every vertex, isolated ones too
            assert tot[1, b] == float(n), key
            assert np.all(pv[1, b] == 1.0), key
    if prec in ("fp64", "u64"):
        base = res[()]
        for key, val in res.items():
            for x, y in zip(base, val):
                assert np.array_equal(x, y), key
