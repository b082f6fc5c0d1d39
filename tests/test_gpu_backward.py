"""Gradient of the weighted colourful count with respect to edge weights.

F(w) = sum_v g_v per_vertex[v](w), each colourful map contributing the
product of its k-1 edge weights.  A tree map uses an edge at most once, so F
is affine in each single weight: dF/dw_e = (F(w) - F(w with w_e = 0)) / w_e
exactly (the oracle computes both in exact dyadic arithmetic), central finite
differences are exact up to rounding for any step, and F is homogeneous of
degree k-1: sum over edges of w_e dF/dw_e = (k-1) F (Euler).
"""
from fractions import Fraction

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


def _exact_grad(g, w, parent, col, edges, seedv=None, num_colours=None):
    """dF/dw_e for the listed undirected edges, exact, from the oracle."""
    ids = si.arc_edge_ids(g)
    base = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, num_colours=num_colours, weights=w)
    bpv = base.per_vertex_values()
    F = sum(Fraction(float(s)) * x for s, x in zip(seedv, bpv)) if seedv is not None else base.total_value()
    out = {}
    for e in edges:
        w0 = w.copy()
        w0[ids == e] = 0.0
        r = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, num_colours=num_colours, weights=w0)
        F0 = sum(Fraction(float(s)) * x for s, x in zip(seedv, r.per_vertex_values())) if seedv is not None \
            else r.total_value()
        out[e] = (F - F0) / Fraction(float(w[ids == e][0]))
    return F, out


@pytest.mark.parametrize("parent", [si.TREE8.parent, (-1, 0, 1, 1), (-1, 0, 0, 0, 0), (-1, 0), (-1, 0, 1, 2, 2, 0)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_matches_exact_differences(sg, parent, prec):
    k = len(parent)
    g = si.chung_lu(600, 3000, 2.3, seed=3)
    w = si.arc_weights(g, si.edge_weights(g, seed=2))
    col = si.colouring(g.n, k, 6)
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(parent)
    grad = np.zeros(g.nnz)
    total = sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.PRECISIONS[prec], grad)
    edges = list(si.sample_indices(12, g.m, seed=k)) + [0, g.m - 1]
    F, exact = _exact_grad(g, w, parent, col, edges)
    tol = 1e-11 if prec == "fp64" else 1e-4
    assert abs(total - float(F)) <= tol * float(F)
    ids = si.arc_edge_ids(g)
    for e, want in exact.items():
        arcs = np.nonzero(ids == e)[0]
        for a in arcs:
            assert abs(grad[a] - float(want)) <= tol * max(abs(float(want)), 1e-300) + 1e-300, (e, grad[a], want)
    # Euler: sum over edges of w_e dF/dw_e = (k - 1) F (each edge appears on two arcs)
    euler = float(np.sum(w.astype(np.float64) * grad)) / 2.0
    assert euler == pytest.approx((k - 1) * float(F), rel=10 * tol)


def test_seeded_per_vertex_gradient_and_autograd(sg):
    import torch

    parent = (-1, 0, 1, 0)
    g = si.chung_lu(500, 2500, 2.3, seed=8)
    w = si.arc_weights(g, si.edge_weights(g, seed=4))
    col = si.colouring(g.n, 4, 9)
    seed = si.uniform53(5, 77, np.arange(g.n)) - 0.25
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(parent)
    grad = np.zeros(g.nnz)
    sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.SG2V_FP64, grad, seed)
    edges = list(si.sample_indices(8, g.m, seed=1))
    _, exact = _exact_grad(g, w, parent, col, edges, seedv=seed)
    ids = si.arc_edge_ids(g)
    for e, want in exact.items():
        for a in np.nonzero(ids == e)[0]:
            assert grad[a] == pytest.approx(float(want), rel=1e-9, abs=1e-9)
    # autograd through weighted_count
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    dcol = torch.from_numpy(col).cuda()
    pv = sg.weighted_count(wt, graph, plan, dcol, "fp64")
    (pv * torch.from_numpy(seed).cuda()).sum().backward()
    assert np.allclose(wt.grad.cpu().numpy(), grad.astype(np.float32), rtol=1e-5)


def test_unweighted_gradient_is_participation(sg):
    """On an unweighted graph dF/dw_e at w = 1 counts the colourful maps that
    use edge e; checked against brute force on a tiny graph."""
    parent = (-1, 0, 1)
    g = si.random_small_graph(9, 1, 2, 4)
    col = si.colouring(g.n, 3, 2)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(parent)
    grad = np.zeros(g.nnz)
    sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.SG2V_FP64, grad)
    ids = si.arc_edge_ids(g)
    full = oracle.brute(g.row_ptr, g.col_idx, parent, 0, col).total
    for e in range(g.m):
        w = np.ones(g.nnz, np.float32)
        w[ids == e] = 0.0
        without = oracle.brute(g.row_ptr, g.col_idx, parent, 0, col, weights=w).total_value()
        uses = full - without
        assert all(grad[a] == float(uses) for a in np.nonzero(ids == e)[0])


def test_chunglu200k_tree8_finite_differences(sg):
    """The differentiable workload: Chung-Lu 200k vertices, avg degree 20,
    gamma 2.3, weights in [0.5, 1.5), tree8, k = 8.  FP32 backward against
    central differences of the FP64 forward on 1,000 sampled edges (exact up
    to rounding because F is affine in each weight), plus Euler's identity."""
    import torch

    g = si.workload_graph("chunglu200k")
    w = si.arc_weights(g, si.edge_weights(g, seed=0))
    col = si.colouring(g.n, 8, 0)
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(si.TREE8.parent)
    dcol = torch.from_numpy(col).cuda()
    grad = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
    total32 = sg.sg2v_count_backward(graph.handle, plan.handle, dcol, sg.SG2V_FP32, grad)
    grad = grad.cpu().numpy()
    _, F64, _ = sg.count(graph, plan, dcol, "fp64", per_vertex=False)
    assert abs(total32 - F64) <= 1e-4 * F64
    ids = si.arc_edge_ids(g)
    first_arc = np.zeros(g.m, dtype=np.int64)
    first_arc[ids[::-1]] = np.arange(g.nnz)[::-1]
    edges = si.sample_indices(1000, g.m, seed=11)
    arcs_of = {}
    order = np.argsort(ids, kind="stable")
    pos = np.searchsorted(ids[order], edges)
    h = 0.25
    wt = torch.from_numpy(w).cuda()
    checked = 0
    for e, p0 in zip(edges, pos):
        a0, a1 = order[p0], order[p0 + 1]
        ww = wt.clone()
        ww[a0] += h
        ww[a1] += h
        sg.sg2v_graph_set_weights(graph.handle, ww)
        _, fp, _ = sg.count(graph, plan, dcol, "fp64", per_vertex=False)
        ww[a0] -= 2 * h
        ww[a1] -= 2 * h
        sg.sg2v_graph_set_weights(graph.handle, ww)
        _, fm, _ = sg.count(graph, plan, dcol, "fp64", per_vertex=False)
        fd = (fp - fm) / (2 * h)
        gv = grad[a0]
        assert grad[a1] == gv
        assert abs(gv - fd) <= 1e-4 * max(abs(fd), 1e-3 * F64 / g.m), (e, gv, fd)
        checked += 1
    assert checked == 1000
    sg.sg2v_graph_set_weights(graph.handle, wt)
    euler = float(np.sum(w.astype(np.float64) * grad)) / 2.0
    assert euler == pytest.approx(7 * F64, rel=1e-4)


@pytest.mark.parametrize("parent", [si.TREE8.parent, si.TREE10.parent, (-1, 0, 1, 2, 3), (-1, 0, 0, 0, 0),
                                    (-1, 0, 1, 1, 0, 4, 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_recompute_form_matches_stored_form(sg, parent, prec, monkeypatch):
    """The recompute form (tables rebuilt from the leaves during the reverse
    walk, Y' replayed) gives the stored form's gradients: bit for bit when no
    row is split (the chunk size here exceeds every degree), and holds less
    device memory at its peak."""
    import torch

    monkeypatch.setenv("SG2V_CHUNK", "100000")
    k = len(parent)
    g = si.chung_lu(2000, 12000, 2.3, seed=9)
    w = si.arc_weights(g, si.edge_weights(g, seed=4))
    col = torch.from_numpy(si.colouring(g.n, k, 2)).cuda()
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(parent)
    seedv = torch.from_numpy(np.linspace(0.25, 2.0, g.n)).cuda()
    out, peak = {}, {}
    for name, flag in (("store", sg.SG2V_BACKWARD_STORE), ("recompute", sg.SG2V_BACKWARD_RECOMPUTE)):
        gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        t = sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.PRECISIONS[prec], gw, seedv, flags=flag)
        peak[name] = sg.sg2v_last_call_peak_bytes()
        out[name] = (t, gw.cpu().numpy())
    if prec == "fp64":
        assert out["store"][0] == out["recompute"][0]
        assert np.array_equal(out["store"][1], out["recompute"][1])
    else:
        # FP32: the recompute form's forward total may use a root kernel form
        # with another summation order than the stored form's Y'-keeping one
        assert abs(out["store"][0] - out["recompute"][0]) <= 1e-4 * abs(out["store"][0])
        np.testing.assert_allclose(out["recompute"][1], out["store"][1], rtol=1e-4,
                                   atol=1e-4 * np.abs(out["store"][1]).max())
    assert 0 < peak["recompute"] < peak["store"]
    # flags = 0 picks a form; its gradients are the same
    gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
    sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.PRECISIONS[prec], gw, seedv)
    assert np.array_equal(gw.cpu().numpy(), out["store"][1]) or prec == "fp32"


def test_recompute_form_with_split_rows(sg, monkeypatch):
    """With rows split into chunks of 64 arcs (folded by atomic adds) the two
    forms agree to the FP64 bar, and both match exact differences of the
    oracle."""
    import torch

    monkeypatch.setenv("SG2V_CHUNK", "64")
    g = si.chung_lu(2000, 12000, 2.3, seed=5)
    w = si.arc_weights(g, si.edge_weights(g, seed=3))
    parent = si.TREE8.parent
    col = si.colouring(g.n, 8, 1)
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(parent)
    assert int(np.diff(g.row_ptr).max()) > 64
    res = {}
    for name, flag in (("store", sg.SG2V_BACKWARD_STORE), ("recompute", sg.SG2V_BACKWARD_RECOMPUTE)):
        gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        sg.sg2v_count_backward(graph.handle, plan.handle, torch.from_numpy(col).cuda(), sg.SG2V_FP64, gw, flags=flag)
        res[name] = gw.cpu().numpy()
    np.testing.assert_allclose(res["recompute"], res["store"], rtol=1e-12, atol=0)
    ids = si.arc_edge_ids(g)
    edges = [int(e) for e in si.sample_indices(12, g.m, seed=2)]
    _, exact = _exact_grad(g, w, parent, col, edges)
    for e in edges:
        for a in np.nonzero(ids == e)[0]:
            assert abs(res["recompute"][a] - float(exact[e])) <= 1e-12 * abs(float(exact[e])) + 1e-300


@pytest.mark.parametrize("parent,kc", [(si.TREE8.parent, 8), (si.TREE10.parent, 10), (si.TREE8.parent, 12),
                                       ((-1, 0, 1, 2, 3), 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sorted_per_arc_gradient_matches_row_form(sg, parent, kc, prec, monkeypatch):
    """The per-arc gradient over colour-sorted arcs (each result sent to its
    arc through the sort's permutation) equals the per-row form
    (SG2V_SDDMM_SORTED=0), with rows split into chunks of 64 arcs (the forward
    folds split rows with atomic adds, so FP64 agrees to rounding, not bit for
    bit), and matches exact differences of the oracle."""
    import torch

    monkeypatch.setenv("SG2V_CHUNK", "64")
    g = si.chung_lu(1500, 9000, 2.3, seed=11)
    assert int(np.diff(g.row_ptr).max()) > 64
    w = si.arc_weights(g, si.edge_weights(g, seed=5))
    col = si.colouring(g.n, kc, 4)
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(parent, num_colours=kc)
    res = {}
    for env in ("1", "0"):
        monkeypatch.setenv("SG2V_SDDMM_SORTED", env)
        gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        sg.sg2v_count_backward(graph.handle, plan.handle, torch.from_numpy(col).cuda(), sg.PRECISIONS[prec], gw)
        res[env] = gw.cpu().numpy()
    rtol = 1e-12 if prec == "fp64" else 1e-5
    np.testing.assert_allclose(res["1"], res["0"], rtol=rtol, atol=rtol * np.abs(res["0"]).max())
    ids = si.arc_edge_ids(g)
    edges = [int(e) for e in si.sample_indices(6, g.m, seed=kc)]
    _, exact = _exact_grad(g, w, parent, col, edges, num_colours=kc)
    tol = 1e-11 if prec == "fp64" else 1e-4
    for e in edges:
        for a in np.nonzero(ids == e)[0]:
            assert abs(res["1"][a] - float(exact[e])) <= tol * abs(float(exact[e])) + 1e-300, (e, res["1"][a])


@pytest.mark.parametrize("parent,kc", [(si.TREE8.parent, 8), (si.TREE10.parent, 10), (si.TREE8.parent, 12),
                                       ((-1, 0, 1, 2, 3), 5), ((-1, 0, 0, 0, 0), 5)])
@pytest.mark.parametrize("prec,weighted", [("fp32", True), ("fp32", False), ("fp64", False), ("fp64", True)])
def test_transposed_spmm_on_run_kernel(sg, parent, kc, prec, weighted, monkeypatch):
    """The transposed SpMM of the backward pass on the run-scatter kernel
    (colour runs of the neighbours' Ybar' rows scattered through the
    transposed run map into the gradient row) gives the gradients of the
    per-colour-accumulator form (SG2V_BWD_RUN=0), with rows split into
    chunks of 64 arcs: bit for bit for unweighted FP64 (integer
    participation counts), to rounding otherwise; and they match exact
    differences of the oracle (weighted) or exact participation counts."""
    import torch

    monkeypatch.setenv("SG2V_CHUNK", "64")
    g = si.chung_lu(1500, 9000, 2.3, seed=13)
    assert int(np.diff(g.row_ptr).max()) > 64
    w = si.arc_weights(g, si.edge_weights(g, seed=7)) if weighted else None
    col = si.colouring(g.n, kc, 6)
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(parent, num_colours=kc)
    res = {}
    for env in ("1", "0"):
        monkeypatch.setenv("SG2V_BWD_RUN", env)
        gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        sg.sg2v_count_backward(graph.handle, plan.handle, torch.from_numpy(col).cuda(), sg.PRECISIONS[prec], gw)
        res[env] = gw.cpu().numpy()
    if prec == "fp64" and not weighted:
        assert np.array_equal(res["1"], res["0"])
    else:
        rtol = 1e-12 if prec == "fp64" else 1e-5
        np.testing.assert_allclose(res["1"], res["0"], rtol=rtol, atol=rtol * np.abs(res["0"]).max())
    ids = si.arc_edge_ids(g)
    edges = [int(e) for e in si.sample_indices(6, g.m, seed=kc + 1)]
    ww = w if weighted else np.ones(g.nnz, dtype=np.float32)
    _, exact = _exact_grad(g, ww, parent, col, edges, num_colours=kc)
    tol = 1e-11 if prec == "fp64" else 1e-4
    for e in edges:
        for a in np.nonzero(ids == e)[0]:
            assert abs(res["1"][a] - float(exact[e])) <= tol * abs(float(exact[e])) + 1e-300, (e, res["1"][a])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_backward_on_column_panel_work_list(sg, prec, monkeypatch):
    """Gradients on a work list in column panels (rows cut at panel
    boundaries and into chunks of 64 arcs, read at graph creation) match
    exact differences of the oracle."""
    import torch

    monkeypatch.setenv("SG2V_PANELS", "2")
    monkeypatch.setenv("SG2V_CHUNK", "64")
    g = si.chung_lu(1500, 9000, 2.3, seed=17)
    w = si.arc_weights(g, si.edge_weights(g, seed=3))
    col = si.colouring(g.n, 8, 2)
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(si.TREE8.parent)
    gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
    sg.sg2v_count_backward(graph.handle, plan.handle, torch.from_numpy(col).cuda(), sg.PRECISIONS[prec], gw)
    got = gw.cpu().numpy()
    ids = si.arc_edge_ids(g)
    edges = [int(e) for e in si.sample_indices(8, g.m, seed=21)]
    _, exact = _exact_grad(g, w, si.TREE8.parent, col, edges)
    tol = 1e-11 if prec == "fp64" else 1e-4
    for e in edges:
        for a in np.nonzero(ids == e)[0]:
            assert abs(got[a] - float(exact[e])) <= tol * abs(float(exact[e])) + 1e-300, (e, got[a])
