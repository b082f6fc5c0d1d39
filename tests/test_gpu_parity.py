"""Parity of the CUDA path (through the C ABI) with the exact CPU oracle.

Bars (colour-coding counts, SubGraph2Vec Alg. 1-5):
  FP64 tables: bit-exact when every table entry is below 2^53 (the oracle
               reports the largest entry), else relative error <= 1e-12;
  FP32 tables: relative error <= 1e-4 on totals and on every non-zero
               per-vertex count, zeros exact;
  estimate:    within 2 ulp of the exact rational total / (P alpha).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import sg2v_inputs as si

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FP32_RTOL = 1e-4
FP64_RTOL = 1e-12


@pytest.fixture(scope="module")
def sg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as s

    return s


def _dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _check_fp64(got_pv, got_total, ref, exact):
    want = np.array([float(x) for x in ref.per_vertex_values()], dtype=np.float64)
    if exact:
        assert np.array_equal(got_pv, want)
        assert got_total == float(ref.total_value())
    else:
        nz = want != 0
        assert np.all(got_pv[~nz] == 0)
        rel = np.abs(got_pv[nz] - want[nz]) / want[nz]
        assert rel.size == 0 or rel.max() <= FP64_RTOL, rel.max()
        tv = float(ref.total_value())
        assert abs(got_total - tv) <= FP64_RTOL * abs(tv)


def _check_fp32(got_pv, got_total, ref):
    want = np.array([float(x) for x in ref.per_vertex_values()], dtype=np.float64)
    nz = want != 0
    assert np.all(got_pv[~nz] == 0)
    if nz.any():
        rel = np.abs(got_pv[nz] - want[nz]) / want[nz]
        assert rel.max() <= FP32_RTOL, rel.max()
    tv = float(ref.total_value())
    assert abs(got_total - tv) <= FP32_RTOL * abs(tv)


def _ulp_close(a: float, exact: Fraction, ulps: int = 2) -> bool:
    b = float(exact)
    return abs(a - b) <= ulps * np.spacing(abs(b)) + 0.0


def _run(sg, g, parent, root, col, kc=None, weights=None):
    graph = sg.Graph(g.row_ptr, g.col_idx, weights)
    plan = sg.Plan(parent, root, kc)
    ref = oracle.count(g.row_ptr, g.col_idx, parent, root, col, kc, weights)
    dcol = _dev(col)
    pv64, t64, e64 = sg.count(graph, plan, dcol, "fp64")
    pv32, t32, e32 = sg.count(graph, plan, dcol, "fp32")
    return ref, plan, (pv64.cpu().numpy(), t64, e64), (pv32.cpu().numpy(), t32, e32)


def test_er2000_path5_fp64_bit_exact(sg):
    """The small workload: ER n=2000 avg degree 8, path of 5 rooted at an end,
    k = 5, one colouring."""
    g = si.workload_graph("er2000")
    col = si.colouring(g.n, 5, 0)
    ref, plan, r64, r32 = _run(sg, g, si.PATH5.parent, 0, col)
    assert ref.max_bits <= 53
    _check_fp64(r64[0], r64[1], ref, exact=True)
    assert _ulp_close(r64[2], oracle.estimate(ref.total, 5, plan.alpha))
    _check_fp32(r32[0], r32[1], ref)


TEMPLATES = [(-1, 0), (-1, 0, 1), (-1, 0, 0), (-1, 0, 1, 1), (-1, 0, 0, 0), si.PATH5.parent, si.TREE7.parent,
             si.STAR7.parent, si.PATH7.parent, si.TREE8.parent, (-1, 0, 1, 2, 2, 0), (-1, 0, 0, 1, 2, 3)]


@pytest.mark.parametrize("parent", TEMPLATES)
def test_templates_on_random_graphs(sg, parent):
    """Every template shape, several roots and colour counts, on graphs whose
    vertex counts span several warps' worth of rows and end ragged."""
    k = len(parent)
    for seed, (n, m) in enumerate([(333, 1400), (1531, 9000)]):
        g = si.erdos_renyi(n, m, seed=seed + 3)
        for kc in (k, min(16, k + 2)):
            for root in sorted({0, k - 1, k // 2}):
                col = si.colouring(n, kc, seed, root)
                ref, plan, r64, r32 = _run(sg, g, parent, root, col, kc)
                _check_fp64(r64[0], r64[1], ref, exact=ref.max_bits <= 53)
                _check_fp32(r32[0], r32[1], ref)
                assert _ulp_close(r64[2], oracle.estimate(ref.total, k, plan.alpha, kc))


def _hub_graph(seed: int):
    """R-MAT base plus three hubs joined to thousands of vertices."""
    base = si.rmat(13, 60000, seed=seed)
    extra = []
    for h, cnt in ((11, 5000), (4000, 3100), (8000, 1500)):
        others = si.sample_indices(cnt, base.n, seed=seed + h)
        extra += [(h, int(o)) for o in others if int(o) != h]
    edges = {tuple(e) for e in base.edges.tolist()} | {(min(a, b), max(a, b)) for a, b in extra}
    return si.from_edges(base.n, sorted(edges), "rmat13_hubs")


@pytest.mark.parametrize("chunk", ["1024", "64"])
def test_split_rows_power_law(sg, chunk, monkeypatch):
    """Rows longer than the row chunk are split across warps (partial sums
    folded by the last chunk); the chunk length is read at graph creation."""
    monkeypatch.setenv("SG2V_CHUNK", chunk)
    g = _hub_graph(5)
    assert g.degrees().max() > 4 * int(chunk)
    col = si.colouring(g.n, 7, 2)
    for parent in (si.TREE7.parent, si.PATH7.parent, si.STAR7.parent):
        ref, plan, r64, r32 = _run(sg, g, parent, 0, col)
        _check_fp64(r64[0], r64[1], ref, exact=ref.max_bits <= 53)
        _check_fp32(r32[0], r32[1], ref)


def test_weighted_graph(sg):
    """Weighted form: products of FP32 edge weights; exact dyadic oracle."""
    g = si.chung_lu(3000, 20000, 2.3, seed=1)
    w = si.arc_weights(g, si.edge_weights(g, seed=1))
    col = si.colouring(g.n, 8, 4)
    ref, plan, r64, r32 = _run(sg, g, si.TREE8.parent, 0, col, weights=w)
    _check_fp64(r64[0], r64[1], ref, exact=False)
    _check_fp32(r32[0], r32[1], ref)


@pytest.mark.parametrize("chunk", ["1024", "64"])
@pytest.mark.parametrize("hist", ["", "0"])
def test_weighted_split_rows(sg, chunk, hist, monkeypatch):
    """Weighted graphs whose hub rows are split across warps: the (2, 1, 1)
    table summed from the sorted arcs' weights (with SG2V_SORT_HIST=0: by the
    node kernels), split chunks adding into zeroed rows, equals the exact
    dyadic oracle in FP64 and FP32, up to 16 colours."""
    monkeypatch.setenv("SG2V_CHUNK", chunk)
    if hist:
        monkeypatch.setenv("SG2V_SORT_HIST", hist)
    g = _hub_graph(11)
    assert g.degrees().max() > 4 * int(chunk)
    w = si.arc_weights(g, si.edge_weights(g, seed=6))
    for parent, colours in ((si.TREE7.parent, (7, 12)), ((-1, 0, 1), (3, 16)), (si.PATH5.parent, (5, 16))):
        for kc in colours:
            col = si.colouring(g.n, kc, 3)
            ref, plan, r64, r32 = _run(sg, g, parent, 0, col, kc, weights=w)
            _check_fp64(r64[0], r64[1], ref, exact=False)
            _check_fp32(r32[0], r32[1], ref)


@pytest.mark.parametrize("wave", ["", "1", "2"])
def test_batched_templates_and_colourings(sg, wave, monkeypatch):
    """Several colourings x several templates in one call equal one oracle
    run per (template, colouring), whatever the number of colourings that
    share a table row (the wave width; read at each call)."""
    import torch

    if wave:
        monkeypatch.setenv("SG2V_WAVE", wave)

    g = si.rmat(12, 30000, seed=7)
    B = 5
    cols = si.colourings(g.n, 7, B, seed=3)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    temps = [si.PATH7, si.STAR7, si.TREE7]
    plans = [sg.Plan(t.parent) for t in temps]
    dcols = _dev(cols)
    for prec in ("fp64", "fp32"):
        pv, tot, est = sg.count_batched(graph, plans, dcols, prec, per_vertex=True)
        pv, tot, est = pv.cpu().numpy(), tot.cpu().numpy(), est.cpu().numpy()
        for i, t in enumerate(temps):
            for b in range(B):
                ref = oracle.count(g.row_ptr, g.col_idx, t.parent, 0, cols[b])
                if prec == "fp64":
                    _check_fp64(pv[i, b], tot[i, b], ref, exact=ref.max_bits <= 53)
                    assert _ulp_close(est[i, b], oracle.estimate(ref.total, 7, plans[i].alpha))
                else:
                    _check_fp32(pv[i, b], tot[i, b], ref)


def test_host_buffers_match_device_buffers(sg):
    """Host (numpy) colours and outputs take the copy path and agree."""
    g = si.erdos_renyi(2500, 12000, seed=9)
    col = si.colouring(g.n, 6, 1)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan((-1, 0, 1, 1, 0, 4))
    pv_dev, t_dev, e_dev = sg.count(graph, plan, _dev(col), "fp64")
    pv_host = np.zeros(g.n, dtype=np.float64)
    t_host, e_host = sg.sg2v_count(graph.handle, plan.handle, col, sg.SG2V_FP64, pv_host)
    assert np.array_equal(pv_dev.cpu().numpy(), pv_host)
    assert t_dev == t_host and e_dev == e_host


def test_single_vertex_and_edge_templates(sg):
    g = si.erdos_renyi(500, 2000, seed=2)
    for parent, kc in (((-1,), 1), ((-1,), 3), ((-1, 0), 2), ((-1, 0), 4)):
        col = si.colouring(g.n, kc, 5)
        ref, plan, r64, r32 = _run(sg, g, parent, 0, col, kc)
        _check_fp64(r64[0], r64[1], ref, exact=True)
        _check_fp32(r32[0], r32[1], ref)


def test_isolated_vertices_and_empty_rows(sg):
    """Rows with no arcs still produce (zero) rows; a graph without edges
    counts nothing for k >= 2."""
    g = si.from_edges(100, [(0, 1), (1, 2), (2, 3), (50, 51)])
    col = (np.arange(100) % 4).astype(np.int8)
    ref, plan, r64, r32 = _run(sg, g, (-1, 0, 1, 2), 0, col)
    _check_fp64(r64[0], r64[1], ref, exact=True)
    g = si.from_edges(10, [])
    col = np.zeros(10, np.int8)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    pv, t, e = sg.count(graph, sg.Plan((-1, 0), 0, 2), _dev(col), "fp64")
    assert t == 0 and not pv.any()


def test_colour_out_of_range_is_reported(sg):
    g = si.erdos_renyi(200, 600, seed=1)
    col = si.colouring(g.n, 4, 1)
    col[17] = 4
    graph = sg.Graph(g.row_ptr, g.col_idx)
    with pytest.raises(sg.Sg2vError) as e:
        sg.count(graph, sg.Plan((-1, 0, 1, 2)), _dev(col), "fp64")
    assert e.value.status == sg.SG2V_ERR_COLOUR_OUT_OF_RANGE
    col[17] = -1
    with pytest.raises(sg.Sg2vError) as e:
        sg.count(graph, sg.Plan((-1, 0, 1, 2)), _dev(col), "fp32")
    assert e.value.status == sg.SG2V_ERR_COLOUR_OUT_OF_RANGE


def test_full_size_rmat20_tree10(sg):
    """The 1M-vertex workload (R-MAT scale 20, 2^24 edges, tree10, k = 10):
    total and 4,000+ sampled per-vertex counts against stored oracle values
    (tests/golden, written by make_golden.py from the oracle only)."""
    import torch

    gold = json.load(open(os.path.join(HERE, "golden", "rmat20_16m_tree10_k10.json")))
    g = si.workload_graph(gold["graph"])
    import hashlib

    h = hashlib.sha256()
    h.update(g.row_ptr.tobytes())
    h.update(g.col_idx.tobytes())
    assert h.hexdigest() == gold["graph_sha256"], "generator did not rebuild the stored graph"
    col = si.colouring(g.n, gold["num_colours"], gold["colouring_seed"], gold["colouring_index"])
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(gold["template"], gold["root"], gold["num_colours"])
    idx = np.array(gold["sample_vertices"])
    want = np.array([float(int(x)) for x in gold["sample_counts"]])
    total = int(gold["total"])
    dcol = _dev(col)
    for prec, tol in (("fp64", FP64_RTOL), ("fp32", FP32_RTOL)):
        pv, t, e = sg.count(graph, plan, dcol, prec)
        got = pv.cpu().numpy()[idx]
        nz = want != 0
        assert np.all(got[~nz] == 0)
        assert (np.abs(got[nz] - want[nz]) / want[nz]).max() <= tol
        assert abs(t - total) <= tol * total
        assert float(e) == pytest.approx(float(oracle.estimate(total, 10, plan.alpha)), rel=tol)
        # the per-vertex counts are the total's parts
        assert float(pv.sum()) == pytest.approx(t, rel=1e-9)
        del pv
        torch.cuda.empty_cache()


SYMMETRIC_ROOTS = [si.TREE10.parent, (-1, 0, 0, 2), (-1, 0, 1, 0, 3, 4)]


@pytest.mark.parametrize("parent", SYMMETRIC_ROOTS)
@pytest.mark.parametrize("chunk", ["1024", "64"])
def test_totals_with_symmetric_root(sg, parent, chunk, monkeypatch):
    """Totals only, root whose active and passive children are one table:
    each edge is gathered from its lower end and the row sums doubled.  The
    totals must equal the oracle's under the usual bars, with and without
    colours beyond k, split rows included, and equal the per-vertex path."""
    monkeypatch.setenv("SG2V_CHUNK", chunk)
    g = _hub_graph(3)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    k = len(parent)
    for kc in (k, k + 1):
        plan = sg.Plan(parent, 0, kc)
        cols = si.colourings(g.n, kc, 3, seed=4)
        refs = [oracle.count(g.row_ptr, g.col_idx, parent, 0, cols[b], kc, per_vertex=False) for b in range(3)]
        for prec in ("fp64", "fp32"):
            _, tot, est = sg.count_batched(graph, [plan], _dev(cols), prec, per_vertex=False)
            pv, tot_pv, _ = sg.count_batched(graph, [plan], _dev(cols), prec, per_vertex=True)
            tot, tot_pv = tot.cpu().numpy()[0], tot_pv.cpu().numpy()[0]
            for b, ref in enumerate(refs):
                if prec == "fp64" and ref.max_bits <= 52:
                    assert tot[b] == float(ref.total) == tot_pv[b]
                else:
                    tol = FP64_RTOL if prec == "fp64" else FP32_RTOL
                    assert abs(tot[b] - ref.total) <= tol * ref.total
                    assert abs(tot_pv[b] - ref.total) <= tol * ref.total


@pytest.mark.parametrize("seed", range(4))
def test_min_work_plans_match_oracle(sg, seed):
    """Counts do not depend on the cut order (Sec. 2.3.2): plans built with
    the work-minimising cuts equal the oracle (FP64 bit-exact)."""
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(4, 10))
    parent = [-1] + [int(rng.integers(0, i)) for i in range(1, k)]
    parents = [tuple(parent), si.TREE10.parent] if seed == 0 else [tuple(parent)]
    g = si.rmat(11, 10000, seed=seed)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    for par in parents:
        kk = len(par)
        plan = sg.Plan(par, 0, kk, cut="min_work", avg_degree=16.0)
        col = si.colouring(g.n, kk, seed)
        ref = oracle.count(g.row_ptr, g.col_idx, par, 0, col)
        pv, tot, _ = sg.count(graph, plan, _dev(col), "fp64")
        _check_fp64(pv.cpu().numpy(), tot, ref, exact=ref.max_bits <= 53)


@pytest.mark.parametrize("knob", ["SG2V_HIST_ROWS", "SG2V_GROUP_ROWS", "SG2V_HALF_ROOT", "SG2V_ROOT_PAIRS",
                                  "SG2V_SORT_HIST", "SG2V_SORT_COUNTS", "SG2V_RUN_KERNEL", "SG2V_PRED_LANES",
                                  "SG2V_RUN_NARROW", "SG2V_SKIP_EMPTY"])
def test_alternative_kernel_forms(sg, knob, monkeypatch):
    """The forms that the 32-row histogram kernel, the lane-group kernel, the
    half-arc root, the paired root sum, the sort-written (2, 1, 1) table, the
    run-scatter kernel (for every row width, or for narrow rows), the FP32
    gathers without lane predicates and the skipping of isolated vertices
    replace on unweighted graphs (they still serve weighted graphs, long
    tasks, other table types and roots with several output sets) equal the
    oracle."""
    monkeypatch.setenv(knob, "0")
    g = _hub_graph(9)
    for parent in (si.TREE10.parent, si.TREE7.parent, si.PATH7.parent, (-1, 0, 0, 2)):
        k = len(parent)
        col = si.colouring(g.n, k, 5)
        ref, plan, r64, r32 = _run(sg, g, parent, 0, col)
        _check_fp64(r64[0], r64[1], ref, exact=ref.max_bits <= 53)
        _check_fp32(r32[0], r32[1], ref)
        graph = sg.Graph(g.row_ptr, g.col_idx)
        _, tot, _ = sg.count_batched(graph, [plan], _dev(col[None, :]), "fp64", per_vertex=False)
        t = float(tot.cpu().numpy()[0, 0])
        if ref.max_bits <= 52:
            assert t == float(ref.total)
        else:
            assert abs(t - ref.total) <= FP64_RTOL * ref.total


def test_split_rows_in_waves(sg, monkeypatch):
    """Split rows (chunks of 64 arcs) with two colourings per wave: every
    chunk adds its partial counts, for each colouring of the wave, into the
    same table rows (the sort-written (2,1,1) table and the scratch rows of
    the gathering nodes)."""
    monkeypatch.setenv("SG2V_CHUNK", "64")
    monkeypatch.setenv("SG2V_WAVE", "2")
    g = _hub_graph(3)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    B = 3
    cols = si.colourings(g.n, 7, B, seed=8)
    plans = [sg.Plan(t.parent) for t in (si.TREE7, si.PATH7)]
    for prec in ("fp64", "u64"):
        pv, tot, _ = sg.count_batched(graph, plans, _dev(cols), prec, per_vertex=True)
        pv, tot = pv.cpu().numpy(), tot.cpu().numpy()
        for i, t in enumerate((si.TREE7, si.PATH7)):
            for b in range(B):
                ref = oracle.count(g.row_ptr, g.col_idx, t.parent, 0, cols[b])
                if prec == "u64" or ref.max_bits <= 53:
                    assert np.array_equal(pv[i, b], np.array([float(int(x)) for x in ref.per_vertex]))
                    assert tot[i, b] == float(int(ref.total))
                else:
                    _check_fp64(pv[i, b], tot[i, b], ref, exact=False)


@pytest.mark.parametrize("panels", ["2", "4"])
@pytest.mark.parametrize("chunk", ["1024", "64"])
def test_column_panel_work_lists(sg, panels, chunk, monkeypatch):
    """Work lists in column panels (the CSC-Split form, Alg. 6: rows of more
    than 64 arcs cut where their neighbours cross into the next range of
    vertices, tasks ordered panel by panel; read at graph creation) give the
    oracle's counts, per vertex and in total, with and without split rows,
    with the symmetric half-arc root and on a graph kept in the caller's
    vertex order (isolated vertices not last)."""
    monkeypatch.setenv("SG2V_PANELS", panels)
    monkeypatch.setenv("SG2V_CHUNK", chunk)
    g = _hub_graph(5)
    col = si.colouring(g.n, 10, 3)
    for parent in (si.TREE10.parent, si.PATH7.parent, (-1, 0, 0, 2)):
        k = len(parent)
        ref, plan, r64, r32 = _run(sg, g, parent, 0, col if k == 10 else si.colouring(g.n, k, 3))
        _check_fp64(r64[0], r64[1], ref, exact=ref.max_bits <= 53)
        _check_fp32(r32[0], r32[1], ref)
    # totals only (the half-arc root) and several colourings per wave
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE10.parent, 0, 10)
    cols = si.colourings(g.n, 10, 3, seed=4)
    _, tot, _ = sg.count_batched(graph, [plan], _dev(cols), "fp64", per_vertex=False)
    tot = tot.cpu().numpy()[0]
    for b in range(3):
        r = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, cols[b], per_vertex=False)
        assert tot[b] == float(r.total) if r.max_bits <= 53 else abs(tot[b] - r.total) <= FP64_RTOL * r.total
    # the caller's vertex order, with isolated vertices scattered through it
    rng = np.random.default_rng(2)
    n2 = g.n + 300
    keep = np.sort(rng.choice(n2, size=g.n, replace=False))
    deg = np.zeros(n2, dtype=np.int64)
    deg[keep] = np.diff(g.row_ptr)
    rp = np.zeros(n2 + 1, dtype=np.int64)
    rp[1:] = np.cumsum(deg)
    ci = keep[g.col_idx].astype(np.int32)
    coli = si.colouring(n2, 7, 8)
    ref = oracle.count(rp, ci, si.TREE7.parent, 0, coli)
    graph = sg.Graph(rp, ci, keep_order=True)
    plan = sg.Plan(si.TREE7.parent, 0)
    for prec in ("fp64", "fp32"):
        pv, t, _ = sg.count(graph, plan, _dev(coli), prec)
        if prec == "fp64":
            _check_fp64(pv.cpu().numpy(), t, ref, exact=ref.max_bits <= 53)
        else:
            _check_fp32(pv.cpu().numpy(), t, ref)


def test_wave_beyond_packed_arc_limit(sg, monkeypatch):
    """The run-scatter kernel addresses a gathered row through a packed 28-bit
    vector offset; a wave of colourings wide enough to pass 2^28 vectors
    (2^20 vertices x 16 colourings x 21 vectors for tree10's (5,1,4)) runs
    those launches on the per-colour-accumulator kernel instead, with the
    same exact counts as one colouring per wave and as the oracle."""
    import torch

    g = si.erdos_renyi(1 << 20, 1 << 20, seed=3)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE10.parent, 0, 10, cut="min_work", avg_degree=2.0)
    B = 16
    cols = si.colourings(g.n, 10, B, seed=8)
    res = {}
    for wave in ("16", "1"):
        monkeypatch.setenv("SG2V_WAVE", wave)
        _, tot, _ = sg.count_batched(graph, [plan], _dev(cols), "fp64", per_vertex=False)
        res[wave] = tot.cpu().numpy()[0]
    assert np.array_equal(res["16"], res["1"])
    ref = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, cols[0], per_vertex=False)
    assert ref.max_bits <= 53 and res["16"][0] == float(ref.total)
