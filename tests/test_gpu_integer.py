"""Exact integer tables (SG2V_U64, SG2V_U128): unsigned 64- and 128-bit counts.

On an unweighted graph every value of the DP (Alg. 3 / 5) is a non-negative
integer, so with integer tables each per-vertex count and each total is the
exact integer while every table entry stays below 2^64 (2^128): past the
2^53 up to which FP64 tables are exact.  The outputs are doubles, so the bar
is bit-equality with the oracle's exact integers correctly rounded to double
(per vertex, and the total summed in 128 bits before its one rounding).  A
count that does not fit must be reported (SG2V_ERR_FP_OVERFLOW), never
returned wrapped.
"""
import json
import os

import numpy as np
import pytest

import oracle
import sg2v_inputs as si

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


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


def _exact(got_pv, got_total, ref):
    want = np.array([float(int(x)) for x in ref.per_vertex], dtype=np.float64)
    assert np.array_equal(np.asarray(got_pv), want)
    assert got_total == float(int(ref.total))


FORMS = {
    "default": {},
    "wide_rows": {"SG2V_WIDE_MIN_WZ": "1"},
    "split_rows": {"SG2V_CHUNK": "40"},
    "warp_per_row": {"SG2V_HIST_ROWS": "0", "SG2V_GROUP_ROWS": "0"},
    "deferred_ema": {"SG2V_DEFER_EMA": "1"},
}


def _hub_graph():
    """R-MAT base plus two hubs (split rows at any chunk size) and isolated
    vertices at the end (empty rows)."""
    base = si.rmat(11, 12000, seed=5)
    edges = {(int(u), int(v)) for u, v in base.edges}
    edges |= {(7, v) for v in range(8, 1900) if v % 3}
    edges |= {(min(1500, v), max(1500, v)) for v in range(0, 2048, 5) if v != 1500}
    return si.from_edges(2100, sorted(edges))


@pytest.mark.parametrize("prec", ["u64", "u128"])
@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("parent", [si.PATH5.parent, si.TREE7.parent, si.TREE8.parent, (-1, 0, 1, 2, 2, 0),
                                    si.STAR7.parent])
def test_integer_tables_match_oracle(sg, parent, form, prec, monkeypatch):
    """Every kernel form (warp rows, lane-group rows, CTA rows, split rows,
    the histogram forms, the deferred eMA) and colour counts k and k + 2."""
    for key, val in FORMS[form].items():
        monkeypatch.setenv(key, val)
    g = _hub_graph()
    graph = sg.Graph(g.row_ptr, g.col_idx)
    k = len(parent)
    for kc in (k, k + 2):
        plan = sg.Plan(parent, 0, kc)
        col = si.colouring(g.n, kc, 7, kc)
        ref = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, kc)
        pv, tot, _ = sg.count(graph, plan, _dev(col), prec)
        _exact(pv.cpu().numpy(), tot, ref)
        assert np.all(pv.cpu().numpy()[2048:] == 0)


def test_u64_exact_beyond_fp64(sg):
    """tree10, k = 10 on R-MAT scale 12 with 2^16 edges: per-vertex counts up
    to 2^61 and a 68-bit total, all exact; FP64 tables are not exact here."""
    g = si.rmat(12, 1 << 16, seed=0)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE10.parent, 0, 10)
    col = si.colouring(g.n, 10, 0, 0)
    ref = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, col, 10)
    assert 53 < ref.max_bits < 64
    assert max(int(x) for x in ref.per_vertex) > 2**53 and int(ref.total) >= 2**64
    # FP32 tables first, so that the memory pool hands the integer tables
    # bytes that are not zero (row padding is never written)
    sg.count_batched(graph, [plan], _dev(si.colourings(g.n, 10, 4, seed=3)), "fp32", per_vertex=True)
    pv, tot, est = sg.count(graph, plan, _dev(col), "u64")
    _exact(pv.cpu().numpy(), tot, ref)
    # totals only: the root gathers half of the arcs and doubles its row sums
    _, t2, _ = sg.count_batched(graph, [plan], _dev(col[None, :]), "u64", per_vertex=False)
    assert float(t2.cpu().numpy()[0, 0]) == float(int(ref.total))


def test_u64_overflow_is_reported(sg):
    """tree10, k = 10 on R-MAT scale 13 with 2^17 edges: per-vertex counts
    reach 2^66, so a call (and a session) keeping them reports the overflow."""
    g = si.rmat(13, 1 << 17, seed=0)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE10.parent, 0, 10)
    col = si.colouring(g.n, 10, 0, 0)
    with pytest.raises(sg.Sg2vError) as e:
        sg.count(graph, plan, _dev(col), "u64")
    assert e.value.status == sg.SG2V_ERR_FP_OVERFLOW
    import torch

    # a session keeping per-vertex counts (the root's rows are those counts)
    ses = sg.Session(graph, [plan], 1, "u64", per_vertex=True, graph_replay=True)
    tot = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    ses.run(_dev(col[None, :]), tot, None, None)
    with pytest.raises(sg.Sg2vError) as e:
        ses.sync()
    assert e.value.status == sg.SG2V_ERR_FP_OVERFLOW
    # totals only: the root sums each edge once (half of each row's arcs), so
    # its rows may fit 64 bits; then the exact 128-bit total comes back
    ref10 = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, col, 10, per_vertex=False)
    ses2 = sg.Session(graph, [plan], 1, "u64", graph_replay=True)
    ses2.run(_dev(col[None, :]), tot, None, None)
    try:
        ses2.sync()
        assert tot.item() == float(ref10.total)
    except sg.Sg2vError as e2:
        assert e2.status == sg.SG2V_ERR_FP_OVERFLOW
    # the same graph with a smaller template fits
    plan5 = sg.Plan(si.PATH5.parent, 0, 5)
    col5 = si.colouring(g.n, 5, 0, 1)
    ref = oracle.count(g.row_ptr, g.col_idx, si.PATH5.parent, 0, col5, 5)
    pv, t, _ = sg.count(graph, plan5, _dev(col5), "u64")
    _exact(pv.cpu().numpy(), t, ref)


@pytest.mark.parametrize("prec", ["u64", "u128"])
def test_integer_tables_batched_waves_and_session(sg, prec, monkeypatch):
    """Three templates x 5 colourings in waves of 2 (shared sub-templates),
    then the same request through a session with graph replay."""
    monkeypatch.setenv("SG2V_WAVE", "2")
    import torch

    g = si.rmat(12, 30000, seed=7)
    temps = [si.PATH7, si.STAR7, si.TREE7]
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plans = [sg.Plan(t.parent) for t in temps]
    B = 5
    cols = si.colourings(g.n, 7, B, seed=9)
    refs = [[oracle.count(g.row_ptr, g.col_idx, t.parent, 0, cols[b]) for b in range(B)] for t in temps]
    pv, tot, _ = sg.count_batched(graph, plans, _dev(cols), prec, per_vertex=True)
    pv, tot = pv.cpu().numpy(), tot.cpu().numpy()
    for i in range(len(temps)):
        for b in range(B):
            _exact(pv[i, b], tot[i, b], refs[i][b])
    ses = sg.Session(graph, plans, B, prec, per_vertex=True, graph_replay=True)
    stot = torch.empty((3, B), dtype=torch.float64, device="cuda")
    spv = torch.empty((3, B, g.n), dtype=torch.float64, device="cuda")
    for _ in range(2):
        ses.run(_dev(cols), stot, None, spv)
        ses.sync()
    stot, spv = stot.cpu().numpy(), spv.cpu().numpy()
    for i in range(len(temps)):
        for b in range(B):
            _exact(spv[i, b], stot[i, b], refs[i][b])


@pytest.mark.parametrize("prec", ["u64", "u128"])
def test_integer_tables_weighted_and_backward_unsupported(sg, prec):
    g = si.erdos_renyi(200, 600, seed=1)
    w = si.arc_weights(g, si.edge_weights(g, seed=1))
    plan = sg.Plan(si.PATH5.parent)
    col = si.colouring(g.n, 5, 1)
    with pytest.raises(sg.Sg2vError) as e:
        sg.count(sg.Graph(g.row_ptr, g.col_idx, w), plan, _dev(col), prec)
    assert e.value.status == sg.SG2V_ERR_UNSUPPORTED
    grad = np.zeros(g.nnz)
    with pytest.raises(sg.Sg2vError) as e:
        sg.sg2v_count_backward(sg.Graph(g.row_ptr, g.col_idx).handle, plan.handle, col, sg.PRECISIONS[prec], grad)
    assert e.value.status == sg.SG2V_ERR_UNSUPPORTED


def test_u128_exact_past_2_64(sg):
    """tree10, k = 10 on R-MAT scale 13 with 2^17 edges: entries reach 2^66
    (64-bit tables report the overflow); 128-bit tables are exact, per vertex
    and for the total, also after FP32 calls dirtied the memory pool."""
    g = si.rmat(13, 1 << 17, seed=0)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE10.parent, 0, 10)
    col = si.colouring(g.n, 10, 0, 0)
    ref = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, col, 10)
    assert 64 < ref.max_bits < 128
    sg.count_batched(graph, [plan], _dev(si.colourings(g.n, 10, 2, seed=3)), "fp32", per_vertex=True)
    pv, tot, _ = sg.count(graph, plan, _dev(col), "u128")
    _exact(pv.cpu().numpy(), tot, ref)
    _, t2, _ = sg.count_batched(graph, [plan], _dev(col[None, :]), "u128", per_vertex=False)
    assert float(t2.cpu().numpy()[0, 0]) == float(int(ref.total))


def _star_graph(leaves: int):
    return si.from_edges(leaves + 1, [(0, v) for v in range(1, leaves + 1)])


def test_u128_star_hub_and_overflow(sg):
    """A 10-vertex star rooted at its centre on a star graph: the hub's count
    is 9! times the product of its neighbours' colour-class sizes (Sec. 2.3's
    colourful maps; the closed form is checked by the oracle's own tests).
    With 4,096 leaves it is about 2^97 (exact); with 2^17 leaves about 2^142,
    which 128-bit tables report as an overflow."""
    star10 = (-1,) + (0,) * 9
    plan = sg.Plan(star10, 0, 10)
    g = _star_graph(4096)
    col = si.colouring(g.n, 10, 4, 0)
    ref = oracle.count(g.row_ptr, g.col_idx, star10, 0, col, 10)
    assert 64 < int(ref.total).bit_length() <= 128
    pv, tot, _ = sg.count(sg.Graph(g.row_ptr, g.col_idx), plan, _dev(col), "u128")
    _exact(pv.cpu().numpy(), tot, ref)
    g = _star_graph(1 << 17)
    col = si.colouring(g.n, 10, 4, 1)
    cnt = np.bincount(col[1:], minlength=10).astype(object)
    want = 362880
    for c in range(10):
        if c != col[0]:
            want *= int(cnt[c])
    assert want >= 2**128
    for prec in ("u64", "u128"):
        with pytest.raises(sg.Sg2vError) as e:
            sg.count(sg.Graph(g.row_ptr, g.col_idx), plan, _dev(col), prec)
        assert e.value.status == sg.SG2V_ERR_FP_OVERFLOW


def test_u128_full_size_rmat20_tree10(sg):
    """The 1M-vertex workload (R-MAT scale 20, 2^24 edges, tree10, k = 10),
    whose tables reach 2^94: 128-bit tables give the stored oracle values
    (tests/golden) exactly, for 4,000+ sampled vertices and for the total."""
    import hashlib

    import torch

    gold = json.load(open(os.path.join(HERE, "golden", "rmat20_16m_tree10_k10.json")))
    assert 64 < gold["max_table_bits"] < 128
    g = si.workload_graph(gold["graph"])
    h = hashlib.sha256()
    h.update(g.row_ptr.tobytes())
    h.update(g.col_idx.tobytes())
    assert h.hexdigest() == gold["graph_sha256"], "generator did not rebuild the stored graph"
    col = si.colouring(g.n, gold["num_colours"], gold["colouring_seed"], gold["colouring_index"])
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(gold["template"], gold["root"], gold["num_colours"])
    idx = np.array(gold["sample_vertices"])
    want = np.array([float(int(x)) for x in gold["sample_counts"]])
    pv, t, _ = sg.count(graph, plan, _dev(col), "u128")
    assert np.array_equal(pv.cpu().numpy()[idx], want)
    assert t == float(int(gold["total"]))
    del pv
    torch.cuda.empty_cache()
    _, t2, _ = sg.count_batched(graph, [plan], _dev(col[None, :]), "u128", per_vertex=False)
    assert float(t2.cpu().numpy()[0, 0]) == float(int(gold["total"]))
