"""FP32 tables with per-row power-of-two exponents (SG2V_FP32_SCALED).

Counts of 15-vertex trees on large graphs pass FP32's 2^128; with a
power-of-two exponent per table row the DP keeps FP32 relative precision at
any magnitude.  The bar is the FP32 one (1e-4 relative to the exact oracle,
zeros exact), on:

* small graphs against the oracle, through every kernel form (warp rows,
  CTA-per-row rows, split rows, the histogram node, waves, sessions);
* weighted graphs whose weights are j * 2^-24, where every count of a
  10-vertex tree (nine edges) lies below FP32's smallest normal;
* the large form's scale-12 and scale-16 siblings against stored oracle
  values (written by tests/golden/make_golden.py); at scale 16 the counts
  reach 2^133, so plain FP32 overflows and is rerun with row exponents.
"""
import json
import os

import numpy as np
import pytest

import oracle
import sg2v_inputs as si

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-4


@pytest.fixture(scope="module")
def sg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as s

    return s


def _close(got, want, tol=TOL):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    nz = want != 0
    assert np.all(got[~nz] == 0)
    if nz.any():
        assert (np.abs(got[nz] - want[nz]) / want[nz]).max() <= tol


def _tiny_weights(g, seed):
    """Edge weights j * 2^-24, j in 1..16: exact for the oracle (multiples of
    2^-24) and small enough that nine-edge products leave FP32's range."""
    j = np.floor(si.edge_weights(g, seed=seed, lo=1.0, hi=17.0)).astype(np.float32)
    return si.arc_weights(g, (j * np.float32(2.0**-24)).astype(np.float32))


@pytest.mark.parametrize("parent", [si.PATH5.parent, si.TREE7.parent, si.TREE8.parent, (-1, 0, 1, 2, 2, 0)])
@pytest.mark.parametrize("wide", [False, True])
def test_scaled_matches_oracle(sg, parent, wide, monkeypatch):
    import torch

    if wide:
        monkeypatch.setenv("SG2V_WIDE_MIN_WZ", "1")
    g = si.rmat(11, 12000, seed=5)
    k = len(parent)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    for kc in (k, k + 2):
        plan = sg.Plan(parent, 0, kc)
        col = si.colouring(g.n, kc, 7)
        ref = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, kc)
        pv, tot, est = sg.count(graph, plan, torch.from_numpy(col).cuda(), "fp32_scaled")
        _close(pv.cpu().numpy(), ref.per_vertex_float())
        assert abs(tot - ref.total) <= TOL * ref.total


@pytest.mark.parametrize("chunk", ["1024", "40"])
def test_scaled_split_rows_and_isolated(sg, chunk, monkeypatch):
    """Hub rows split into chunks (their reference exponent is the maximum
    over every chunk) and isolated vertices (empty rows)."""
    monkeypatch.setenv("SG2V_CHUNK", chunk)
    import torch

    base = si.erdos_renyi(3000, 9000, seed=2)
    edges = {(int(u), int(v)) for u, v in base.edges}
    edges |= {(0, v) for v in range(1, 2400) if v % 3}  # a hub
    g = si.from_edges(3200, sorted(edges))  # vertices 3000.. are isolated
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE7.parent)
    col = si.colouring(g.n, 7, 3)
    ref = oracle.count(g.row_ptr, g.col_idx, si.TREE7.parent, 0, col)
    pv, tot, _ = sg.count(graph, plan, torch.from_numpy(col).cuda(), "fp32_scaled")
    pv = pv.cpu().numpy()
    _close(pv, ref.per_vertex_float())
    assert np.all(pv[3000:] == 0)


def test_scaled_weighted_below_fp32_range(sg):
    """Weights j * 2^-24: every per-vertex count of the 10-vertex tree lies
    below 2^-126 (FP32's smallest normal); row exponents keep full precision."""
    import torch

    g = si.chung_lu(4000, 30000, 2.3, seed=3)
    w = _tiny_weights(g, 3)
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(si.TREE10.parent)
    col = si.colouring(g.n, 10, 1)
    ref = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, col, weights=w)
    want = ref.per_vertex_float()
    assert want[want > 0].max() < 2.0**-126
    pv, tot, _ = sg.count(graph, plan, torch.from_numpy(col).cuda(), "fp32_scaled")
    _close(pv.cpu().numpy(), want)
    assert abs(tot - float(ref.total_value())) <= TOL * float(ref.total_value())


def test_scaled_batched_waves_and_session(sg, monkeypatch):
    """Three templates x 5 colourings in waves of 2, then the same request
    through a session (graph replay)."""
    monkeypatch.setenv("SG2V_WAVE", "2")
    import torch

    g = si.rmat(12, 30000, seed=7)
    temps = [si.PATH7, si.STAR7, si.TREE7]
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plans = [sg.Plan(t.parent) for t in temps]
    B = 5
    cols = si.colourings(g.n, 7, B, seed=9)
    pv, tot, est = sg.count_batched(graph, plans, torch.from_numpy(cols).cuda(), "fp32_scaled", per_vertex=True)
    pv, tot = pv.cpu().numpy(), tot.cpu().numpy()
    refs = [[oracle.count(g.row_ptr, g.col_idx, t.parent, 0, cols[b]) for b in range(B)] for t in temps]
    for i in range(len(temps)):
        for b in range(B):
            _close(pv[i, b], refs[i][b].per_vertex_float())
            assert abs(tot[i, b] - refs[i][b].total) <= TOL * refs[i][b].total
    ses = sg.Session(graph, plans, B, "fp32_scaled", per_vertex=True, graph_replay=True)
    stot = torch.empty((3, B), dtype=torch.float64, device="cuda")
    spv = torch.empty((3, B, g.n), dtype=torch.float64, device="cuda")
    for _ in range(2):
        ses.run(torch.from_numpy(cols).cuda(), stot, None, spv)
        ses.sync()
    stot, spv = stot.cpu().numpy(), spv.cpu().numpy()
    for i in range(len(temps)):
        for b in range(B):
            _close(spv[i, b], refs[i][b].per_vertex_float())
            assert abs(stot[i, b] - refs[i][b].total) <= TOL * refs[i][b].total


def test_scaled_backward_is_unsupported(sg):
    g = si.erdos_renyi(200, 600, seed=1)
    w = si.arc_weights(g, si.edge_weights(g, seed=1))
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(si.PATH5.parent)
    col = si.colouring(g.n, 5, 1)
    grad = np.zeros(g.nnz)
    with pytest.raises(sg.Sg2vError) as e:
        sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.SG2V_FP32_SCALED, grad)
    assert e.value.status == sg.SG2V_ERR_UNSUPPORTED


def _large(sg, name, precisions):
    import torch

    gold = json.load(open(os.path.join(HERE, "golden", name)))
    g = si.rmat(gold["scale"], gold["m"], seed=0)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(gold["template"], 0, 15)
    B = len(gold["colourings"])
    cols = torch.from_numpy(si.colourings(g.n, 15, B, seed=0)).cuda()
    idx = np.array(gold["sample_vertices"])
    for prec, tol in precisions:
        pv, tot, _ = sg.count_batched(graph, [plan], cols, prec, per_vertex=True)
        pv, tot = pv.cpu().numpy(), tot.cpu().numpy()
        for b, rec in enumerate(gold["colourings"]):
            total = int(rec["total"])
            assert abs(tot[0, b] - total) <= tol * total
            _close(pv[0, b, idx], [float(int(x)) for x in rec["sample_counts"]], tol)
        del pv
    return gold


def test_large_form_scale12_scaled(sg):
    _large(sg, "rmat12_large_sibling_tree15_k15.json", [("fp32_scaled", TOL)])


def test_large_form_scale16_beyond_fp32_range(sg):
    """Counts reach 2^133: plain FP32 overflows and is rerun with row
    exponents inside the call; FP64 and explicit scaled FP32 agree too."""
    gold = _large(sg, "rmat16_large_sibling_tree15_k15.json",
                  [("fp32", TOL), ("fp32_scaled", TOL), ("fp64", 1e-12)])
    assert max(int(r["max_table_bits"]) for r in gold["colourings"]) > 128
