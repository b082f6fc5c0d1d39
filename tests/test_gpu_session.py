"""Sessions: preallocated buffers, CUDA-graph replay, device-side totals and
estimates, wave autotuning (the batched form of the counting DP).

Results must equal the exact oracle under the same bars as the direct
calls (FP64 bit-exact below 2^53, FP32 1e-4 relative, estimates within
2 ulp of total / (P alpha))."""
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


def _ulp_close(a: float, exact: Fraction, ulps: int = 2) -> bool:
    b = float(exact)
    return abs(a - b) <= ulps * np.spacing(abs(b))


def _check(prec, got_pv, got_total, ref):
    want = np.array([float(x) for x in ref.per_vertex_values()])
    nz = want != 0
    assert np.all(got_pv[~nz] == 0)
    tv = float(ref.total_value())
    if prec == "fp64" and ref.max_bits <= 53:
        assert np.array_equal(got_pv, want)
        assert got_total == tv
    else:
        tol = 1e-12 if prec == "fp64" else 1e-4
        if nz.any():
            assert (np.abs(got_pv[nz] - want[nz]) / want[nz]).max() <= tol
        assert abs(got_total - tv) <= tol * abs(tv)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("replay", [True, False])
def test_session_runs_match_oracle(sg, prec, replay):
    """Two runs with different colourings (the second replays the captured
    graph) against one oracle count per (template, colouring)."""
    import torch

    g = si.rmat(12, 30000, seed=7)
    B = 3
    temps = [si.PATH7, si.STAR7, si.TREE7]
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plans = [sg.Plan(t.parent) for t in temps]
    ses = sg.Session(graph, plans, B, prec, per_vertex=True, graph_replay=replay)
    for seed in (3, 4):
        cols = si.colourings(g.n, 7, B, seed=seed)
        tot = torch.empty((3, B), dtype=torch.float64, device="cuda")
        est = torch.empty((3, B), dtype=torch.float64, device="cuda")
        pv = torch.empty((3, B, g.n), dtype=torch.float64, device="cuda")
        ses.run(torch.from_numpy(cols).cuda(), tot, est, pv)
        ses.sync()
        tot, est, pv = tot.cpu().numpy(), est.cpu().numpy(), pv.cpu().numpy()
        for i, t in enumerate(temps):
            for b in range(B):
                ref = oracle.count(g.row_ptr, g.col_idx, t.parent, 0, cols[b])
                _check(prec, pv[i, b], tot[i, b], ref)
                if prec == "fp64":
                    assert _ulp_close(est[i, b], oracle.estimate(ref.total, 7, plans[i].alpha))
    wave, captured = ses.info()
    assert captured == replay
    assert 1 <= wave <= B


def test_session_autotune_and_host_outputs(sg):
    g = si.erdos_renyi(3000, 15000, seed=4)
    B = 5
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE8.parent)
    ses = sg.Session(graph, [plan], B, "fp32", autotune=True)
    cols = si.colourings(g.n, 8, B, seed=2)
    tot = np.zeros((1, B))
    est = np.zeros((1, B))
    ses.run(cols, tot, est)  # host colourings, host outputs
    ses.sync()
    wave, captured = ses.info()
    assert 1 <= wave <= B and captured
    for b in range(B):
        ref = oracle.count(g.row_ptr, g.col_idx, si.TREE8.parent, 0, cols[b], per_vertex=False)
        assert abs(tot[0, b] - ref.total) <= 1e-4 * ref.total
        assert est[0, b] == pytest.approx(float(oracle.estimate(ref.total, 8, plan.alpha)), rel=1e-4)


def test_session_reports_bad_colours(sg):
    g = si.erdos_renyi(400, 1600, seed=1)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    ses = sg.Session(graph, [sg.Plan((-1, 0, 1, 2))], 2, "fp64")
    cols = si.colourings(g.n, 4, 2, seed=1)
    ses.run(cols)
    ses.sync()
    cols[1, 7] = 9
    ses.run(cols)
    with pytest.raises(sg.Sg2vError) as e:
        ses.sync()
    assert e.value.status == sg.SG2V_ERR_COLOUR_OUT_OF_RANGE


def test_session_single_vertex_and_weighted(sg):
    """Single-vertex templates (every vertex counts once) and a weighted
    graph through the session path."""
    import torch

    g = si.chung_lu(3000, 20000, 2.3, seed=1)
    w = si.arc_weights(g, si.edge_weights(g, seed=1))
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plans = [sg.Plan((-1,), 0, 8), sg.Plan(si.TREE8.parent)]
    ses = sg.Session(graph, plans, 2, "fp64", per_vertex=True)
    cols = si.colourings(g.n, 8, 2, seed=5)
    tot = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    pv = torch.empty((2, 2, g.n), dtype=torch.float64, device="cuda")
    ses.run(torch.from_numpy(cols).cuda(), tot, None, pv)
    ses.sync()
    assert torch.all(pv[0] == 1.0) and torch.all(tot[0] == g.n)
    for b in range(2):
        ref = oracle.count(g.row_ptr, g.col_idx, si.TREE8.parent, 0, cols[b], weights=w)
        _check("fp64", pv[1, b].cpu().numpy(), tot[1, b].item(), ref)


def test_estimator_loop_on_a_session(sg):
    """Alg. 1's loop driven by a session (the GPU counter): the same
    colourings through the exact oracle give the same average."""
    from paper_2009_11665_b300 import estimator as E

    g = si.erdos_renyi(500, 2500, seed=8)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.PATH5.parent)
    ses = sg.Session(graph, [plan], 8, "fp64")
    colouring = lambda i: si.colouring(g.n, 5, 21, i)
    res = E.ColourCodingEstimator(E.session_counter(ses), colouring, 5, eps=0.02, delta=0.05, wave=8,
                                  min_colourings=16, max_colourings=96).run()
    alpha = oracle.automorphisms(si.PATH5.parent)
    vals = []
    for i in range(res.colourings):
        tot = oracle.count(g.row_ptr, g.col_idx, si.PATH5.parent, 0, colouring(i), per_vertex=False).total
        vals.append(float(oracle.estimate(tot, 5, alpha)))
    assert res.estimate[0] == pytest.approx(np.mean(vals), rel=1e-12)


def test_form_autotuning_is_exact_and_cached(sg, tmp_path, monkeypatch):
    """Autotuning picks each node's kernel form by timing; every form gives
    the same counts (oracle-exact totals in FP64), and a second session with
    the same cache file takes the stored forms."""
    import json

    import torch

    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SG2V_TUNE_CACHE", str(cache))
    g = si.rmat(12, 40000, seed=11)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    parents = [si.PATH7.parent, si.STAR7.parent, si.TREE7.parent]
    plans = [sg.Plan(p) for p in parents]
    B = 4
    cols = si.colourings(g.n, 7, B, seed=6)
    refs = [[oracle.count(g.row_ptr, g.col_idx, p, 0, cols[b]) for b in range(B)] for p in parents]
    forms = []
    for rep in range(2):
        ses = sg.Session(graph, plans, B, "fp64", autotune=True)
        tot = torch.empty((len(plans), B), dtype=torch.float64, device="cuda")
        ses.run(torch.from_numpy(cols).cuda(), tot)
        ses.sync()
        info = ses.tuning()
        assert info["tuned"] and len(info["nodes"]) > 0
        forms.append([n["form"] for n in info["nodes"]])
        t = tot.cpu().numpy()
        for i in range(len(plans)):
            for b in range(B):
                r = refs[i][b]
                if r.max_bits <= 53:
                    assert t[i, b] == float(r.total)
                else:
                    assert abs(t[i, b] - r.total) <= 1e-12 * r.total
        ses.close()
        stored = json.loads(cache.read_text())
        assert len(stored) >= len(info["nodes"])
    assert forms[0] == forms[1]


def test_split_schedule_autotuning(sg, tmp_path, monkeypatch):
    """The autotuner also picks the split schedule (the chunk size at which
    long rows are cut into tasks) by timing the session's step on each
    candidate work list; counts do not depend on it (FP64 oracle-exact),
    the choice is cached, and SG2V_CHUNK fixes it instead."""
    import json

    import torch

    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SG2V_TUNE_CACHE", str(cache))
    monkeypatch.delenv("SG2V_CHUNK", raising=False)
    g = si.rmat(12, 40000, seed=11)
    deg = np.diff(g.row_ptr)
    assert deg.max() > 256  # rows that every candidate below 512 splits
    graph = sg.Graph(g.row_ptr, g.col_idx)
    parents = [si.PATH7.parent, si.TREE7.parent]
    plans = [sg.Plan(p) for p in parents]
    B = 3
    cols = si.colourings(g.n, 7, B, seed=9)
    refs = [[oracle.count(g.row_ptr, g.col_idx, p, 0, cols[b], per_vertex=False) for b in range(B)]
            for p in parents]
    chunks = []
    for rep in range(2):
        ses = sg.Session(graph, plans, B, "fp64", autotune=True)
        tot = torch.empty((len(plans), B), dtype=torch.float64, device="cuda")
        ses.run(torch.from_numpy(cols).cuda(), tot)
        ses.sync()
        # a second run replays the captured graph on the chosen work list
        ses.run(torch.from_numpy(cols).cuda(), tot)
        ses.sync()
        info = ses.tuning()
        assert info["chunk"] in (256, 512, 1024, 2048, 4096, 8192) and info["panels"] in (1, 2, 4)
        chunks.append(info["chunk"])
        t = tot.cpu().numpy()
        for i in range(len(plans)):
            for b in range(B):
                _exact_or_close(t[i, b], refs[i][b])
        ses.close()
    stored = json.loads(cache.read_text())
    split = [v for k, v in stored.items() if k.startswith("split|")]
    assert split and int(split[0].split(",")[0]) == chunks[0] == chunks[1]
    # a fixed chunk size (read when the graph is created) is kept
    monkeypatch.setenv("SG2V_CHUNK", "300")
    graph2 = sg.Graph(g.row_ptr, g.col_idx)
    ses = sg.Session(graph2, plans, B, "fp64", autotune=True)
    tot = torch.empty((len(plans), B), dtype=torch.float64, device="cuda")
    ses.run(torch.from_numpy(cols).cuda(), tot)
    ses.sync()
    assert ses.tuning()["chunk"] == 300
    t = tot.cpu().numpy()
    for i in range(len(plans)):
        for b in range(B):
            _exact_or_close(t[i, b], refs[i][b])
    ses.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotuned_session_on_weighted_graph(sg, prec, tmp_path, monkeypatch):
    """An autotuned session on a weighted graph with rows long enough to be
    split: whichever split schedule, wave width and node forms the tuner
    picks (the weighted (2, 1, 1) node has one form), the replayed step's
    per-vertex counts and totals equal the exact dyadic oracle."""
    import torch

    monkeypatch.setenv("SG2V_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.delenv("SG2V_CHUNK", raising=False)
    g = si.rmat(12, 40000, seed=11)
    assert np.diff(g.row_ptr).max() > 256
    w = si.arc_weights(g, si.edge_weights(g, seed=8))
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plans = [sg.Plan(si.TREE8.parent), sg.Plan(si.PATH5.parent, 0, 8)]
    B = 2
    cols = si.colourings(g.n, 8, B, seed=12)
    ses = sg.Session(graph, plans, B, prec, per_vertex=True, autotune=True)
    tot = torch.empty((len(plans), B), dtype=torch.float64, device="cuda")
    pv = torch.empty((len(plans), B, g.n), dtype=torch.float64, device="cuda")
    for _ in range(2):  # the tuning run, then a graph replay
        ses.run(torch.from_numpy(cols).cuda(), tot, None, pv)
        ses.sync()
        for i, parent in enumerate((si.TREE8.parent, si.PATH5.parent)):
            for b in range(B):
                ref = oracle.count(g.row_ptr, g.col_idx, parent, 0, cols[b], 8, w)
                _check(prec, pv[i, b].cpu().numpy(), tot[i, b].item(), ref)
    ses.close()


def _exact_or_close(got: float, ref) -> None:
    if ref.max_bits <= 53:
        assert got == float(ref.total)
    else:
        assert abs(got - ref.total) <= 1e-12 * ref.total
