"""Parity at the full sizes of the benchmark's workloads.

Expected values are stored in tests/golden (written by make_golden.py from the
exact CPU oracle only).  Each test rebuilds its input from the generator's
seeds, checks the graph fingerprint, and compares:

* the benchmark's timed step exactly as it runs (R-MAT scale 20 with 2^24
  edges, tree10, the work-minimising plan, 4 colourings in one call, FP32,
  totals only, so the root gathers half the arcs) against the exact totals;
  the same call in 128-bit integers must reproduce the totals bit for bit and
  the estimates to within 2 ulp of the exactly rounded value (Alg. 1
  finalCount);
* the batched form (R-MAT scale 18, average degree 16, path7 / star7 / tree7,
  k = 7, the benchmark's 64-colouring session) on its first two colourings,
  totals and 4,000+ sampled per-vertex counts;
* the differentiable form (Chung-Lu, 200k vertices, FP32 weights, tree8):
  the exact weighted forward and the exact per-edge gradient
  (F - F(w_e = 0)) / w_e of 64 sampled edges, from both backward forms
  (tables kept, and tables rebuilt during the reverse walk);
* the large form (R-MAT scale 20 with 5e7 edges, tree15, k = 15) on two
  colourings: FP32 with per-row exponents against the FP64 tables, which are
  themselves oracle-checked on the scale-12 and scale-16 siblings (the exact
  oracle does not fit this host at full size).

Bars: FP64 1e-12 relative (entries pass 2^53), FP32 1e-4 relative, zeros
exact; integer tables exact.
"""
import hashlib
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import sg2v_inputs as si

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FP64_RTOL = 1e-12
FP32_RTOL = 1e-4


@pytest.fixture(scope="module")
def sg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as s

    return s


def _gold(name):
    return json.load(open(os.path.join(HERE, "golden", name)))


def _graph(gold):
    g = si.workload_graph(gold["graph"])
    h = hashlib.sha256()
    h.update(g.row_ptr.tobytes())
    h.update(g.col_idx.tobytes())
    assert h.hexdigest() == gold["graph_sha256"], "generator did not rebuild the stored graph"
    return g


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frac(s: str) -> Fraction:
    num, den = s.split("/")
    return Fraction(int(num), int(den))


def _ulps(a: float, b: float) -> float:
    return abs(a - b) / np.spacing(max(abs(a), abs(b)))


def test_bench_step_matches_oracle(sg):
    import torch

    gold = _gold("rmat20_16m_tree10_k10_bench_step.json")
    g = _graph(gold)
    B = len(gold["colourings"])
    cols = _dev(si.colourings(g.n, 10, B, seed=gold["colouring_seed"]))
    graph = sg.Graph(g.row_ptr, g.col_idx)
    # the benchmark's plan: work-minimising cuts for average degree 32
    plan = sg.Plan(gold["template"], gold["root"], 10, cut="min_work", avg_degree=32.0)
    totals = [int(c["total"]) for c in gold["colourings"]]
    exact_est = [oracle.estimate(t, 10, plan.alpha) for t in totals]
    for prec, tol in (("fp32", FP32_RTOL), ("fp64", FP64_RTOL)):
        _, tot, est = sg.count_batched(graph, [plan], cols, prec, per_vertex=False)
        tot, est = tot.cpu().numpy()[0], est.cpu().numpy()[0]
        for b in range(B):
            assert abs(tot[b] - totals[b]) <= tol * totals[b], (prec, b)
            assert abs(est[b] - float(exact_est[b])) <= tol * float(exact_est[b]), (prec, b)
    # the benchmark's autotuned session: the first run tunes (split schedule,
    # wave width, node forms), the second replays the captured CUDA graph
    ses = sg.Session(graph, [plan], B, "fp32", autotune=True)
    stot = torch.empty((1, B), dtype=torch.float64, device="cuda")
    sest = torch.empty((1, B), dtype=torch.float64, device="cuda")
    for rep in range(2):
        ses.run(cols, stot, sest)
        ses.sync()
        tot, est = stot.cpu().numpy()[0], sest.cpu().numpy()[0]
        for b in range(B):
            assert abs(tot[b] - totals[b]) <= FP32_RTOL * totals[b], ("session", rep, b)
            assert abs(est[b] - float(exact_est[b])) <= FP32_RTOL * float(exact_est[b]), ("session", rep, b)
    ses.close()
    # exact integer tables: the totals bit for bit, the estimates within 2 ulp
    _, tot, est = sg.count_batched(graph, [plan], cols, "u128", per_vertex=False)
    tot, est = tot.cpu().numpy()[0], est.cpu().numpy()[0]
    for b in range(B):
        assert tot[b] == float(totals[b])
        assert _ulps(float(est[b]), float(exact_est[b])) <= 2.0, b
    del graph
    torch.cuda.empty_cache()


def test_batched_form_matches_oracle(sg):
    import torch

    gold = _gold("rmat18_d16_k7_batched.json")
    g = _graph(gold)
    nb = len(gold["templates"][0]["colourings"])
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plans = [sg.Plan(t["template"], t["root"], 7) for t in gold["templates"]]
    idx = np.array(gold["sample_vertices"])
    # the benchmark's session: 64 colourings, CUDA-graph replay, autotuned
    # waves; its first colourings are the stored ones
    cols64 = si.colourings(g.n, 7, 64, seed=gold["colouring_seed"])
    ses = sg.Session(graph, plans, 64, "fp32", autotune=True)
    tot = torch.empty((len(plans), 64), dtype=torch.float64, device="cuda")
    ses.run(_dev(cols64), tot)
    ses.sync()
    tot = tot.cpu().numpy()
    ses.close()
    for i, t in enumerate(gold["templates"]):
        for b in range(nb):
            want = int(t["colourings"][b]["total"])
            assert abs(tot[i, b] - want) <= FP32_RTOL * want, (t["name"], b)
    # per-vertex counts of the stored colourings, FP32 and FP64
    for prec, tol in (("fp32", FP32_RTOL), ("fp64", FP64_RTOL)):
        pv, tt, _ = sg.count_batched(graph, plans, _dev(cols64[:nb]), prec, per_vertex=True)
        pv, tt = pv.cpu().numpy(), tt.cpu().numpy()
        for i, t in enumerate(gold["templates"]):
            for b in range(nb):
                c = t["colourings"][b]
                want = np.array([float(int(x)) for x in c["sample_counts"]])
                got = pv[i, b][idx]
                nz = want != 0
                assert np.all(got[~nz] == 0), (prec, t["name"], b)
                assert (np.abs(got[nz] - want[nz]) / want[nz]).max() <= tol, (prec, t["name"], b)
                if prec == "fp64" and c["max_table_bits"] <= 53:
                    assert tt[i, b] == float(int(c["total"]))
                else:
                    assert abs(tt[i, b] - int(c["total"])) <= tol * int(c["total"])


def test_differentiable_form_matches_oracle(sg):
    import torch

    gold = _gold("chunglu200k_tree8_k8_weighted.json")
    g = _graph(gold)
    w = si.arc_weights(g, si.edge_weights(g, seed=gold["weights_seed"]))
    col = si.colouring(g.n, 8, gold["colouring_seed"])
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(gold["template"], gold["root"], 8)
    F = _frac(gold["total"])
    idx = np.array(gold["sample_vertices"])
    want = np.array([float(_frac(x)) for x in gold["sample_values"]])
    ids = si.arc_edge_ids(g)
    edges = np.array(gold["edges"])
    grads = np.array([float(_frac(x)) for x in gold["gradients"]])
    for prec, tol in (("fp64", FP64_RTOL), ("fp32", FP32_RTOL)):
        pv, tot, _ = sg.count(graph, plan, _dev(col), prec)
        got = pv.cpu().numpy()[idx]
        nz = want != 0
        assert np.all(got[~nz] == 0), prec
        assert (np.abs(got[nz] - want[nz]) / want[nz]).max() <= tol, prec
        assert abs(tot - float(F)) <= tol * float(F), prec
        # both backward forms: every table kept, or rebuilt during the reverse walk
        for flag in (sg.SG2V_BACKWARD_STORE, sg.SG2V_BACKWARD_RECOMPUTE):
            gw = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
            t2 = sg.sg2v_count_backward(graph.handle, plan.handle, _dev(col), sg.PRECISIONS[prec], gw, flags=flag)
            assert abs(t2 - float(F)) <= tol * float(F), prec
            gw = gw.cpu().numpy()
            for e, gref in zip(edges, grads):
                arcs = np.nonzero(ids == e)[0]
                assert len(arcs) == 2
                for a in arcs:
                    assert abs(gw[a] - gref) <= tol * abs(gref) + 1e-300, (prec, flag, int(e))


def test_large_form_fp32_matches_fp64(sg):
    import torch

    g = si.workload_graph("rmat20_50m")
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE15.parent, 0, 15)
    cols = _dev(si.colourings(g.n, 15, 2, seed=0))
    pv64, t64, _ = sg.count_batched(graph, [plan], cols, "fp64", per_vertex=True)
    pv64, t64 = pv64.cpu().numpy()[0], t64.cpu().numpy()[0]
    torch.cuda.empty_cache()
    # plain FP32 overflows at these counts and is rerun with per-row exponents
    pv32, t32, _ = sg.count_batched(graph, [plan], cols, "fp32", per_vertex=True)
    pv32, t32 = pv32.cpu().numpy()[0], t32.cpu().numpy()[0]
    for b in range(2):
        assert t64[b] > 2.0 ** 128
        assert abs(t32[b] - t64[b]) <= FP32_RTOL * t64[b]
        nz = pv64[b] != 0
        assert np.all(pv32[b][~nz] == 0)
        assert (np.abs(pv32[b][nz] - pv64[b][nz]) / pv64[b][nz]).max() <= FP32_RTOL
    del graph
    torch.cuda.empty_cache()
