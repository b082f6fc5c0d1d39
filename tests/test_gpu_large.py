"""The large form: a 15-vertex tree, k = 15 colours, 8 colourings per call.

Compressed rows reach C(14, 4) = 1001 columns, beyond one warp's register
tile, so those nodes run on the CTA-per-row kernel.  Parity with stored
oracle values (tests/golden, written by make_golden.py from the oracle only)
on the scaled sibling of the full workload (same R-MAT parameters and
edge/vertex ratio); the wide kernel is also driven through the small
parity cases by lowering the width at which it takes over."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_large_form_sibling_scale12(sg, prec):
    import torch

    gold = json.load(open(os.path.join(HERE, "golden", "rmat12_large_sibling_tree15_k15.json")))
    g = si.rmat(gold["scale"], gold["m"], seed=0)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(gold["template"], 0, 15)
    B = len(gold["colourings"])
    cols = si.colourings(g.n, 15, B, seed=0)
    pv, tot, est = sg.count_batched(graph, [plan], torch.from_numpy(cols).cuda(), prec, per_vertex=True)
    pv, tot = pv.cpu().numpy(), tot.cpu().numpy()
    idx = np.array(gold["sample_vertices"])
    tol = 1e-12 if prec == "fp64" else 1e-4
    for b, rec in enumerate(gold["colourings"]):
        total = int(rec["total"])
        assert abs(tot[0, b] - total) <= tol * total
        want = np.array([float(int(x)) for x in rec["sample_counts"]])
        got = pv[0, b, idx]
        nz = want != 0
        assert np.all(got[~nz] == 0)
        assert (np.abs(got[nz] - want[nz]) / want[nz]).max() <= tol


@pytest.mark.parametrize("parent", [si.TREE7.parent, si.TREE8.parent, si.PATH7.parent, (-1, 0, 1, 2, 2, 0)])
@pytest.mark.parametrize("chunk", ["1024", "48"])
def test_wide_kernel_on_small_cases(sg, parent, chunk, monkeypatch):
    """Every gathering node forced onto the CTA-per-row kernel (and split rows
    with a small chunk) still equals the oracle."""
    monkeypatch.setenv("SG2V_WIDE_MIN_WZ", "1")
    monkeypatch.setenv("SG2V_CHUNK", chunk)
    import torch

    g = si.rmat(11, 12000, seed=3)
    k = len(parent)
    for kc in (k, k + 2):
        col = si.colouring(g.n, kc, 4)
        graph = sg.Graph(g.row_ptr, g.col_idx)
        plan = sg.Plan(parent, 0, kc)
        ref = oracle.count(g.row_ptr, g.col_idx, parent, 0, col, kc)
        want = np.array([float(x) for x in ref.per_vertex])
        for prec, tol in (("fp64", 0.0), ("fp32", 1e-4)):
            pv, t, e = sg.count(graph, plan, torch.from_numpy(col).cuda(), prec)
            got = pv.cpu().numpy()
            if prec == "fp64" and ref.max_bits <= 53:
                assert np.array_equal(got, want)
            else:
                nz = want != 0
                assert np.all(got[~nz] == 0)
                assert (np.abs(got[nz] - want[nz]) / want[nz]).max() <= max(tol, 1e-12)


@pytest.mark.parametrize("parent", [si.TREE8.parent, (-1, 0, 1, 2, 2, 0), si.TREE7.parent])
@pytest.mark.parametrize("wide", ["", "1"])
def test_deferred_ema_on_small_cases(sg, parent, wide, monkeypatch):
    """Every non-root node with a >= 2 forced onto the separate eMA launch
    (blocks of four rows), on the warp and the CTA-per-row gather, in FP64,
    FP32 and scaled FP32, against the oracle."""
    monkeypatch.setenv("SG2V_DEFER_EMA", "1")
    if wide:
        monkeypatch.setenv("SG2V_WIDE_MIN_WZ", "1")
    import torch

    g = si.rmat(11, 12000, seed=6)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    k = len(parent)
    for kc in (k, k + 2):
        plan = sg.Plan(parent, 0, kc)
        cols = si.colourings(g.n, kc, 3, seed=8)
        refs = [oracle.count(g.row_ptr, g.col_idx, parent, 0, cols[b], kc) for b in range(3)]
        for prec in ("fp64", "fp32", "fp32_scaled"):
            pv, tot, _ = sg.count_batched(graph, [plan], torch.from_numpy(cols).cuda(), prec, per_vertex=True)
            pv = pv.cpu().numpy()
            for b, ref in enumerate(refs):
                want = np.array([float(x) for x in ref.per_vertex])
                if prec == "fp64" and ref.max_bits <= 53:
                    assert np.array_equal(pv[0, b], want)
                else:
                    nz = want != 0
                    assert np.all(pv[0, b][~nz] == 0)
                    tol = 1e-12 if prec == "fp64" else 1e-4
                    assert (np.abs(pv[0, b][nz] - want[nz]) / want[nz]).max() <= tol


PATH15 = tuple([-1] + list(range(14)))


@pytest.mark.parametrize("prec", ["fp32", "fp64", "u64", "u128"])
def test_widest_rows_column_tiles(sg, prec, monkeypatch):
    """A 15-vertex path, k = 15: its (9, 1, 8) node gathers compressed rows of
    C(14, 7) = 3,432 columns, the widest any 15-vertex tree has.  FP32 keeps
    Z in shared memory; FP64 and the integer tables walk the arcs once per
    column tile of the CTA (2 and 4 tiles) with Z in global memory.  Split
    rows too (chunks of 40 arcs)."""
    import torch

    g = si.erdos_renyi(150, 450, seed=1)
    edges = {(int(u), int(v)) for u, v in g.edges} | {(0, v) for v in range(1, 120)}
    g = si.from_edges(150, sorted(edges))
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(PATH15, 0, 15)
    assert max(int(n[2]) for n in plan.nodes()) == 14
    for chunk in ("1024", "40"):
        monkeypatch.setenv("SG2V_CHUNK", chunk)
        graph = sg.Graph(g.row_ptr, g.col_idx)
        for b in range(2):
            col = si.colouring(g.n, 15, 2, b)
            ref = oracle.count(g.row_ptr, g.col_idx, PATH15, 0, col, 15)
            pv, tot, _ = sg.count(graph, plan, torch.from_numpy(col).cuda(), prec)
            pv = pv.cpu().numpy()
            want = np.array([float(int(x)) for x in ref.per_vertex])
            if prec == "fp32":
                nz = want != 0
                assert np.all(pv[~nz] == 0)
                if nz.any():
                    assert (np.abs(pv[nz] - want[nz]) / want[nz]).max() <= 1e-4
                assert abs(tot - float(int(ref.total))) <= 1e-4 * float(int(ref.total))
            else:
                assert ref.max_bits <= 53
                assert np.array_equal(pv, want)
                assert tot == float(int(ref.total))


PATH16 = tuple([-1] + list(range(15)))


@pytest.mark.parametrize("prec", ["fp32", "fp64", "u128"])
def test_sixteen_colours_widest_rows(sg, prec):
    """A 16-vertex path, k = 16: its (9, 1, 8) node gathers rows of
    C(15, 7) = 6,435 columns, so Z holds 16 x 6,436 elements (beyond 16-bit
    expansion offsets and shared memory): two column tiles even in FP32,
    32-bit offsets, Z in global memory."""
    import torch

    g = si.erdos_renyi(120, 360, seed=1)
    edges = {(int(u), int(v)) for u, v in g.edges} | {(0, v) for v in range(1, 100)}
    g = si.from_edges(120, sorted(edges))
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(PATH16, 0, 16)
    col = si.colouring(g.n, 16, 2, 0)
    ref = oracle.count(g.row_ptr, g.col_idx, PATH16, 0, col, 16)
    pv, tot, _ = sg.count(graph, plan, torch.from_numpy(col).cuda(), prec)
    pv = pv.cpu().numpy()
    want = np.array([float(int(x)) for x in ref.per_vertex])
    if prec == "fp32":
        nz = want != 0
        assert np.all(pv[~nz] == 0)
        assert (np.abs(pv[nz] - want[nz]) / want[nz]).max() <= 1e-4
        assert abs(tot - float(int(ref.total))) <= 1e-4 * float(int(ref.total))
    else:
        assert ref.max_bits <= 53
        assert np.array_equal(pv, want)
        assert tot == float(int(ref.total))
