"""Graph ingest (sg2v_graph_create) rejects every malformed input with its
status before any device work, and the allocator hook's arguments are
checked.  The method needs a simple undirected graph (Sec. 2.2.1) stored as a
CSR adjacency matrix (Sec. 5.1): each case below breaks one of those
requirements.  These run on the host only: validation happens before the
library touches a device."""
import numpy as np
import pytest

import sg2v_inputs as si


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as s

    return s


def _status(sg, rp, ci, w=None, flags=0, n=None):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
    n = len(rp) - 1 if n is None else n
    try:
        h = sg.sg2v_graph_create(n, len(ci), rp, ci, w, flags)
    except sg.Sg2vError as e:
        return e.status
    sg.sg2v_graph_destroy(h)
    return sg.SG2V_OK


def _csr(n, edges):
    g = si.from_edges(n, edges)
    return g.row_ptr.copy(), g.col_idx.copy()


def _no_device():
    try:
        import torch

        return not torch.cuda.is_available()
    except Exception:
        return True


# triangle 0-1-2 plus the edge 2-3
BASE = [(0, 1), (1, 2), (0, 2), (2, 3)]


def test_valid_graph_reaches_the_device_step(sg):
    rp, ci = _csr(4, BASE)
    st = _status(sg, rp, ci)
    if _no_device():
        assert st == sg.SG2V_ERR_CUDA  # validation passed; no device to copy to
    else:
        assert st == sg.SG2V_OK


def test_self_loop(sg):
    rp, ci = _csr(4, BASE)
    # row 3 = [2] -> [2, 3]
    ci2 = np.concatenate([ci, [3]])
    rp2 = rp.copy()
    rp2[4] += 1
    assert _status(sg, rp2, ci2) == sg.SG2V_ERR_GRAPH_NOT_SIMPLE


def test_duplicate_arc(sg):
    rp, ci = _csr(4, BASE)
    # row 3 = [2] -> [2, 2] and row 2 gets a second 3
    ci2 = np.concatenate([ci[:rp[3]], [3], ci[rp[3]:], [2]])
    rp2 = rp.copy()
    rp2[3:] += 1
    rp2[4] += 1
    assert _status(sg, rp2, ci2) == sg.SG2V_ERR_GRAPH_NOT_SIMPLE


def test_asymmetric_arc(sg):
    rp, ci = _csr(4, [(0, 1), (1, 2), (0, 2)])
    # add 3 -> 0 without 0 -> 3
    ci2 = np.concatenate([ci, [0]])
    rp2 = rp.copy()
    rp2[4] += 1
    assert _status(sg, rp2, ci2) == sg.SG2V_ERR_GRAPH_NOT_SIMPLE


def test_unsorted_row(sg):
    rp, ci = _csr(4, BASE)
    lo, hi = rp[2], rp[3]  # row 2 = [0, 1, 3]
    ci2 = ci.copy()
    ci2[lo:hi] = ci[lo:hi][::-1]
    assert _status(sg, rp, ci2) == sg.SG2V_ERR_GRAPH_NOT_SIMPLE


def test_column_out_of_range(sg):
    rp, ci = _csr(4, BASE)
    for bad in (4, 1000, -1):
        ci2 = ci.copy()
        ci2[-1] = bad
        assert _status(sg, rp, ci2) == sg.SG2V_ERR_INVALID_ARGUMENT


def test_row_pointer_errors(sg):
    rp, ci = _csr(4, BASE)
    rp2 = rp.copy()
    rp2[2], rp2[3] = rp[3], rp[2]  # a negative step
    assert _status(sg, rp2, ci) == sg.SG2V_ERR_INVALID_ARGUMENT
    rp3 = rp.copy()
    rp3[0] = 1
    assert _status(sg, rp3, ci) == sg.SG2V_ERR_INVALID_ARGUMENT
    rp4 = rp.copy()
    rp4[-1] -= 1  # does not end at nnz
    assert _status(sg, rp4, ci) == sg.SG2V_ERR_INVALID_ARGUMENT


def test_weight_errors(sg):
    rp, ci = _csr(4, BASE)
    g = si.from_edges(4, BASE)
    w = si.arc_weights(g, np.array([0.5, 1.0, 1.25, 0.75]))
    good = _status(sg, rp, ci, w)
    assert good in (sg.SG2V_OK, sg.SG2V_ERR_CUDA)
    for bad in ("asymmetric", "negative", "nan", "inf"):
        w2 = w.copy()
        if bad == "asymmetric":
            w2[0] += 0.5
        elif bad == "negative":
            ids = si.arc_edge_ids(g)
            w2[ids == ids[0]] = -1.0  # both arcs of one edge
        elif bad == "nan":
            w2[:] = np.nan
        else:
            w2[:] = np.inf
        assert _status(sg, rp, ci, w2) == sg.SG2V_ERR_GRAPH_NOT_SIMPLE, bad


def test_sizes_and_flags(sg):
    rp, ci = _csr(4, BASE)
    assert _status(sg, [0], np.zeros(0, np.int32), n=0) == sg.SG2V_ERR_INVALID_ARGUMENT
    assert _status(sg, rp, ci, flags=0x80) == sg.SG2V_ERR_INVALID_ARGUMENT


def test_skip_validation_trusts_the_csr(sg):
    rp, ci = _csr(4, BASE)
    lo, hi = rp[2], rp[3]
    ci2 = ci.copy()
    ci2[lo:hi] = ci[lo:hi][::-1]  # unsorted: accepted when validation is skipped
    st = _status(sg, rp, ci2, flags=sg.SG2V_GRAPH_SKIP_VALIDATION)
    assert st == (sg.SG2V_ERR_CUDA if _no_device() else sg.SG2V_OK)


def test_allocator_hook_arguments(sg):
    with pytest.raises(ValueError):
        sg.sg2v_set_allocator(lambda n, s: 0, None)
    # the C entry point refuses one function without the other
    st = sg._lib.sg2v_set_allocator(sg.ALLOC_FN(lambda n, s, u: None), sg.FREE_FN(), None)
    assert st == sg.SG2V_ERR_INVALID_ARGUMENT
    sg.sg2v_set_allocator(lambda n, s: 0, lambda p, s: None)
    sg.sg2v_set_allocator(None, None)
