"""sg2v_sum_counts_noalloc: totals without any device allocation.

The entry point serves callers that cannot allocate device memory where they
need a total (serving loops whose memory is reserved up front by their own
allocator, code that must not stall other streams).  It sums per-vertex counts the caller already holds, with its
scratch in a fixed device array inside the library.  These tests compare its
totals with those of sg2v_count / sg2v_count_batched on the same counts, on
two calls in a row (the shared scratch must not carry anything over).  This
file is collected last so that a run stopping at its first failure has run
every other test.
"""
import numpy as np
import pytest

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


def test_noalloc_total_matches_count(sg):
    import torch

    g = si.workload_graph("er2000")
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.PATH5.parent)
    col = torch.from_numpy(si.colouring(g.n, 5, 0)).cuda()
    pv, total, _ = sg.count(graph, plan, col, "fp64")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        sg.sg2v_sum_counts_noalloc(pv, g.n, 1, out)
        torch.cuda.synchronize()
        assert out.item() == total  # exact integer sum rounded once, as sg2v_count


def test_noalloc_batched_segments_match(sg):
    import torch

    g = si.rmat(12, 30000, seed=7)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plans = [sg.Plan(t.parent) for t in (si.PATH7, si.STAR7, si.TREE7)]
    cols = torch.from_numpy(si.colourings(g.n, 7, 4, seed=3)).cuda()
    for prec in ("fp64", "fp32"):
        pv, tot, _ = sg.count_batched(graph, plans, cols, prec, per_vertex=True)
        out = torch.empty(12, dtype=torch.float64, device="cuda")
        for _ in range(2):
            out.fill_(-1.0)
            sg.sg2v_sum_counts_noalloc(pv, g.n, 12, out)
            torch.cuda.synchronize()
            assert torch.equal(out, tot.reshape(-1))


def test_noalloc_weighted_values(sg):
    """Non-integral counts (weighted graph): compensated sum, same tolerance
    as the FP64 parity tests."""
    import torch

    g = si.chung_lu(3000, 20000, 2.3, seed=1)
    w = si.arc_weights(g, si.edge_weights(g, seed=1))
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(si.TREE8.parent)
    col = torch.from_numpy(si.colouring(g.n, 8, 4)).cuda()
    pv, total, _ = sg.count(graph, plan, col, "fp64")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        sg.sg2v_sum_counts_noalloc(pv, g.n, 1, out)
        torch.cuda.synchronize()
        assert abs(out.item() - total) <= 1e-12 * abs(total)


def test_noalloc_rejects_oversized_and_host_requests(sg):
    import torch

    vals = torch.ones((1025, 4), dtype=torch.float64, device="cuda")
    out = torch.empty(1025, dtype=torch.float64, device="cuda")
    with pytest.raises(sg.Sg2vError) as e:
        sg.sg2v_sum_counts_noalloc(vals, 4, 1025, out)
    assert e.value.status == sg.SG2V_ERR_INVALID_ARGUMENT
    host = np.ones(4)
    with pytest.raises(sg.Sg2vError) as e:
        sg.sg2v_sum_counts_noalloc(host, 4, 1, out)
    assert e.value.status == sg.SG2V_ERR_INVALID_ARGUMENT
    # the largest accepted request still works
    vals = torch.arange(1024 * 3, dtype=torch.float64, device="cuda").reshape(1024, 3)
    sg.sg2v_sum_counts_noalloc(vals, 3, 1024, out)
    torch.cuda.synchronize()
    assert torch.equal(out[:1024], vals.sum(dim=1))


def test_noalloc_sum_past_2_128_takes_the_compensated_sum(sg):
    """Values whose exact 128-bit sum passes 2^128 must not come back wrapped.
    With n = 192 each of the 64 blocks sums three consecutive values; block 1
    holds 2^128 - 2^75, 2^75 - 2^64 and 2^64 - 2^11 (its partial has the high
    word 2^64 - 1 and the low word 2^64 - 2^11), block 0 holds 4096, so the
    final combination carries out of the low word into a high word of
    2^64 - 1: the sum 2^128 + 2^11 must be reported as the compensated FP64
    sum (2^128 after rounding), not as 2^11."""
    import torch

    vals = np.zeros(192)
    vals[0] = 4096.0
    vals[3] = 2.0 ** 128 - 2.0 ** 75
    vals[4] = 2.0 ** 75 - 2.0 ** 64
    vals[5] = 2.0 ** 64 - 2.0 ** 11
    dv = torch.from_numpy(vals).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        sg.sg2v_sum_counts_noalloc(dv, 192, 1, out)
        torch.cuda.synchronize()
        assert out.item() == 2.0 ** 128
    # below 2^128 the same values stay exact: drop the 4096
    dv[0] = 0.0
    sg.sg2v_sum_counts_noalloc(dv, 192, 1, out)
    torch.cuda.synchronize()
    assert out.item() == 2.0 ** 128 - 2.0 ** 11


def test_noalloc_replays_inside_a_cuda_graph(sg):
    """The entry point's purpose: after one warm-up call it can be recorded
    in stream capture (it allocates nothing and does not synchronise), and
    each replay of the captured graph sums the values the buffer holds at
    that moment, exactly (integral values: the 128-bit integer path)."""
    import torch

    n, nseg = 100_003, 3
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    vals = torch.randint(0, 1 << 20, (nseg, n), generator=gen, device="cuda").to(torch.float64)
    totals = torch.full((nseg,), -1.0, dtype=torch.float64, device="cuda")
    sg.sg2v_sum_counts_noalloc(vals, n, nseg, totals)  # the warm-up call the header asks for
    torch.cuda.synchronize()
    assert torch.equal(totals, vals.sum(dim=1))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sg.sg2v_sum_counts_noalloc(vals, n, nseg, totals)
    for seed in (11, 12):
        gen.manual_seed(seed)
        vals.copy_(torch.randint(0, 1 << 20, (nseg, n), generator=gen, device="cuda").to(torch.float64))
        totals.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(totals, vals.sum(dim=1))
