"""The allocator hook (sg2v_set_allocator): per-call workspaces and session
buffers come from the caller's allocator, a failing allocator gives
SG2V_ERR_OUT_OF_MEMORY with everything already taken given back, and results
do not depend on where the memory came from."""
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

    yield s
    s.sg2v_set_allocator(None, None)


class Budget:
    """Device memory from torch's caching allocator up to a byte budget."""

    def __init__(self, limit):
        import torch

        self.limit, self.used, self.live, self.calls = limit, 0, {}, 0
        self.torch = torch

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.used + nbytes > self.limit:
            return 0
        p = self.torch.cuda.caching_allocator_alloc(nbytes, self.torch.cuda.current_device(), stream)
        self.live[p] = nbytes
        self.used += nbytes
        return p

    def free(self, ptr, stream):
        self.used -= self.live.pop(ptr)
        self.torch.cuda.caching_allocator_delete(ptr)


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_hook_serves_the_call_and_gets_everything_back(sg):
    g = si.rmat(11, 16000, seed=3)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE10.parent)
    col = si.colouring(g.n, 10, 1)
    ref = oracle.count(g.row_ptr, g.col_idx, si.TREE10.parent, 0, col)
    pool_pv, pool_tot, _ = sg.count(graph, plan, _dev(col), "fp64")
    b = Budget(1 << 40)
    sg.sg2v_set_allocator(b.alloc, b.free)
    try:
        pv, tot, _ = sg.count(graph, plan, _dev(col), "fp64")
    finally:
        sg.sg2v_set_allocator(None, None)
    assert b.calls > 0 and not b.live and b.used == 0
    assert tot == pool_tot
    assert np.array_equal(pv.cpu().numpy(), pool_pv.cpu().numpy())
    if ref.max_bits <= 53:
        assert tot == float(ref.total)


@pytest.mark.parametrize("limit", [1 << 12, 1 << 20, 3 << 20])
def test_out_of_memory_is_reported_and_nothing_leaks(sg, limit):
    g = si.rmat(12, 40000, seed=5)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plan = sg.Plan(si.TREE10.parent)
    col = _dev(si.colouring(g.n, 10, 2))
    b = Budget(limit)
    sg.sg2v_set_allocator(b.alloc, b.free)
    try:
        with pytest.raises(sg.Sg2vError) as e:
            sg.count(graph, plan, col, "fp32")
        assert e.value.status == sg.SG2V_ERR_OUT_OF_MEMORY
    finally:
        sg.sg2v_set_allocator(None, None)
    assert not b.live and b.used == 0
    # the library is still usable afterwards
    _, tot, _ = sg.count(graph, plan, col, "fp32")
    assert tot > 0


def test_session_buffers_come_from_the_hook(sg):
    import torch

    g = si.rmat(10, 8000, seed=2)
    graph = sg.Graph(g.row_ptr, g.col_idx)
    plans = [sg.Plan(t.parent) for t in (si.TREE7, si.PATH7)]
    cols = _dev(si.colourings(g.n, 7, 4, seed=8))
    want = sg.count_batched(graph, plans, cols, "fp64")[1].cpu().numpy()
    b = Budget(1 << 40)
    sg.sg2v_set_allocator(b.alloc, b.free)
    try:
        ses = sg.Session(graph, plans, 4, "fp64")
    finally:
        sg.sg2v_set_allocator(None, None)
    held = b.used
    assert held > 0
    tot = torch.empty((2, 4), dtype=torch.float64, device="cuda")
    for _ in range(2):
        ses.run(cols, tot)
        ses.sync()
        assert np.array_equal(tot.cpu().numpy(), want)
    assert b.used == held  # runs allocate nothing
    ses.close()
    assert not b.live and b.used == 0


def test_torch_allocator_backward(sg):
    import torch

    g = si.chung_lu(500, 2500, 2.3, seed=4)
    w = si.arc_weights(g, si.edge_weights(g, seed=1))
    graph = sg.Graph(g.row_ptr, g.col_idx, w)
    plan = sg.Plan(si.TREE8.parent)
    col = _dev(si.colouring(g.n, 8, 0))
    g0 = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
    t0 = sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.SG2V_FP64, g0)
    sg.use_torch_allocator()
    try:
        g1 = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        t1 = sg.sg2v_count_backward(graph.handle, plan.handle, col, sg.SG2V_FP64, g1)
    finally:
        sg.sg2v_set_allocator(None, None)
    assert t1 == t0
    assert torch.equal(g0, g1)
