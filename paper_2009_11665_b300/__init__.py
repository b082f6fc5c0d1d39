"""B300-native colour-coding tree counting (SubGraph2Vec, arXiv 2009.11665).

Thin ctypes binding of ``libsg2v.so`` (the C ABI declared in
``include/sg2v.h``).  Every function named ``sg2v_*`` here marshals its
arguments and calls the C entry point of the same name; all counting runs in
the library's CUDA kernels.  Arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA); streams default to torch's current stream.

The library must have been built (``python -m paper_2009_11665_b300.build``
or ``__graft_entry__.build()``); importing this package without it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsg2v.so")

SG2V_OK = 0
SG2V_ERR_INVALID_ARGUMENT = 1
SG2V_ERR_NOT_A_TREE = 2
SG2V_ERR_COLOUR_OUT_OF_RANGE = 3
SG2V_ERR_GRAPH_NOT_SIMPLE = 4
SG2V_ERR_OUT_OF_MEMORY = 5
SG2V_ERR_FP_OVERFLOW = 6
SG2V_ERR_CUDA = 7
SG2V_ERR_TIMEOUT = 8
SG2V_ERR_UNSUPPORTED = 9

SG2V_FP64 = 0
SG2V_FP32 = 1
SG2V_FP32_SCALED = 2
SG2V_U64 = 3
SG2V_U128 = 4
SG2V_GRAPH_SKIP_VALIDATION = 0x1
SG2V_GRAPH_KEEP_ORDER = 0x2
SG2V_CUT_LAST = 0
SG2V_CUT_MIN_WORK = 1
SG2V_BACKWARD_RECOMPUTE = 0x1
SG2V_BACKWARD_STORE = 0x2
SG2V_SESSION_PER_VERTEX = 0x1
SG2V_SESSION_NO_GRAPH = 0x2
SG2V_SESSION_AUTOTUNE = 0x4

PRECISIONS = {"fp64": SG2V_FP64, "fp32": SG2V_FP32, "fp32_scaled": SG2V_FP32_SCALED, "u64": SG2V_U64, "u128": SG2V_U128}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2009_11665_b300.build`")

_lib = ctypes.CDLL(LIB_PATH)
_p = ctypes.c_void_p
_i32, _i64, _u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32

# name -> (argtypes); every function returns an int status except where noted
_SIGNATURES = {
    "sg2v_graph_create": [_i64, _i64, _p, _p, _p, _u32, ctypes.POINTER(_p)],
    "sg2v_graph_destroy": [_p],
    "sg2v_graph_info": [_p, _p, _p, _p, _p],
    "sg2v_template_plan": [_i32, _p, _i32, _i32, _p, ctypes.POINTER(_p)],
    "sg2v_plan_destroy": [_p],
    "sg2v_plan_info": [_p, _p, _p, _p],
    "sg2v_plan_nodes": [_p, _p, _i64],
    "sg2v_plan_estimate_scale": [_p, _p],
    "sg2v_count": [_p, _p, _p, ctypes.c_int, _p, _p, _p, _p],
    "sg2v_count_batched": [_p, _p, _i32, _p, _i32, ctypes.c_int, _p, _p, _p, _p],
    "sg2v_sum_counts_noalloc": [_p, _i64, _i32, _p, _p],
    "sg2v_session_create": [_p, _p, _i32, _i32, ctypes.c_int, _u32, ctypes.POINTER(_p)],
    "sg2v_session_run": [_p, _p, _p, _p, _p, _p],
    "sg2v_session_sync": [_p, _p],
    "sg2v_session_info": [_p, _p, _p],
    "sg2v_session_tuning": [_p, ctypes.c_char_p, _i64, _p],
    "sg2v_session_destroy": [_p],
    "sg2v_count_backward": [_p, _p, _p, ctypes.c_int, _p, _p, _p, _u32, _p],
    "sg2v_graph_set_weights": [_p, _p, _p],
}
for _name, _args in _SIGNATURES.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.sg2v_status_string.argtypes = [ctypes.c_int]
_lib.sg2v_status_string.restype = ctypes.c_char_p
_lib.sg2v_last_error.argtypes = []
_lib.sg2v_last_error.restype = ctypes.c_char_p
_lib.sg2v_version.argtypes = []
_lib.sg2v_version.restype = ctypes.c_int32
_lib.sg2v_launch_count.argtypes = []
_lib.sg2v_launch_count.restype = ctypes.c_int64
_lib.sg2v_last_call_peak_bytes.restype = ctypes.c_int64
_lib.sg2v_last_call_peak_bytes.argtypes = []


class PlanOpts(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("cut", ctypes.c_int32), ("avg_degree", ctypes.c_float)]


class KernelRecord(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 64), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes_per_launch", ctypes.c_double)]


for _name, _args in {"sg2v_profile_enable": [_i32], "sg2v_profile_reset": [],
                     "sg2v_profile_read": [_p, _i32, ctypes.POINTER(_i32)]}.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int

EXPORTED = tuple(_SIGNATURES) + ("sg2v_status_string", "sg2v_last_error", "sg2v_version", "sg2v_profile_enable",
                                 "sg2v_profile_reset", "sg2v_profile_read", "sg2v_launch_count")


class Sg2vError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = _lib.sg2v_last_error().decode()
        super().__init__(f"{where}: {_lib.sg2v_status_string(status).decode()} ({detail})")


def _check(status: int, where: str) -> int:
    if status != SG2V_OK:
        raise Sg2vError(status, where)
    return status


def _ptr(x) -> Optional[int]:
    """Address of a numpy array / torch tensor (None for None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream) -> Optional[int]:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch

        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


# ------------------------------------------------------------ raw entry points

def sg2v_version() -> int:
    return int(_lib.sg2v_version())


def sg2v_status_string(status: int) -> str:
    return _lib.sg2v_status_string(status).decode()


def sg2v_last_error() -> str:
    return _lib.sg2v_last_error().decode()


def sg2v_graph_create(n: int, nnz: int, row_ptr, col_idx, weights=None, flags: int = 0) -> int:
    h = _p()
    _check(_lib.sg2v_graph_create(n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(weights), flags, ctypes.byref(h)),
           "sg2v_graph_create")
    return h.value


def sg2v_graph_destroy(handle) -> None:
    _check(_lib.sg2v_graph_destroy(handle), "sg2v_graph_destroy")


def sg2v_graph_info(handle):
    n, nnz, md, w = _i64(), _i64(), _i64(), _i32()
    _check(_lib.sg2v_graph_info(handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(md), ctypes.byref(w)),
           "sg2v_graph_info")
    return n.value, nnz.value, md.value, bool(w.value)


def sg2v_template_plan(parent: Sequence[int], root: int = 0, num_colours: Optional[int] = None,
                       cut: Optional[int] = None, avg_degree: float = 0.0) -> int:
    par = np.ascontiguousarray(parent, dtype=np.int32)
    k = int(par.shape[0])
    h = _p()
    opts = None
    if cut is not None:
        opts = PlanOpts(ctypes.sizeof(PlanOpts), int(cut), float(avg_degree))
    _check(_lib.sg2v_template_plan(k, _ptr(par), int(root), int(num_colours or k),
                                   ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)),
           "sg2v_template_plan")
    return h.value


def sg2v_plan_destroy(handle) -> None:
    _check(_lib.sg2v_plan_destroy(handle), "sg2v_plan_destroy")


def sg2v_plan_info(handle):
    a, nn, mc = _i64(), _i32(), _i64()
    _check(_lib.sg2v_plan_info(handle, ctypes.byref(a), ctypes.byref(nn), ctypes.byref(mc)), "sg2v_plan_info")
    return a.value, nn.value, mc.value


def sg2v_plan_nodes(handle) -> list:
    _, nn, _ = sg2v_plan_info(handle)
    out = np.zeros(max(6 * nn, 1), dtype=np.int32)
    _check(_lib.sg2v_plan_nodes(handle, _ptr(out), out.shape[0]), "sg2v_plan_nodes")
    return [tuple(int(x) for x in out[6 * i:6 * i + 6]) for i in range(nn)]


def sg2v_plan_estimate_scale(handle) -> float:
    s = ctypes.c_double()
    _check(_lib.sg2v_plan_estimate_scale(handle, ctypes.byref(s)), "sg2v_plan_estimate_scale")
    return s.value


def sg2v_count(graph, plan, colours, precision: int = SG2V_FP64, per_vertex=None, stream=None):
    """Returns (total, estimate); fills per_vertex ([n] float64) when given."""
    t, e = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sg2v_count(graph, plan, _ptr(colours), int(precision), _ptr(per_vertex), ctypes.byref(t),
                           ctypes.byref(e), _stream(stream)), "sg2v_count")
    return t.value, e.value


def sg2v_count_batched(graph, plans: Sequence[int], colours, B: int, precision: int = SG2V_FP32,
                       per_vertex=None, totals=None, estimates=None, stream=None) -> None:
    arr = (_p * len(plans))(*plans)
    _check(_lib.sg2v_count_batched(graph, arr, len(plans), _ptr(colours), int(B), int(precision),
                                   _ptr(per_vertex), _ptr(totals), _ptr(estimates), _stream(stream)),
           "sg2v_count_batched")


def sg2v_sum_counts_noalloc(values, n: int, nseg: int, totals, stream=None) -> None:
    """Sums device values [nseg][n] into device totals [nseg] without
    allocating (see include/sg2v.h); stream-ordered, no synchronisation.
    Torch tensors are checked first (float64, at least nseg * n values and
    nseg totals, on a CUDA device): the C entry point cannot see sizes, and a
    short or float32 buffer would be read past its end on the device."""
    tensors = [(name, t, need) for name, t, need in (("values", values, int(nseg) * int(n)),
                                                      ("totals", totals, int(nseg)))
               if hasattr(t, "dtype") and hasattr(t, "numel")]
    if tensors:
        import torch

        for name, t, need in tensors:
            if t.dtype != torch.float64:
                raise ValueError(f"sg2v_sum_counts_noalloc: {name} must be float64, got {t.dtype}")
            if t.numel() < need:
                raise ValueError(f"sg2v_sum_counts_noalloc: {name} holds {t.numel()} values, needs {need}")
        for name, t, _ in tensors:
            if not t.is_cuda:
                raise ValueError(f"sg2v_sum_counts_noalloc: {name} must be a CUDA tensor")
            if not t.is_contiguous():
                raise ValueError(f"sg2v_sum_counts_noalloc: {name} must be contiguous")
    _check(_lib.sg2v_sum_counts_noalloc(_ptr(values), int(n), int(nseg), _ptr(totals), _stream(stream)),
           "sg2v_sum_counts_noalloc")


def sg2v_count_backward(graph, plan, colours, precision: int, grad_weights, grad_per_vertex=None,
                        stream=None, flags: int = 0) -> float:
    """Fills grad_weights ([nnz] float64) with dF/dw_e per arc; returns the
    forward total.  flags: 0 (form chosen by memory), SG2V_BACKWARD_STORE or
    SG2V_BACKWARD_RECOMPUTE."""
    t = ctypes.c_double()
    _check(_lib.sg2v_count_backward(graph, plan, _ptr(colours), int(precision), _ptr(grad_per_vertex),
                                    _ptr(grad_weights), ctypes.byref(t), int(flags), _stream(stream)),
           "sg2v_count_backward")
    return t.value


def sg2v_last_call_peak_bytes() -> int:
    """Peak per-call device workspace of this thread's last count call."""
    return int(_lib.sg2v_last_call_peak_bytes())


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
# every callback pair ever installed stays alive: sessions keep the functions
# they were created with until they are destroyed, after any later change
_allocator_refs = []
_lib.sg2v_set_allocator.argtypes = [ALLOC_FN, FREE_FN, _p]
_lib.sg2v_set_allocator.restype = ctypes.c_int


def sg2v_set_allocator(alloc=None, free=None) -> None:
    """Routes the library's per-call workspaces (and new sessions' buffers)
    through Python callables alloc(bytes, stream) -> int device pointer (0 when
    out of memory) and free(ptr, stream); both None restores the library's
    pool.  See include/sg2v.h."""
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        _check(_lib.sg2v_set_allocator(ALLOC_FN(), FREE_FN(), None), "sg2v_set_allocator")
        return

    def _a(nbytes, stream, user):
        try:
            return int(alloc(int(nbytes), stream)) or None
        except Exception:  # an exception must not cross the C ABI
            return None

    def _f(ptr, stream, user):
        try:
            free(ptr, stream)
        except Exception:
            pass

    refs = (ALLOC_FN(_a), FREE_FN(_f))
    _allocator_refs.append(refs)
    _check(_lib.sg2v_set_allocator(refs[0], refs[1], None), "sg2v_set_allocator")


def use_torch_allocator(device: Optional[int] = None) -> None:
    """Serves the library's workspaces from PyTorch's caching allocator."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, dev, stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    sg2v_set_allocator(alloc, free)


def sg2v_graph_set_weights(graph, weights, stream=None) -> None:
    _check(_lib.sg2v_graph_set_weights(graph, _ptr(weights), _stream(stream)), "sg2v_graph_set_weights")


def sg2v_session_create(graph, plans: Sequence[int], B: int, precision: int = SG2V_FP32, flags: int = 0) -> int:
    arr = (_p * len(plans))(*plans)
    h = _p()
    _check(_lib.sg2v_session_create(graph, arr, len(plans), int(B), int(precision), int(flags), ctypes.byref(h)),
           "sg2v_session_create")
    return h.value


def sg2v_session_run(session, colours, totals=None, estimates=None, per_vertex=None, stream=None) -> None:
    _check(_lib.sg2v_session_run(session, _ptr(colours), _ptr(totals), _ptr(estimates), _ptr(per_vertex),
                                 _stream(stream)), "sg2v_session_run")


def sg2v_session_sync(session, stream=None) -> None:
    _check(_lib.sg2v_session_sync(session, _stream(stream)), "sg2v_session_sync")


def sg2v_session_info(session):
    w, gr = _i32(), _i32()
    _check(_lib.sg2v_session_info(session, ctypes.byref(w), ctypes.byref(gr)), "sg2v_session_info")
    return w.value, bool(gr.value)


def sg2v_session_tuning(session) -> dict:
    """The session's wave and per-node kernel forms (see include/sg2v.h)."""
    import json

    n = ctypes.c_int64()
    _check(_lib.sg2v_session_tuning(session, None, 0, ctypes.byref(n)), "sg2v_session_tuning")
    buf = ctypes.create_string_buffer(int(n.value) + 1)
    _check(_lib.sg2v_session_tuning(session, buf, len(buf), None), "sg2v_session_tuning")
    return json.loads(buf.value.decode())


def sg2v_session_destroy(session) -> None:
    _check(_lib.sg2v_session_destroy(session), "sg2v_session_destroy")


def sg2v_profile_enable(enable: bool = True) -> None:
    _check(_lib.sg2v_profile_enable(1 if enable else 0), "sg2v_profile_enable")


def sg2v_profile_reset() -> None:
    _check(_lib.sg2v_profile_reset(), "sg2v_profile_reset")


def sg2v_profile_read() -> list:
    """[{name, launches, total_ms, bytes_per_launch}] of the kernels timed so far."""
    cnt = _i32()
    _check(_lib.sg2v_profile_read(None, 0, ctypes.byref(cnt)), "sg2v_profile_read")
    recs = (KernelRecord * max(cnt.value, 1))()
    _check(_lib.sg2v_profile_read(ctypes.cast(recs, _p), cnt.value, ctypes.byref(cnt)), "sg2v_profile_read")
    return [dict(name=r.name.decode(), launches=r.launches, total_ms=r.total_ms, bytes_per_launch=r.bytes_per_launch)
            for r in recs[:cnt.value]]


def sg2v_launch_count() -> int:
    return int(_lib.sg2v_launch_count())


# ------------------------------------------------------------ convenience

class Graph:
    """Owns a library graph handle (CSR copied onto the current device)."""

    def __init__(self, row_ptr, col_idx, weights=None, validate: bool = True, keep_order: bool = False):
        rp = row_ptr if hasattr(row_ptr, "data_ptr") else np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = col_idx if hasattr(col_idx, "data_ptr") else np.ascontiguousarray(col_idx, dtype=np.int32)
        w = None
        if weights is not None:
            w = weights if hasattr(weights, "data_ptr") else np.ascontiguousarray(weights, dtype=np.float32)
        self.n = int(rp.shape[0]) - 1
        self.nnz = int(ci.shape[0])
        flags = (0 if validate else SG2V_GRAPH_SKIP_VALIDATION) | (SG2V_GRAPH_KEEP_ORDER if keep_order else 0)
        self.handle = sg2v_graph_create(self.n, self.nnz, rp, ci, w, flags)

    def info(self):
        return sg2v_graph_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sg2v_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owns a template plan handle."""

    def __init__(self, parent: Sequence[int], root: int = 0, num_colours: Optional[int] = None,
                 cut: Optional[str] = None, avg_degree: float = 0.0):
        self.parent = tuple(int(x) for x in parent)
        self.k = len(self.parent)
        self.kc = int(num_colours or self.k)
        self.root = root
        c = None if cut is None else {"last": SG2V_CUT_LAST, "min_work": SG2V_CUT_MIN_WORK}[cut]
        self.handle = sg2v_template_plan(self.parent, root, self.kc, c, avg_degree)
        self.alpha, self.num_nodes, self.max_cols = sg2v_plan_info(self.handle)
        self.scale = sg2v_plan_estimate_scale(self.handle)

    def nodes(self):
        return sg2v_plan_nodes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sg2v_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count(graph: Graph, plan: Plan, colours, precision: str = "fp64", per_vertex: bool = True, stream=None):
    """One colouring: returns (per_vertex float64 tensor on colours' device or
    None, total, estimate)."""
    import torch

    dev = colours.device if hasattr(colours, "device") else torch.device("cuda")
    pv = torch.empty(graph.n, dtype=torch.float64, device=dev) if per_vertex else None
    total, est = sg2v_count(graph.handle, plan.handle, colours, PRECISIONS[precision], pv, stream)
    return pv, total, est


class Session:
    """Repeated batched counting with preallocated buffers and CUDA-graph
    replay (see sg2v_session_create)."""

    def __init__(self, graph: Graph, plans: Sequence[Plan], B: int, precision: str = "fp32",
                 per_vertex: bool = False, graph_replay: bool = True, autotune: bool = False):
        flags = (SG2V_SESSION_PER_VERTEX if per_vertex else 0) | (0 if graph_replay else SG2V_SESSION_NO_GRAPH) | \
                (SG2V_SESSION_AUTOTUNE if autotune else 0)
        self.graph, self.plans, self.B = graph, list(plans), int(B)
        self.handle = sg2v_session_create(graph.handle, [p.handle for p in plans], B, PRECISIONS[precision], flags)

    def run(self, colours, totals=None, estimates=None, per_vertex=None, stream=None):
        sg2v_session_run(self.handle, colours, totals, estimates, per_vertex, stream)

    def sync(self, stream=None):
        sg2v_session_sync(self.handle, stream)

    def info(self):
        return sg2v_session_info(self.handle)

    def tuning(self):
        return sg2v_session_tuning(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sg2v_session_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count_batched(graph: Graph, plans: Sequence[Plan], colours, precision: str = "fp32", per_vertex: bool = False,
                  stream=None):
    """B colourings ([B, n] int8) x len(plans) templates: returns
    (per_vertex [P, B, n] or None, totals [P, B], estimates [P, B]) as float64
    tensors on colours' device."""
    import torch

    B = int(colours.shape[0])
    dev = colours.device if hasattr(colours, "device") else torch.device("cuda")
    P = len(plans)
    pv = torch.empty((P, B, graph.n), dtype=torch.float64, device=dev) if per_vertex else None
    tot = torch.empty((P, B), dtype=torch.float64, device=dev)
    est = torch.empty((P, B), dtype=torch.float64, device=dev)
    sg2v_count_batched(graph.handle, [p.handle for p in plans], colours, B, PRECISIONS[precision], pv, tot, est,
                       stream)
    return pv, tot, est


def weighted_count(weights, graph: Graph, plan: Plan, colours, precision: str = "fp32"):
    """Differentiable per-vertex colourful counts of a weighted graph: each
    colourful map contributes the product of its edge weights.  `weights` is
    a float32 CUDA tensor [nnz] (symmetric: both arcs of an edge equal); the
    graph must have been created with weights.  Returns per_vertex [n]
    float64; gradients flow back to `weights` through sg2v_count_backward."""
    import torch

    class _WeightedCount(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w):
            sg2v_graph_set_weights(graph.handle, w.detach().contiguous())
            pv, _, _ = count(graph, plan, colours, precision)
            ctx.save_for_backward(w)
            return pv

        @staticmethod
        def backward(ctx, grad_pv):
            (w,) = ctx.saved_tensors
            sg2v_graph_set_weights(graph.handle, w.detach().contiguous())
            g = torch.empty(w.shape[0], dtype=torch.float64, device=w.device)
            sg2v_count_backward(graph.handle, plan.handle, colours, PRECISIONS[precision], g,
                                grad_pv.detach().to(torch.float64).contiguous())
            return g.to(w.dtype)

    return _WeightedCount.apply(weights)
