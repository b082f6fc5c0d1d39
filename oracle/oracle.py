"""Python face of the exact CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  The product (the CUDA library and its
binding) never imports, loads or calls anything under ``oracle/``.

Functions (paper: SubGraph2Vec, arXiv 2009.11665):

* ``count``      colourful-embedding counts by the partition DP, in exact
                 integers (Alg. 3 and Eq. 1 by default, Alg. 2 with
                 ``mode="standard"``);
* ``brute``      the same counts (or, with ``injective_only``, counts of
                 all injective embeddings) by enumerating every map;
* ``automorphisms``  alpha of Alg. 1: injective maps of the template onto itself;
* ``colourful_probability``, ``estimate``  P and finalCount of Alg. 1 as
                 exact rationals;
* ``py_brute``   a pure-Python enumerator for tiny inputs, written separately
                 from the C code so that it pins the C arithmetic too.

Weighted inputs are float32 edge weights; every float32 is a dyadic rational,
so the oracle scales them by 2^24 to integers (exact for weights in
[2^-24, 2^39)), counts in integers and divides the result by
2^(24 (k-1)) exactly (a tree embedding uses k-1 edges).
"""
from __future__ import annotations

import ctypes
import dataclasses
import itertools
import os
from fractions import Fraction
from math import factorial
from typing import Optional, Sequence

import numpy as np

from . import build as _build

DECOUPLED, STANDARD = 0, 1
CUT_LAST, CUT_FIRST = 0, 1
WEIGHT_SHIFT = 24

_libs = {}


def _lib(limbs: int):
    if limbs not in _libs:
        path = _build.lib_path(limbs)
        if not os.path.exists(path):
            _build.build()
        lib = ctypes.CDLL(path)
        p = ctypes.c_void_p
        lib.oracle_dp.argtypes = [ctypes.c_int64, p, p, p, ctypes.c_int, p, ctypes.c_int, ctypes.c_int, p,
                                  ctypes.c_int, ctypes.c_int, p, p, p, ctypes.c_int]
        lib.oracle_dp.restype = ctypes.c_int
        lib.oracle_brute.argtypes = [ctypes.c_int64, p, p, p, ctypes.c_int, p, ctypes.c_int, ctypes.c_int, p,
                                     ctypes.c_int, p, p, ctypes.c_int]
        lib.oracle_brute.restype = ctypes.c_int
        lib.oracle_limbs.restype = ctypes.c_int
        assert lib.oracle_limbs() == limbs
        _libs[limbs] = lib
    return _libs[limbs]


@dataclasses.dataclass
class Result:
    total: int                      # exact integer (unweighted) ...
    per_vertex: Optional[list]      # list of exact ints, or None
    max_bits: int = -1              # bits of the largest table entry (DP only)
    weight_scale_log2: int = 0      # weighted: true value = integer / 2^weight_scale_log2
    limbs: int = 2

    def total_value(self):
        """Exact value: int (unweighted) or Fraction (weighted)."""
        if self.weight_scale_log2:
            return Fraction(self.total, 1 << self.weight_scale_log2)
        return self.total

    def per_vertex_values(self):
        if self.per_vertex is None:
            return None
        if self.weight_scale_log2:
            d = 1 << self.weight_scale_log2
            return [Fraction(x, d) for x in self.per_vertex]
        return self.per_vertex

    def per_vertex_float(self) -> np.ndarray:
        """Per-vertex values, each rounded once to the nearest double."""
        vals = self.per_vertex_values()
        return np.array([float(x) for x in vals], dtype=np.float64)


def _limbs_to_ints(arr: np.ndarray, limbs: int) -> list:
    arr = arr.reshape(-1, limbs)
    if limbs == 2 and not arr[:, 1].any():
        return [int(x) for x in arr[:, 0]]
    out = []
    for row in arr:
        v = 0
        for i in range(limbs - 1, -1, -1):
            v = (v << 64) | int(row[i])
        out.append(v)
    return out


def _ints(row_ptr, col_idx, colours):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    co = np.ascontiguousarray(colours, dtype=np.int8)
    return rp, ci, co


def weights_to_int(weights) -> np.ndarray:
    """float32 arc weights -> exact integers w * 2^24 (uint64)."""
    w = np.asarray(weights, dtype=np.float32).astype(np.float64)
    scaled = w * float(1 << WEIGHT_SHIFT)
    if np.any(scaled < 0) or np.any(scaled != np.floor(scaled)) or np.any(scaled >= 2.0**63):
        raise ValueError("weights must be non-negative float32 values >= 2^-24")
    return np.ascontiguousarray(scaled.astype(np.uint64))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def count(row_ptr, col_idx, parent: Sequence[int], root: int, colours, num_colours: Optional[int] = None,
          weights=None, mode: str = "decoupled", cut: str = "last", per_vertex: bool = True,
          threads: int = 0, min_limbs: int = 2) -> Result:
    """Exact colourful counts by the DP.  Raises on invalid input.  min_limbs
    skips integer widths known to be too narrow (the result is the same)."""
    rp, ci, co = _ints(row_ptr, col_idx, colours)
    n = rp.shape[0] - 1
    par = np.ascontiguousarray(parent, dtype=np.int32)
    k = par.shape[0]
    kc = k if num_colours is None else int(num_colours)
    wint = None if weights is None else weights_to_int(weights)
    m = DECOUPLED if mode == "decoupled" else STANDARD
    c = CUT_LAST if cut == "last" else CUT_FIRST
    for limbs in _build.WIDTHS:
        if limbs < min_limbs and limbs != _build.WIDTHS[-1]:
            continue
        lib = _lib(limbs)
        pv = np.zeros((max(n, 1), limbs), dtype=np.uint64) if per_vertex else None
        tot = np.zeros(limbs, dtype=np.uint64)
        mb = np.zeros(1, dtype=np.int32)
        rc = lib.oracle_dp(n, _ptr(rp), _ptr(ci), _ptr(wint), k, _ptr(par), int(root), kc, _ptr(co), m, c,
                           _ptr(pv), _ptr(tot), _ptr(mb), int(threads))
        if rc == 1:
            continue
        if rc != 0:
            raise ValueError(f"oracle_dp rejected the input (code {rc})")
        total = _limbs_to_ints(tot, limbs)[0]
        pvl = _limbs_to_ints(pv[:n], limbs) if per_vertex else None
        return Result(total, pvl, int(mb[0]), WEIGHT_SHIFT * (k - 1) if wint is not None else 0, limbs)
    raise OverflowError("counts exceed the widest oracle build")


def brute(row_ptr, col_idx, parent: Sequence[int], root: int, colours=None, num_colours: Optional[int] = None,
          weights=None, injective_only: bool = False, threads: int = 0) -> Result:
    """Counts by enumerating every map of the template (small inputs only)."""
    n = np.asarray(row_ptr).shape[0] - 1
    par = np.ascontiguousarray(parent, dtype=np.int32)
    k = par.shape[0]
    kc = k if num_colours is None else int(num_colours)
    if colours is None:
        colours = np.zeros(n, dtype=np.int8)
    rp, ci, co = _ints(row_ptr, col_idx, colours)
    wint = None if weights is None else weights_to_int(weights)
    for limbs in _build.WIDTHS:
        lib = _lib(limbs)
        pv = np.zeros((max(n, 1), limbs), dtype=np.uint64)
        tot = np.zeros(limbs, dtype=np.uint64)
        rc = lib.oracle_brute(n, _ptr(rp), _ptr(ci), _ptr(wint), k, _ptr(par), int(root), kc, _ptr(co),
                              1 if injective_only else 0, _ptr(pv), _ptr(tot), int(threads))
        if rc == 1:
            continue
        if rc != 0:
            raise ValueError(f"oracle_brute rejected the input (code {rc})")
        return Result(_limbs_to_ints(tot, limbs)[0], _limbs_to_ints(pv[:n], limbs), -1,
                      WEIGHT_SHIFT * (k - 1) if wint is not None else 0, limbs)
    raise OverflowError("counts exceed the widest oracle build")


def template_csr(parent: Sequence[int]):
    k = len(parent)
    adj = [[] for _ in range(k)]
    for i, p in enumerate(parent):
        if p >= 0:
            adj[i].append(p)
            adj[p].append(i)
    rp = np.zeros(k + 1, dtype=np.int64)
    ci = []
    for i in range(k):
        nb = sorted(adj[i])
        ci.extend(nb)
        rp[i + 1] = rp[i] + len(nb)
    return rp, np.asarray(ci, dtype=np.int32)


def automorphisms(parent: Sequence[int]) -> int:
    """alpha (Alg. 1): the number of injective maps of T onto itself that keep
    edges, i.e. its automorphisms (unrooted)."""
    rp, ci = template_csr(parent)
    return brute(rp, ci, parent, 0, injective_only=True).total


def colourful_probability(k: int, num_colours: Optional[int] = None) -> Fraction:
    """P of Alg. 1: probability that k given vertices get pairwise distinct
    colours when each draws one of kc colours uniformly."""
    kc = k if num_colours is None else num_colours
    return Fraction(factorial(kc), factorial(kc - k) * kc**k)


def estimate(total, k: int, alpha: int, num_colours: Optional[int] = None) -> Fraction:
    """finalCount of Alg. 1 for one colouring: total / (P * alpha), exact."""
    return Fraction(total) / (colourful_probability(k, num_colours) * alpha)


def py_brute(n: int, edges: Sequence[Sequence[int]], parent: Sequence[int], root: int, colours: Sequence[int],
             weights: Optional[dict] = None):
    """Pure-Python enumeration over all |V|^k vertex tuples (tiny inputs only).
    Returns (per_vertex list, total) as exact ints (or Fractions with weights:
    `weights[(u, v)]` for u < v)."""
    k = len(parent)
    tedges = [(i, p) for i, p in enumerate(parent) if p >= 0]
    eset = set()
    for u, v in edges:
        eset.add((u, v))
        eset.add((v, u))
    per = [0] * n
    for phi in itertools.product(range(n), repeat=k):
        if len({colours[x] for x in phi}) != k:
            continue
        if not all((phi[a], phi[b]) in eset for a, b in tedges):
            continue
        val = 1
        if weights is not None:
            val = Fraction(1)
            for a, b in tedges:
                x, y = phi[a], phi[b]
                val *= Fraction(weights[(min(x, y), max(x, y))])
        per[phi[root]] += val
    return per, sum(per)
