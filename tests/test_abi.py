"""Host-side checks of the C ABI: the library loads, exports every entry
point its header declares, and its planner (pure host code) agrees with the
paper's definitions (Sec. 2.3.2 partitioning, Alg. 1 alpha and P)."""
import os
import re
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import oracle
import sg2v_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2009_11665_b300 as s

    return s


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sg2v_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "sg2v_count" in declared and "sg2v_graph_create" in declared
    for name in declared:
        assert hasattr(lib._lib, name), name
    assert set(lib.EXPORTED) <= declared


def test_binding_constants_match_header(lib):
    """Every enumerator and flag the header defines has the same value in
    the Python binding (the binding only marshals)."""
    text = open(os.path.join(ROOT, "include", "sg2v.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = {m[0]: int(m[1]) for m in re.findall(r"\b(SG2V_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    consts.update({m[0]: int(m[1], 16) for m in re.findall(r"#define\s+(SG2V_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+)u", text)})
    assert "SG2V_FP32_SCALED" in consts and "SG2V_SESSION_AUTOTUNE" in consts
    for name, value in consts.items():
        assert getattr(lib, name) == value, name


def test_version_and_status_strings(lib):
    assert lib.sg2v_version() >= 100
    for code in range(10):
        assert lib.sg2v_status_string(code)
    assert lib.sg2v_status_string(3) == "colour out of range"


TREES = [(-1,), (-1, 0), (-1, 0, 1), (-1, 0, 0), (-1, 0, 1, 1), (-1, 0, 0, 0), si.PATH5.parent, si.PATH7.parent,
         si.STAR7.parent, si.TREE7.parent, si.TREE8.parent, si.TREE10.parent, si.TREE15.parent,
         (-1, 0, 1, 2, 2, 0), (-1, 0, 0, 1, 2, 3)]


@pytest.mark.parametrize("parent", TREES)
def test_automorphisms_match_oracle(lib, parent):
    """The planner's alpha (AHU canonical forms) equals the oracle's
    brute-force count of self-maps."""
    plan = lib.Plan(parent)
    assert plan.alpha == oracle.automorphisms(parent)


def _subtree_sizes(parent, root):
    k = len(parent)
    adj = [[] for _ in range(k)]
    for i, p in enumerate(parent):
        if p >= 0:
            adj[i].append(p)
            adj[p].append(i)
    size = {}

    def go(x, frm):
        s = 1
        for y in adj[x]:
            if y != frm:
                s += go(y, x)
        size[x] = s
        return s

    go(root, -1)
    return [size[v] for v in range(k) if v != root]


@pytest.mark.parametrize("parent", TREES)
def test_plan_structure(lib, parent):
    """Children precede parents, t = a + p, the root node has t = k and the
    passive sub-templates are exactly the subtrees hanging below rho's
    descendants (sum over cuts of C(kc, p) = sum over non-root v of
    C(kc, |subtree(v)|) before sharing)."""
    k = len(parent)
    for root in range(k):
        plan = lib.Plan(parent, root)
        nodes = plan.nodes()
        if k == 1:
            assert nodes == []
            continue
        sizes = {}
        for i, (t, a, p, ia, ip, is_root) in enumerate(nodes):
            assert t == a + p and a >= 1 and p >= 1
            for child, sz in ((ia, a), (ip, p)):
                if child == -1:
                    assert sz == 1
                else:
                    assert 0 <= child < i and nodes[child][0] == sz
            sizes[i] = t
            assert is_root == (i == len(nodes) - 1)
        assert nodes[-1][0] == k
        # expand shared nodes back into the full partition tree and compare
        def passives(i):
            t, a, p, ia, ip, _ = nodes[i]
            out = [p]
            if ia != -1:
                out += passives(ia)
            if ip != -1:
                out += passives(ip)
            return out

        assert sorted(passives(len(nodes) - 1)) == sorted(_subtree_sizes(parent, root))


def test_estimate_scale(lib):
    """1/(P alpha) with P = kc!/((kc-k)! kc^k) (Alg. 1)."""
    for parent in TREES:
        k = len(parent)
        for kc in (k, k + 1):
            if kc > 16:
                continue
            plan = lib.Plan(parent, 0, kc)
            expect = Fraction(kc ** k * factorial(kc - k), factorial(kc) * plan.alpha)
            assert plan.scale == float(expect)


def test_invalid_templates(lib):
    with pytest.raises(lib.Sg2vError) as e:
        lib.Plan((-1, -1, 0))
    assert e.value.status == lib.SG2V_ERR_NOT_A_TREE
    with pytest.raises(lib.Sg2vError) as e:
        lib.Plan((1, 2, 0))
    assert e.value.status == lib.SG2V_ERR_NOT_A_TREE
    with pytest.raises(lib.Sg2vError) as e:
        lib.Plan((-1, 0, 5))
    assert e.value.status == lib.SG2V_ERR_NOT_A_TREE
    with pytest.raises(lib.Sg2vError) as e:
        lib.Plan((-1, 0), root=2)
    assert e.value.status == lib.SG2V_ERR_NOT_A_TREE
    with pytest.raises(lib.Sg2vError) as e:
        lib.Plan((-1, 0, 1), num_colours=2)
    assert e.value.status == lib.SG2V_ERR_INVALID_ARGUMENT
    with pytest.raises(lib.Sg2vError) as e:
        lib.Plan((-1,) + (0,) * 16)
    assert e.value.status == lib.SG2V_ERR_UNSUPPORTED


def test_plan_options(lib):
    """Plan options: a wrong struct size, cut rule or degree is rejected;
    cut-last options give the default plan."""
    import ctypes

    par = np.ascontiguousarray(si.TREE10.parent, dtype=np.int32)
    h = ctypes.c_void_p()
    for size, cut, deg in ((4, 0, 0.0), (ctypes.sizeof(lib.PlanOpts), 7, 0.0),
                           (ctypes.sizeof(lib.PlanOpts), 1, -1.0)):
        o = lib.PlanOpts(size, cut, deg)
        st = lib._lib.sg2v_template_plan(10, par.ctypes.data_as(ctypes.c_void_p), 0, 10, ctypes.byref(o),
                                         ctypes.byref(h))
        assert st == lib.SG2V_ERR_INVALID_ARGUMENT
    assert lib.Plan(si.TREE10.parent, cut="last").nodes() == lib.Plan(si.TREE10.parent).nodes()


def _check_decomposition(nodes, k):
    """Every node splits t = a + p with children that exist and have those
    sizes; the root covers the template."""
    size = {-1: 1}
    for i, (t, a, p, ia, ip, is_root) in enumerate(nodes):
        assert t == a + p and a >= 1 and p >= 1
        assert ia < i and ip < i
        assert size[ia] == a and size[ip] == p
        size[i] = t
    assert nodes[-1][5] == 1 and nodes[-1][0] == k
    assert sum(n[5] for n in nodes) == 1


@pytest.mark.parametrize("seed", range(6))
def test_min_work_plans_are_decompositions(lib, seed):
    """Work-minimising cut orders still give a valid partition of the
    template (Sec. 2.3.2), with the same alpha and estimate scale; tree10
    takes the alternative plan (a (4,2,2) node) at average degree 32."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(3, 13))
    parent = [-1] + [int(rng.integers(0, i)) for i in range(1, k)]
    for deg in (8.0, 32.0, 95.0):
        a = lib.Plan(parent)
        b = lib.Plan(parent, cut="min_work", avg_degree=deg)
        _check_decomposition(b.nodes(), k)
        assert (a.alpha, a.scale) == (b.alpha, b.scale)
    t10 = lib.Plan(si.TREE10.parent, cut="min_work", avg_degree=32.0).nodes()
    _check_decomposition(t10, 10)
    assert [n[:3] for n in t10] == [(2, 1, 1), (4, 2, 2), (5, 1, 4), (10, 5, 5)]


def test_sharing_of_isomorphic_subtemplates(lib):
    """tree10's two halves below the root are isomorphic rooted trees: the
    root node reads one shared table as both children."""
    nodes = lib.Plan(si.TREE10.parent).nodes()
    assert len(nodes) == 5
    t, a, p, ia, ip, _ = nodes[-1]
    assert (t, a, p) == (10, 5, 5) and ia == ip
