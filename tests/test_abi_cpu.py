"""CPU-only checks of the C ABI: the library loads, exports every symbol that
include/tree_ot.h declares, and its host-side logic (validation, two-colouring)
agrees with the oracle.  No CUDA compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import gen
from oracle import tree_ot as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tree_ot.h")


@pytest.fixture(scope="module")
def T():
    import paper_2406_10849_gb300 as T
    if not os.path.exists(T.LIB_PATH):
        from paper_2406_10849_gb300 import _build
        _build.build()
    T.load()
    return T


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tree_ot_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(T):
    lib = ctypes.CDLL(T.LIB_PATH)
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(T.SIGNATURES), set(names) ^ set(T.SIGNATURES)


def test_error_strings(T):
    lib = T.load()
    for code in [0, 1, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10, -11]:
        assert lib.tree_ot_error_string(code)


def test_default_options(T):
    o = T.options()
    assert o.tol == 1e-6 and o.check_every == 32 and o.use_graph == 1


def header_option_bits():
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (TREE_OT_OPT_[A-Z_0-9]+)\s+(\d+)u", open(HEADER).read())}


def test_option_flags_match_header(T):
    """The binding's option names set the bits the header defines, each bit once."""
    bits = header_option_bits()
    assert len(set(bits.values())) == len(bits)
    want = {("dense_kernel", "tma"): "DENSE_TMA", ("dense_kernel", "ldg"): "DENSE_LDG",
            ("exact_dist", True): "EXACT_DIST", ("transpose", False): "NO_TRANSPOSE",
            ("test_stall", True): "TEST_STALL", ("sk_product", "mma"): "SK_MMA_SYNC",
            ("sk_product", "one_cta"): "SK_ONE_CTA", ("persistent", True): "PERSISTENT",
            ("node_finish", "defer"): "NODE_DEFER", ("node_finish", "arrive"): "NODE_ARRIVE"}
    assert set(want.values()) == {k[len("TREE_OT_OPT_"):] for k in bits}
    assert T.options().flags == 0
    for (key, value), name in want.items():
        assert T.options(**{key: value}).flags == bits["TREE_OT_OPT_" + name], (key, value)


@pytest.mark.parametrize("J", [2, 3, 7, 64, 200])
def test_bipartition_matches_oracle(T, J):
    rng = np.random.default_rng(J)
    edges = gen.uniform_pruefer_tree(J, rng)
    np.testing.assert_array_equal(T.bipartition(J, edges), O.bipartition(J, edges))


def _kind(T, p):
    return T.treeot.ERR.get(T.validate(p), "OK") if T.validate(p) else "OK"


def test_validation_codes_match_oracle(T):
    cases = []
    p = gen.chain_problem(n=6)
    cases.append(p)
    bad = gen.chain_problem(n=6)
    bad.edges = np.array([[0, 1], [1, 2], [2, 0], [3, 4]], np.int32)
    cases.append(bad)
    bad = gen.chain_problem(n=6)
    bad.fixed[2] = True
    bad.marginals[2] = np.full(6, 1 / 6)
    cases.append(bad)
    bad = gen.chain_problem(n=6)
    bad.marginals[0] = bad.marginals[0] * 2
    cases.append(bad)
    bad = gen.chain_problem(n=6)
    bad.eps = -1.0
    cases.append(bad)
    bad = gen.chain_problem(n=6)
    bad.marginals[4] = bad.marginals[4].copy()
    bad.marginals[4][0] = -0.1
    bad.marginals[4][1] += 0.1
    cases.append(bad)
    two = gen.chain_problem(J=2, n=3)
    cases.append(two)
    for c in cases:
        try:
            O.validate(c)
            want = "OK"
        except O.TreeError as e:
            want = e.kind
        got = _kind(T, c)
        assert got == want, (c.name, got, want)


def test_disconnected_and_self_loop(T):
    p = gen.chain_problem(J=4, n=3)
    p.edges = np.array([[0, 1], [1, 1], [2, 3]], np.int32)
    assert T.validate(p) == -2
    p.edges = np.array([[0, 1], [0, 1], [2, 3]], np.int32)
    assert T.validate(p) == -2


def test_junction_tree_structure_checks_on_host(T):
    """tree_ot_jt_create checks def:jt_general and ass:inclusion on the host before
    any device call: broken structures are refused with their codes."""
    from paper_2406_10849_gb300.treeot import JunctionSolver, TreeOTError

    def code_of(jt):
        try:
            JunctionSolver(jt).close()
        except TreeOTError as e:
            return e.kind
        return "OK"

    bad = gen.nested_junction_tree(9000, d=2)
    bad.sep_cliques = [[2, 0, 1], [0], [1], [2]]        # first two intersections differ
    assert code_of(bad) == "NOT_TREE"
    bad = gen.nested_junction_tree(9000, d=2)
    bad.sep_gamma = list(bad.sep_gamma)
    bad.sep_gamma[0] = (4,)                              # constraint outside the smallest intersection
    bad.sep_mu = list(bad.sep_mu)
    assert code_of(bad) == "NOT_TREE"
    bad = gen.nested_junction_tree(9000, d=2)
    bad.sep_cliques = [[0, 1, 2], [0], [1], [1]]         # clique 1 joins three separators, clique 2 one
    assert code_of(bad) == "NOT_TREE"
    bad = gen.nested_junction_tree(9000, d=2)
    bad.sep_mu = list(bad.sep_mu)
    bad.sep_mu[2] = np.asarray(bad.sep_mu[2]) * 0.5     # not a probability vector
    assert code_of(bad) == "MARGINAL"
    bad = gen.nested_junction_tree(9000, d=2)
    bad.eps = 0.0
    assert code_of(bad) == "EPS"
    bad = gen.nested_junction_tree(9000, d=2)
    bad.clique_costs = list(bad.clique_costs)
    bad.clique_costs[1] = np.array(bad.clique_costs[1], dtype=np.float64)
    bad.clique_costs[1].reshape(-1)[0] = np.nan
    assert code_of(bad) == "NONFINITE"
