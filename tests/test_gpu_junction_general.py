"""General modified junction trees on the GPU (tree_ot_jt_*): the separator update
of prop:general_algo for nested inclusion sequences, run in FP64 on the device,
against the junction-tree oracle on the same (FP32-rounded) costs.

Both sides compute the same iterates in FP64 in the same order of operations up
to summation order, so dual variables, plans and the stopping quantity agree to
1e-9 (relative, with an absolute floor for entries near zero)."""
import numpy as np
import pytest

import gen
from oracle import junction_tree as JT
from oracle import tree_ot as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    return T


def fp32_costs(jt):
    jt.clique_costs = [np.asarray(C, np.float32).astype(np.float64) for C in jt.clique_costs]
    return jt


def close(a, b, rtol=1e-9, atol=1e-12):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return bool(np.all(np.abs(a - b) <= atol + rtol * np.abs(b)))


def compare_iterates(T, jt, steps):
    from paper_2406_10849_gb300.treeot import JunctionSolver
    ref = JT.run_half_steps(jt, steps)
    with JunctionSolver(jt) as s:
        s.half_steps(steps)
        for (sp, i), (vars_, lu) in ref.items():
            got = s.dual(sp, i)
            fin = np.isfinite(lu)
            assert np.array_equal(np.isfinite(got), fin), (sp, i)
            assert close(np.asarray(got)[fin], np.asarray(lu)[fin], 1e-9, 1e-9), (sp, i, steps)
        plans = JT.plans(jt, ref)
        for c, B in enumerate(plans):
            assert close(s.plan(c), B), (c, steps)
        rs, rm = s.residual()
        ors, orm = JT.residual(jt, ref)
        assert abs(rs - ors) <= 1e-9 * max(1.0, ors) and abs(rm - orm) <= 1e-9 * max(1.0, orm)
        assert abs(s.transport_cost() - JT.transport_cost(jt, ref)) <= 1e-9 * max(1.0, JT.transport_cost(jt, ref))


@pytest.mark.parametrize("d,seed", [(2, 8500), (3, 8501), (4, 8502)])
@pytest.mark.parametrize("steps", [1, 2, 5])
def test_nested_example_iterates(T, d, seed, steps):
    """The nested example of ass:inclusion (separator {x1, x3, x4} meeting its
    cliques in {1,3,4}, {1,3,4}, {1,3}, constraint {x3}; l = 3)."""
    compare_iterates(T, fp32_costs(gen.nested_junction_tree(seed, d=d, eps=0.3)), steps)


@pytest.mark.parametrize("J,d", [(3, 5), (5, 7)])
def test_wls_general_path_iterates(T, J, d):
    """The WLS junction tree (trivially nested, l = J on the free separator) through the
    general update, not the reduction to a tree of separators."""
    jt = fp32_costs(gen.wls_junction_tree(8600 + J, J, d))
    for steps in (1, 3):
        compare_iterates(T, jt, steps)


def test_tree_as_junction_tree_matches_tree_oracle(T):
    """A tree problem written as a junction tree (separators = single nodes) gives the
    tree oracle's plans (Sec. 4 contains Sec. 3)."""
    from paper_2406_10849_gb300.treeot import JunctionSolver
    p = gen.chain_problem(seed=8700, J=4, n=9, eps=0.1)
    jt = gen.tree_as_junction_tree(p)
    steps = 6
    f = O.run_half_steps(p, steps)
    with JunctionSolver(jt) as s:
        s.half_steps(steps)
        for c, (a, b) in enumerate(np.asarray(p.edges)):
            B = O.plan(p, f, int(a), int(b))
            assert close(s.plan(c), B, 1e-8, 1e-12), c


def test_nested_solve_and_cost(T):
    from paper_2406_10849_gb300.treeot import JunctionSolver
    jt = fp32_costs(gen.nested_junction_tree(8800, d=3, eps=0.3))
    du, _, r = JT.solve(jt, tol=1e-10, max_half_steps=200000)
    with JunctionSolver(jt) as s:
        rc, hs, res = s.solve(tol=1e-10, tol_kind="sum", max_half_steps=200000, check_every=8)
        assert rc == 0 and res < 1e-10 and hs > 0
        tc = s.transport_cost()
        plans = [s.plan(c) for c in range(len(jt.clique_vars))]
    assert abs(tc - JT.transport_cost(jt, du)) <= 1e-8 * JT.transport_cost(jt, du)
    for B, Bo in zip(plans, JT.plans(jt, du)):
        assert float(np.abs(B - Bo).sum()) <= 1e-8


def test_reset_and_colours(T):
    from paper_2406_10849_gb300.treeot import JunctionSolver
    jt = fp32_costs(gen.nested_junction_tree(8900, d=2, eps=0.5))
    with JunctionSolver(jt) as s:
        assert list(s.colours()) == list(JT.colours(jt))
        s.half_steps(3)
        a = s.plan(0)
        s.reset()
        s.half_steps(3)
        assert np.array_equal(s.plan(0), a)


def test_broken_structures_are_rejected(T):
    from paper_2406_10849_gb300.treeot import JunctionSolver, TreeOTError
    jt = gen.nested_junction_tree(9000, d=2)
    bad = gen.nested_junction_tree(9000, d=2)
    bad.sep_cliques = [[2, 0, 1], [0], [1], [2]]   # first two intersections differ
    with pytest.raises(TreeOTError) as e:
        JunctionSolver(bad)
    assert e.value.kind == "NOT_TREE"
    bad = gen.nested_junction_tree(9000, d=2)
    bad.sep_mu = list(bad.sep_mu)
    bad.sep_mu[1] = np.asarray(bad.sep_mu[1]) * 2.0   # not a probability vector
    with pytest.raises(TreeOTError) as e:
        JunctionSolver(bad)
    assert e.value.kind == "MARGINAL"
    with JunctionSolver(jt) as s:   # a valid one still works
        s.half_steps(1)


def test_graph_replay_matches_single_half_steps(T):
    """Runs of two or more half-steps replay a captured pair of half-steps; the
    iterates are bit-identical to the same half-steps launched one at a time."""
    from paper_2406_10849_gb300.treeot import JunctionSolver
    jt = fp32_costs(gen.nested_junction_tree(9100, d=3, eps=0.3))
    with JunctionSolver(jt) as a, JunctionSolver(jt) as b:
        a.half_steps(1)
        a.half_steps(6)        # odd start: one single, then three pairs
        a.half_steps(2)
        for _ in range(9):
            b.half_steps(1)
        for c in range(len(jt.clique_vars)):
            assert np.array_equal(a.plan(c), b.plan(c)), c
