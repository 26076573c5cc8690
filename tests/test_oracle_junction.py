"""Pins for the junction-tree oracle (Sec. 4: eq. ot_graph_local_reg, prop:local_reg_dual,
prop:general_algo).

* A tree problem written as a modified junction tree (cliques = edges, separators =
  nodes) gives the same plans as the tree oracle after every half-step, which is
  pinned independently (tests/test_oracle_pins.py): the separator update with equal
  intersections is the free-node update of thm:tree_dual_var.
* On the nested example of Sec. 4 (intersections {1,3,4} = {1,3,4} >= {1,3}, gamma
  = {3}) and on a Wasserstein least-squares instance, the converged plans equal
  those of a generic convex solver of eq. ot_graph_local_reg, blind to the
  algorithm (Newton on the Lagrangian dual).
* The transport cost is at least the optimum of the unregularised multi-marginal
  LP over the joint distribution (the coupled problem over a junction tree has the
  same optimum) and approaches it as eps shrinks.
* Planted mistakes in the nested update fail the generic-solver pin.
"""
import numpy as np
import pytest

import gen
from oracle import junction_tree as JT
from oracle import tree_ot as O
import textbook_ot as TB
from test_oracle_pins import random_small_tree


@pytest.mark.parametrize("seed,J", [(21, 3), (22, 5), (41, 7)])
def test_tree_as_junction_tree_equals_tree_oracle(seed, J):
    p = random_small_tree(seed, J, nmin=2, nmax=4, eps=0.3)
    jt = gen.tree_as_junction_tree(p)
    JT.validate(jt)
    for T in (1, 2, 3, 8):
        f = O.run_half_steps(p, T)
        du = JT.run_half_steps(jt, T)
        Bj = JT.plans(jt, du)
        for e, (a, b) in enumerate(np.asarray(p.edges)):
            B = O.plan(p, f, int(a), int(b))
            got = Bj[e] if int(a) < int(b) else Bj[e].T
            np.testing.assert_allclose(got, B, rtol=1e-12, atol=1e-15)


def _converged(jt, tol=1e-13, max_half_steps=200000):
    du, T, r = JT.solve(jt, tol=tol, max_half_steps=max_half_steps)
    assert r < tol, (T, r)
    return du


@pytest.mark.parametrize("seed,d", [(2, 2), (3, 3)])
def test_nested_example_matches_generic_solver(seed, d, max_half_steps=200000):
    jt = gen.nested_junction_tree(seed, d=d, eps=0.5)
    JT.validate(jt)
    du = _converged(jt, max_half_steps=max_half_steps)
    plans, val = TB.jt_primal_generic(jt)
    for B, Bg in zip(JT.plans(jt, du), plans):
        np.testing.assert_allclose(B, Bg, rtol=1e-8, atol=1e-13)
    assert abs(JT.primal(jt, du) - val) < 1e-10


def test_wls_matches_generic_solver():
    jt = gen.wls_junction_tree(5, 3, 4)
    jt.eps = 0.2
    du = _converged(jt, tol=1e-12)
    plans, val = TB.jt_primal_generic(jt)
    for B, Bg in zip(JT.plans(jt, du), plans):
        np.testing.assert_allclose(B, Bg, rtol=1e-7, atol=1e-13)
    assert abs(JT.primal(jt, du) - val) < 1e-9


@pytest.mark.parametrize("make", ["nested", "wls"])
def test_lp_limit(make):
    """OPT_MOT <= TC(B_eps), and TC(B_eps) - OPT_MOT shrinks with eps."""
    base = gen.nested_junction_tree(4, d=2) if make == "nested" else gen.wls_junction_tree(6, 2, 3)
    opt = TB.mot_lp_optimum(base)
    gaps = []
    for eps in (0.2, 0.05, 0.0125):
        base.eps = eps
        du = _converged(base, tol=1e-11)
        tc = JT.transport_cost(base, du)
        assert tc >= opt - 1e-9, (eps, tc, opt)
        gaps.append(tc - opt)
    assert gaps[2] < gaps[0] and gaps[2] < 0.1


def test_validation_rejects_broken_structures():
    jt = gen.nested_junction_tree(2)
    jt.sep_cliques[0] = [2, 0, 1]          # {1,3} first: not an inclusion sequence
    with pytest.raises(ValueError):
        JT.validate(jt)
    jt = gen.nested_junction_tree(2)
    jt.sep_cliques[1] = [0, 1]             # clique 1 joined to three separators
    with pytest.raises(ValueError):
        JT.validate(jt)


def _nested_pin_passes():
    try:
        test_nested_example_matches_generic_solver(2, 2, max_half_steps=2000)
        test_tree_as_junction_tree_equals_tree_oracle(22, 5)
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _nested_pin_passes()
    real_project, real_chain, real_inter = JT.project, JT.geometric_chain, JT.intermediates

    def projection_as_max(t, keep):          # a marginal taken by max instead of sum
        vars_, a = t
        axes = tuple(i for i, v in enumerate(vars_) if v not in keep)
        if not axes:
            return real_project(t, keep)
        out = np.max(np.asarray(a, dtype=np.float64), axis=axes)
        kept = tuple(v for v in vars_ if v in keep)
        order = [kept.index(v) for v in keep]
        return tuple(keep), np.transpose(out, order) if np.ndim(out) > 1 else out

    def chain_without_weight(k, sets):       # q_i = (P(q_{i-1}) k_i)^(1/i): the exponent i-1 dropped
        q, Pq = real_chain(k, sets)
        for i in range(3, len(k) + 1):
            q[i] = (sets[i - 1], (Pq[i][1] + k[i - 1][1]) / i)
        return q, Pq

    def plain_mean_scale(jt, q, Pq, sets, g):  # v_{l+1} without its power l
        a = real_inter(jt, q, Pq, sets, g)
        l = len(sets)
        return [None if x is None else (x[0], x[1] - (l - 1) / l * JT.expand((g, -JT.project(q[l], g)[1]), x[0], jt.d))
                for x in a]

    for name, attr, fn in [("projection by max", "project", projection_as_max),
                           ("nested mean without its weight", "geometric_chain", chain_without_weight),
                           ("v_{l+1} without its power", "intermediates", plain_mean_scale)]:
        monkeypatch.setattr(JT, attr, fn)
        assert not _nested_pin_passes(), name
        monkeypatch.setattr(JT, "project", real_project)
        monkeypatch.setattr(JT, "geometric_chain", real_chain)
        monkeypatch.setattr(JT, "intermediates", real_inter)
    assert _nested_pin_passes()
