"""Pins for the oracle's rounding (the rounding algorithm of Sec. 3.1 with Altschuler,
Weed and Rigollet's Algorithm 2; lemmas lem:round and lem:round_applied, Sec. 3.2).

Each test checks the oracle against something other than itself: a 2 x 2 rounding
and a 3-leaf star worked by hand, the guarantees Altschuler et al. prove for their
routine, exact feasibility of the rounded plans for the unregularised problem, the
paper's two error bounds, and an LP solver (a feasible plan cannot beat the LP
optimum).  Planted mistakes each fail at least one of them.
"""
import math
import os

import numpy as np
import pytest

import gen
from oracle import tree_ot as O
import textbook_ot as TB
from test_oracle_pins import _read_golden, _star3_problem, random_small_tree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_round_matrix_2x2():
    """F = [[.2, .3], [.1, .4]], r = (.4, .6), c = F^T 1 = (.3, .7): rows scaled by
    (min(.4/.5, 1), min(.6/.5, 1)) = (.8, 1); the columns of F' = [[.16, .24], [.1, .4]]
    sum to (.26, .64) <= c; err_r = (0, .1), err_c = (.04, .06), E = .1;
    G = F' + err_r err_c^T / E = [[.16, .24], [.14, .46]]."""
    F = np.array([[0.2, 0.3], [0.1, 0.4]])
    G = O.round_matrix(F, np.array([0.4, 0.6]), F.sum(axis=0))
    np.testing.assert_allclose(G, [[0.16, 0.24], [0.14, 0.46]], rtol=0, atol=1e-16)


def test_golden_star_rounding_after_one_half_step():
    g = _read_golden("star3_residual_2pt.txt")
    r = _read_golden("star3_round_2pt.txt")
    p = _star3_problem(g)
    f = O.run_half_steps(p, 1)
    side = O.mismatched_side(1)
    colour = O.bipartition(p.num_nodes, p.edges)
    assert side == 1 and all(colour[k] == 1 for k in (1, 2, 3))
    R = O.round_plans(p, f, side)
    assert sorted(R) == [(1, 0), (2, 0), (3, 0)]
    for k in (1, 2, 3):
        np.testing.assert_allclose(R[(k, 0)].reshape(-1), r[f"plan_{k}"], rtol=0, atol=1e-15)
    assert abs(O.rounded_transport_cost(p, R) - r["rounded_transport_cost"][0]) < 1e-15
    assert abs(O.final_check(p, f)["transport_cost"] - r["transport_cost"][0]) < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_round_matrix_guarantees(seed):
    """Altschuler et al., Lemma 7: G >= 0, G 1 = r, G^T 1 = c and
    ||G - F||_1 <= 2 (||F 1 - r||_1 + ||F^T 1 - c||_1), for any F >= 0 and any r, c of equal mass."""
    rng = np.random.default_rng(seed)
    m, n = rng.integers(1, 9, size=2)
    F = rng.random((m, n)) * (rng.random((m, n)) > 0.3)
    r = rng.dirichlet(np.ones(m))
    c = rng.dirichlet(np.ones(n))
    G = O.round_matrix(F, r, c)
    assert np.all(G >= 0)
    np.testing.assert_allclose(G.sum(axis=1), r, rtol=0, atol=1e-15)
    np.testing.assert_allclose(G.sum(axis=0), c, rtol=0, atol=1e-15)
    bound = 2 * (np.abs(F.sum(axis=1) - r).sum() + np.abs(F.sum(axis=0) - c).sum())
    assert np.abs(G - F).sum() <= bound + 1e-15


def _trajectory_rounds(p, Ts):
    colour = O.bipartition(p.num_nodes, p.edges)
    f = O.zero_potentials(p)
    out = {}
    for t in range(1, max(Ts) + 1):
        f, _ = O.half_step(p, f, colour, 0 if t % 2 == 1 else 1)
        if t in Ts:
            out[t] = (dict(f), O.round_plans(p, f, O.mismatched_side(t)))
    return out


def _feasibility_gap(p, R):
    """Largest violation of the constraints of the unregularised problem: fixed node
    marginals equal mu, every free node's plans share one marginal, masses 1."""
    nb = O.neighbours(p.num_nodes, p.edges)

    def marg(j, k):
        return R[(j, k)].sum(axis=1) if (j, k) in R else R[(k, j)].sum(axis=0)
    worst = 0.0
    for j in range(p.num_nodes):
        qs = [marg(j, k) for k in nb[j]]
        ref = p.marginals[j] if p.fixed[j] else qs[0]
        worst = max(worst, max(float(np.abs(q - ref).sum()) for q in qs), abs(float(qs[0].sum()) - 1.0))
        assert all(np.all(R[key] >= 0) for key in R)
    return worst


@pytest.mark.parametrize("seed,J", [(61, 4), (62, 6), (63, 9)])
def test_rounded_plans_are_feasible_and_keep_the_updated_side(seed, J):
    p = random_small_tree(seed, J, nmin=2, nmax=5, eps=0.1)
    for t, (f, R) in _trajectory_rounds(p, {1, 2, 3, 8}).items():
        assert _feasibility_gap(p, R) <= 1e-14, t
        # the side updated last keeps its marginals: the column sums of every rounded plan
        for (j, k), B in R.items():
            np.testing.assert_allclose(B.sum(axis=0), O.plan(p, f, j, k).sum(axis=0), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed,J", [(71, 4), (72, 5), (73, 6)])
def test_rounding_error_bounds(seed, J):
    """Lemma lem:round: |TC(B) - TC(B^)| <= 2 C_inf r(B); lemma lem:round_applied:
    TC(B^) - OPT <= 2 eps |E| log d + 4 C_inf r(B); and OPT <= TC(B^) because the rounded
    plans are feasible for the unregularised problem (OPT from an LP solver)."""
    p = random_small_tree(seed, J, nmin=3, nmax=4, eps=0.05)
    costs = [O.cost(p, int(a), int(b)) for a, b in p.edges]
    opt = TB.lp_optimum(p.num_nodes, [tuple(map(int, e)) for e in p.edges], [int(x) for x in p.n],
                        p.fixed, p.marginals, costs)
    cinf = O.c_infinity(p)
    d = int(p.n.max())
    for t, (f, R) in _trajectory_rounds(p, {1, 2, 5, 20, 200}).items():
        r = O.residual(p, f)[0]
        tc = O.final_check(p, f)["transport_cost"]
        tr = O.rounded_transport_cost(p, R)
        assert abs(tc - tr) <= 2 * cinf * r + 1e-13, t
        assert opt - 1e-9 <= tr <= opt + 2 * p.eps * p.num_edges * math.log(d) + 4 * cinf * r + 1e-12, t


def test_rounding_changes_converged_plans_only_by_the_residual():
    p = random_small_tree(74, 6, nmin=3, nmax=5, eps=0.2)
    f, T, r = O.solve(p, tol=1e-12)
    R = O.round_plans(p, f, O.mismatched_side(T))
    for (j, k), B in R.items():
        assert np.abs(B - O.plan(p, f, j, k)).sum() <= 4 * r + 1e-15


def _round_pins_pass():
    try:
        test_golden_round_matrix_2x2()
        test_golden_star_rounding_after_one_half_step()
        for s in range(3):
            test_round_matrix_guarantees(s)
        test_rounded_plans_are_feasible_and_keep_the_updated_side(61, 4)
        test_rounding_error_bounds(71, 4)
    except Exception:
        return False
    return True


def test_planted_rounding_mistakes_are_caught(monkeypatch):
    assert _round_pins_pass()
    real_round_matrix = O.round_matrix
    real_side = O.mismatched_side
    real_round_plans = O.round_plans

    def no_correction(F, r, c):
        x = np.minimum(r / np.maximum(F.sum(axis=1), 1e-300), 1.0)
        return x[:, None] * F

    def plain_row_scaling(F, r, c):      # rows to r exactly, columns left to drift
        return (r / np.maximum(F.sum(axis=1), 1e-300))[:, None] * F

    def no_column_scale(F, r, c):        # the column step skipped and the correction added anyway
        x = np.minimum(r / np.maximum(F.sum(axis=1), 1e-300), 1.0)
        F1 = x[:, None] * F
        er, ec = r - F1.sum(axis=1), F.sum(axis=0) - F1.sum(axis=0)
        return F1 + np.outer(er, ec) / max(er.sum(), 1e-300)

    for name, fn in [("no rank-one correction", no_correction), ("plain row scaling", plain_row_scaling),
                     ("column errors against F instead of c", no_column_scale)]:
        monkeypatch.setattr(O, "round_matrix", fn)
        assert not _round_pins_pass(), name
    monkeypatch.setattr(O, "round_matrix", real_round_matrix)

    monkeypatch.setattr(O, "mismatched_side", lambda T: (T + 1) % 2)
    assert not _round_pins_pass(), "rounds the side updated last"
    monkeypatch.setattr(O, "mismatched_side", real_side)

    def geometric_target(problem, f, side):
        colour = O.bipartition(problem.num_nodes, problem.edges)
        nb = O.neighbours(problem.num_nodes, problem.edges)
        out = {}
        for j in range(problem.num_nodes):
            if colour[j] != side:
                continue
            Bs = {k: O.plan(problem, f, j, k) for k in nb[j]}
            if problem.fixed[j]:
                target = problem.marginals[j]
            else:
                target = np.exp(sum(np.log(B.sum(axis=1)) for B in Bs.values()) / len(nb[j]))
            for k in nb[j]:
                out[(j, k)] = O.round_matrix(Bs[k], target, Bs[k].sum(axis=0))
        return out
    monkeypatch.setattr(O, "round_plans", geometric_target)
    assert not _round_pins_pass(), "geometric mean as the free node's target"

    def own_rows_target(problem, f, side):
        colour = O.bipartition(problem.num_nodes, problem.edges)
        nb = O.neighbours(problem.num_nodes, problem.edges)
        out = {}
        for j in range(problem.num_nodes):
            if colour[j] != side:
                continue
            for k in nb[j]:
                B = O.plan(problem, f, j, k)
                target = problem.marginals[j] if problem.fixed[j] else B.sum(axis=1)
                out[(j, k)] = O.round_matrix(B, target, B.sum(axis=0))
        return out
    monkeypatch.setattr(O, "round_plans", own_rows_target)
    assert not _round_pins_pass(), "each free edge rounded to its own row sums"
    monkeypatch.setattr(O, "round_plans", real_round_plans)
    assert _round_pins_pass()
