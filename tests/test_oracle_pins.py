"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form
worked by hand, an independent textbook algorithm, a general-purpose optimiser,
an LP solver, or an inequality the paper proves.  A dropped term, a wrong sign,
a wrong index or a transposed operand in the oracle fails at least one of them
(``test_planted_mistakes_are_caught`` plants such mistakes and checks that).
"""
import math
import os

import numpy as np
import pytest

import gen
from gen.problems import TreeProblem
from oracle import tree_ot as O
import textbook_ot as TB

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_problem(edges, n, fixed, marginals, costs, eps, name="t"):
    edges = np.asarray(edges, np.int32).reshape(-1, 2)
    n = np.asarray(n, np.int32)
    J = n.shape[0]
    coords = [np.zeros((int(n[j]), 1), np.float32) for j in range(J)]
    return TreeProblem(name=name, edges=edges, n=n, fixed=np.asarray(fixed, bool), marginals=marginals,
                       eps=eps, coords=coords, cost_scale=1.0, cost_kind="dense",
                       dense_costs=[np.asarray(C, np.float32) for C in costs])


def random_small_tree(seed, J, nmin=2, nmax=5, eps=0.3):
    """Small random tree with fixed leaves, unequal supports and FP32-exact costs."""
    rng = np.random.default_rng(seed)
    edges = gen.uniform_pruefer_tree(J, rng)
    fixed = gen.leaves_of(J, edges)
    n = rng.integers(nmin, nmax + 1, size=J)
    marg = {j: gen.dirichlet_marginal(int(n[j]), rng) for j in range(J) if fixed[j]}
    costs = [rng.random((int(n[a]), int(n[b]))).astype(np.float32) for a, b in edges]
    return dense_problem(edges, n, fixed, marg, costs, eps)


def converged(p, tol=1e-13, max_half_steps=20000):
    f, T, r = O.solve(p, tol=tol, max_half_steps=max_half_steps)
    assert r < tol, (T, r)
    return f


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=")
            vals[k.strip()] = np.array([float(t) for t in v.split()])
    return vals


def test_golden_single_edge_two_points():
    g = _read_golden("single_edge_2pt.txt")
    p = dense_problem([[0, 1]], [2, 2], [True, False], {0: g["mu"]}, [g["cost"].reshape(2, 2)],
                      float(g["eps"][0]))
    f = O.run_half_steps(p, 2)
    B = O.plan(p, f, 0, 1)
    np.testing.assert_allclose(B.reshape(-1), g["plan"], rtol=0, atol=1e-15)
    fc = O.final_check(p, f)
    np.testing.assert_allclose(fc["marginals"][1], g["free_marginal"], rtol=0, atol=1e-15)
    assert abs(fc["transport_cost"] - g["transport_cost"][0]) < 1e-15


def _star3_problem(g):
    """Centre 0 free, leaves 1..3 fixed, two points each; C_(0,k) = [[0, c_k], [c_k, 0]]."""
    mus = {k + 1: np.array([g["p"][k], 1.0 - g["p"][k]]) for k in range(3)}
    costs = [np.array([[0.0, ck], [ck, 0.0]]) for ck in g["c"]]
    return dense_problem([[0, 1], [0, 2], [0, 3]], [2, 2, 2, 2], [False, True, True, True], mus, costs,
                         float(g["eps"][0]))


def test_golden_stopping_quantity_away_from_convergence():
    """The stopping quantity at u = 1 and after one and two half-steps, against the hand-worked
    values of a 3-leaf star (arithmetic mean qbar in the free-node terms; the update's geometric
    mean gives other values at degree 3)."""
    g = _read_golden("star3_residual_2pt.txt")
    p = _star3_problem(g)
    order = [(1, 0), (2, 0), (3, 0), (0, 1), (0, 2), (0, 3)]
    for t in range(3):
        f = O.run_half_steps(p, t)
        r, rmax, terms = O.residual(p, f)
        np.testing.assert_allclose([terms[k] for k in order], g[f"terms_t{t}"], rtol=0, atol=1e-14)
        assert abs(r - g[f"sum_t{t}"][0]) < 1e-14
        assert abs(rmax - g[f"max_t{t}"][0]) < 1e-15


@pytest.mark.parametrize("fixed_first", [True, False])
def test_single_edge_closed_form(fixed_first):
    """Fixed-free edge: B = diag(mu ./ (K 1)) K after one update of each node."""
    rng = np.random.default_rng(7)
    na, nb = 5, 7
    mu = gen.dirichlet_marginal(na, rng)
    C = rng.random((na, nb)).astype(np.float32)
    if fixed_first:
        p = dense_problem([[0, 1]], [na, nb], [True, False], {0: mu}, [C], 0.2)
        fx, fr = 0, 1
    else:
        p = dense_problem([[0, 1]], [nb, na], [False, True], {1: mu}, [C.T.copy()], 0.2)
        fx, fr = 1, 0
    K = np.exp(-C.astype(np.float64) / 0.2)
    expect = mu[:, None] * K / K.sum(axis=1, keepdims=True)
    f = O.run_half_steps(p, 2)
    np.testing.assert_allclose(O.plan(p, f, fx, fr), expect, rtol=1e-13, atol=1e-16)
    f = O.run_half_steps(p, 6)
    np.testing.assert_allclose(O.plan(p, f, fx, fr), expect, rtol=1e-13, atol=1e-16)


# ---------------------------------------------------------------------------
# special cases that reduce to textbook algorithms
# ---------------------------------------------------------------------------

def test_chain_with_identity_edge_is_two_marginal_sinkhorn():
    """Fixed-free-fixed chain whose second edge forbids moving mass (C = 0 on the
    diagonal, +inf elsewhere): B_23 is diagonal, mu_2 = mu_3, and B_12 solves
    entropic OT between mu_1 and mu_3 -- the plain two-marginal Sinkhorn problem."""
    rng = np.random.default_rng(11)
    n1, n = 6, 5
    mu1 = gen.dirichlet_marginal(n1, rng)
    mu3 = gen.dirichlet_marginal(n, rng)
    C12 = rng.random((n1, n)).astype(np.float32)
    C23 = np.full((n, n), np.inf, np.float32)
    np.fill_diagonal(C23, 0.0)
    eps = 0.15
    p = dense_problem([[0, 1], [1, 2]], [n1, n, n], [True, False, True], {0: mu1, 2: mu3}, [C12, C23], eps)
    f = converged(p)
    P = TB.sinkhorn(mu1, mu3, C12.astype(np.float64), eps)
    np.testing.assert_allclose(O.plan(p, f, 0, 1), P, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(O.plan(p, f, 1, 2), np.diag(mu3), rtol=1e-9, atol=1e-14)


def test_star_is_ibp_barycenter():
    """Star with fixed leaves and a free centre = entropic barycenter with uniform
    weights (the iterative Bregman projection problem the paper relates to)."""
    p = gen.star_problem(seed=2001, leaves=3, side=5, eps=0.05)
    f = converged(p, tol=1e-13)
    Cs = [O.cost(p, l, 0) for l in range(1, 4)]
    plans, bar = TB.ibp_barycenter([p.marginals[l] for l in range(1, 4)], Cs, p.eps)
    for l in range(1, 4):
        np.testing.assert_allclose(O.plan(p, f, l, 0), plans[l - 1], rtol=1e-8, atol=1e-14)
    fc = O.final_check(p, f)
    np.testing.assert_allclose(fc["marginals"][0], bar, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("seed,J", [(21, 3), (22, 4), (23, 5)])
def test_general_optimiser_finds_same_plans(seed, J):
    """The local-entropy primal (eq. ot_graph_pairwise_mass) solved by a generic convex method."""
    p = random_small_tree(seed, J, nmin=2, nmax=4, eps=0.3)
    f = converged(p, tol=1e-13)
    costs = [O.cost(p, int(a), int(b)) for a, b in p.edges]
    plans, val = TB.primal_generic(p.num_nodes, [tuple(map(int, e)) for e in p.edges], [int(x) for x in p.n],
                                   p.fixed, p.marginals, costs, p.eps)
    for e, (a, b) in enumerate(p.edges):
        np.testing.assert_allclose(O.plan(p, f, int(a), int(b)), plans[e], rtol=1e-9, atol=1e-13)
    fc = O.final_check(p, f)
    assert abs(fc["primal"] - val) < 1e-11


@pytest.mark.parametrize("seed,J", [(31, 4), (32, 6)])
def test_lp_limit_within_entropic_bound(seed, J):
    """OPT_LP <= TC(B_eps) <= OPT_LP + 2 eps |E| log d (lemma lem:round_applied with zero residual)."""
    p = random_small_tree(seed, J, nmin=3, nmax=4, eps=0.02)
    f = converged(p, tol=1e-12)
    costs = [O.cost(p, int(a), int(b)) for a, b in p.edges]
    opt = TB.lp_optimum(p.num_nodes, [tuple(map(int, e)) for e in p.edges], [int(x) for x in p.n],
                        p.fixed, p.marginals, costs)
    tc = O.final_check(p, f)["transport_cost"]
    d = int(p.n.max())
    assert opt - 1e-9 <= tc <= opt + 2 * p.eps * p.num_edges * math.log(d) + 1e-9


# ---------------------------------------------------------------------------
# invariants proved in Sec. 3.2
# ---------------------------------------------------------------------------

def _trajectory(p, T):
    colour = O.bipartition(p.num_nodes, p.edges)
    f = O.zero_potentials(p)
    traj = [f]
    for t in range(1, T + 1):
        f, _ = O.half_step(p, f, colour, 0 if t % 2 == 1 else 1)
        traj.append(f)
    return traj


@pytest.fixture(scope="module")
def tree_traj():
    p = random_small_tree(41, 7, nmin=3, nmax=6, eps=0.1)
    return p, _trajectory(p, 60)


def test_unit_mass_every_half_step(tree_traj):
    """Lemma cor:tree_mass: ||B_e||_1 = 1 after every update."""
    p, traj = tree_traj
    for f in traj[1:]:
        for a, b in p.edges:
            assert abs(O.plan(p, f, int(a), int(b)).sum() - 1.0) < 1e-12


def test_potential_oscillation_bound(tree_traj):
    """Lemma lem:tree_dual_varia_bounds: max lambda - min lambda <= 2 C_inf on every directed edge, every iterate."""
    p, traj = tree_traj
    cinf = O.c_infinity(p)
    for f in traj:
        for v in f.values():
            assert v.max() - v.min() <= 2 * cinf + 1e-12


def test_dual_decrease_and_gap_bounds(tree_traj):
    """Lemma lem:f_upper_bound_tree (f^t - f* <= 2C_inf/eps * r_t) and lemma lem:f_lower_bound_tree
    (f^t - f^{t+1} >= r_t^2/(22|E|))."""
    p, traj = tree_traj
    fstar = O.dual_objective(p, converged(p, tol=1e-13))
    cinf = O.c_infinity(p)
    E = p.num_edges
    # the bounds are stated for the iterates of the algorithm, i.e. after the first update
    for t in range(1, len(traj) - 1):
        ft = O.dual_objective(p, traj[t])
        ft1 = O.dual_objective(p, traj[t + 1])
        r = O.residual(p, traj[t])[0]
        assert ft - ft1 >= r * r / (22 * E) - 1e-12
        assert ft - fstar <= 2 * cinf / p.eps * r + 1e-12
        assert ft1 <= ft + 1e-13


def test_iteration_bound():
    """Theorem thm:num_iter: r <= delta' within 2 + 88 |E| C_inf / (delta' eps) half-steps."""
    p = random_small_tree(43, 6, eps=0.2)
    delta = 1e-3
    _, T, r = O.solve(p, tol=delta)
    assert r < delta
    assert T <= 2 + 88 * p.num_edges * O.c_infinity(p) / (delta * p.eps)


def test_primal_dual_gap_closes():
    p = random_small_tree(44, 6, eps=0.1)
    fc = O.final_check(p, converged(p, tol=1e-13))
    assert abs(fc["primal"] - fc["dual"]) < 1e-11 * max(1.0, abs(fc["primal"]))


# ---------------------------------------------------------------------------
# algorithmic equivalences
# ---------------------------------------------------------------------------

def test_listing_form_equals_closed_form():
    """Proposition cor:equi: the multiplicative updates of the listing equal thm:tree_dual_var from u = 1."""
    p = random_small_tree(51, 7, eps=0.3)
    colour = O.bipartition(p.num_nodes, p.edges)
    f = O.zero_potentials(p)
    u = {k: np.ones_like(v) for k, v in f.items()}
    for t in range(1, 25):
        side = 0 if t % 2 == 1 else 1
        f, _ = O.half_step(p, f, colour, side)
        u = O.multiplicative_half_step(p, u, colour, side)
        for key in f:
            np.testing.assert_allclose(p.eps * np.log(u[key]), f[key], rtol=0, atol=1e-12)


def test_any_schedule_reaches_the_same_plans():
    """Strict convexity: Gauss-Seidel updates in a random node order reach the same B."""
    p = random_small_tree(52, 7, eps=0.2)
    fa = converged(p, tol=1e-13)
    rng = np.random.default_rng(0)
    nb = O.neighbours(p.num_nodes, p.edges)
    f = O.zero_potentials(p)
    for sweep in range(5000):
        for j in rng.permutation(p.num_nodes):
            upd, _ = O.update_node(p, f, int(j), nb)
            f.update(upd)
        if O.residual(p, f)[0] < 1e-13:
            break
    for a, b in p.edges:
        np.testing.assert_allclose(O.plan(p, f, int(a), int(b)), O.plan(p, fa, int(a), int(b)), atol=1e-11)


def test_leaf_permutation_symmetry():
    """Relabelling the leaves of a star permutes the potentials and keeps the centre marginal."""
    p = gen.star_problem(seed=2002, leaves=4, side=4, eps=0.1)
    perm = [0, 3, 1, 4, 2]
    q = gen.star_problem(seed=2002, leaves=4, side=4, eps=0.1)
    q.marginals = {perm[l]: p.marginals[l] for l in range(1, 5)}
    fp = O.run_half_steps(p, 9)
    fq = O.run_half_steps(q, 9)
    for l in range(1, 5):
        np.testing.assert_allclose(fp[(l, 0)], fq[(perm[l], 0)], atol=1e-13)
        np.testing.assert_allclose(fp[(0, l)], fq[(0, perm[l])], atol=1e-13)


# ---------------------------------------------------------------------------
# input checks
# ---------------------------------------------------------------------------

def test_validation_errors():
    p = gen.chain_problem(n=4)
    O.validate(p)
    bad = gen.chain_problem(n=4)
    bad.edges = np.array([[0, 1], [1, 2], [2, 0], [3, 4]], np.int32)
    with pytest.raises(O.TreeError) as ei:
        O.validate(bad)
    assert ei.value.kind == "NOT_TREE"
    bad = gen.chain_problem(n=4)
    bad.fixed[2] = True
    bad.marginals[2] = np.full(4, 0.25)
    with pytest.raises(O.TreeError) as ei:
        O.validate(bad)
    assert ei.value.kind == "FIXED_NOT_LEAF"
    two = dense_problem([[0, 1]], [2, 2], [True, True], {0: np.array([.5, .5]), 1: np.array([.5, .5])},
                        [np.zeros((2, 2))], 1.0)
    with pytest.raises(O.TreeError) as ei:
        O.validate(two)
    assert ei.value.kind == "FIXED_ADJACENT"
    bad = gen.chain_problem(n=4)
    bad.marginals[0] = bad.marginals[0] * 2
    with pytest.raises(O.TreeError) as ei:
        O.validate(bad)
    assert ei.value.kind == "MARGINAL"
    bad = gen.chain_problem(n=4)
    bad.eps = 0.0
    with pytest.raises(O.TreeError) as ei:
        O.validate(bad)
    assert ei.value.kind == "EPS"


def test_bipartition_is_proper():
    rng = np.random.default_rng(3)
    for J in [2, 3, 10, 64]:
        edges = gen.uniform_pruefer_tree(J, rng)
        c = O.bipartition(J, edges)
        assert c[0] == 0
        assert all(c[a] != c[b] for a, b in edges)


def test_prufer_generator_leaf_count():
    rng = np.random.default_rng(5)
    edges = gen.pruefer_tree_with_leaves(64, 32, rng)
    assert gen.leaves_of(64, edges).sum() == 32
    assert len(set(map(tuple, np.sort(edges, axis=1).tolist()))) == 63


# ---------------------------------------------------------------------------
# the pins catch plausible mistakes (planted in the oracle, on the CPU)
# ---------------------------------------------------------------------------

def _pins_pass():
    """A quick subset of the pins above; True when all hold."""
    try:
        test_golden_single_edge_two_points()
        test_golden_stopping_quantity_away_from_convergence()
        test_chain_with_identity_edge_is_two_marginal_sinkhorn()
        test_star_is_ibp_barycenter()
        p = random_small_tree(41, 5, nmin=3, nmax=4, eps=0.1)
        traj = _trajectory(p, 12)
        for f in traj[1:]:
            for a, b in p.edges:
                assert abs(O.plan(p, f, int(a), int(b)).sum() - 1.0) < 1e-12
        test_general_optimiser_finds_same_plans(21, 3)
    except Exception:  # a shape error from a wrong operand counts as caught too
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    real_message = O.message
    real_log_gamma = O.log_gamma
    real_cost = O.cost

    mistakes = {
        "dropped log-gamma term": lambda: monkeypatch.setattr(
            O, "message", lambda p, f, j, k, rows=None: O.logsumexp(
                (f[(k, j)][None, :] - real_cost(p, j, k, rows)) / p.eps, axis=1)),
        "wrong sign of the cost": lambda: monkeypatch.setattr(
            O, "message", lambda p, f, j, k, rows=None: O.logsumexp(
                (f[(k, j)][None, :] + real_cost(p, j, k, rows)) / p.eps
                + real_log_gamma(p, k)[None, :], axis=1)),
        "reads own potential instead of the neighbour's": lambda: monkeypatch.setattr(
            O, "message", lambda p, f, j, k, rows=None: O.logsumexp(
                (np.resize(f[(j, k)], p.n[k])[None, :] - real_cost(p, j, k, rows)) / p.eps
                + real_log_gamma(p, k)[None, :], axis=1)),
        "gamma ignored in the plan": lambda: monkeypatch.setattr(
            O, "log_gamma", lambda p, j: np.zeros(int(p.n[j]))),
    }
    for name, plant in mistakes.items():
        monkeypatch.setattr(O, "message", real_message)
        monkeypatch.setattr(O, "log_gamma", real_log_gamma)
        plant()
        assert not _pins_pass(), name
    monkeypatch.setattr(O, "message", real_message)
    monkeypatch.setattr(O, "log_gamma", real_log_gamma)

    # transposed operand: C_(j,k) taken in the stored orientation even when j is the column node
    def untransposed_cost(p, j, k, rows=None):
        e, transposed = O.edge_index(p)[(j, k)]
        a, b = (k, j) if transposed else (j, k)
        C = real_cost(p, a, b)
        if C.shape[0] != int(p.n[j]):
            C = C.reshape(int(p.n[j]), -1) if C.size == int(p.n[j]) * int(p.n[k]) else C
        return C if rows is None else C[np.asarray(rows)]
    monkeypatch.setattr(O, "cost", untransposed_cost)
    assert not _pins_pass(), "transposed cost"
    monkeypatch.setattr(O, "cost", real_cost)

    # a wrong mean (sum instead of mean) in the free-node update
    real_update = O.update_node

    def bad_update(p, f, j, nb):
        upd, rho = real_update(p, f, j, nb)
        if p.fixed[j] or len(nb[j]) < 2:
            return upd, rho
        return {key: v * 1.5 for key, v in upd.items()}, rho
    monkeypatch.setattr(O, "update_node", bad_update)
    assert not _pins_pass(), "scaled free update"


def test_planted_stopping_rule_mistakes_are_caught(monkeypatch):
    """Plausible mistakes in the stopping quantity: the geometric mean (the update's eq. q) in
    place of the arithmetic qbar, the sum of the terms reported as the largest term, and the
    free-node terms measured against the first neighbour's q instead of the mean."""
    assert _pins_pass()
    real_residual = O.residual

    def planted(kind):
        def residual(p, f):
            nb = O.neighbours(p.num_nodes, p.edges)
            terms = {}
            for j in range(p.num_nodes):
                if p.fixed[j]:
                    (k,) = nb[j]
                    terms[(j, k)] = float(np.abs(O.edge_marginal(p, f, j, k) - p.marginals[j]).sum())
                    continue
                qs = {k: O.edge_marginal(p, f, j, k) for k in nb[j]}
                if kind == "geometric":
                    qbar = np.exp(sum(np.log(q) for q in qs.values()) / len(qs))
                elif kind == "first":
                    qbar = qs[nb[j][0]]
                else:
                    qbar = sum(qs.values()) / len(qs)
                for k in nb[j]:
                    terms[(j, k)] = float(np.abs(qs[k] - qbar).sum())
            r = float(sum(terms.values()))
            return r, (r if kind == "max_is_sum" else float(max(terms.values()))), terms
        return residual

    for kind in ["geometric", "max_is_sum", "first"]:
        monkeypatch.setattr(O, "residual", planted(kind))
        assert not _pins_pass(), kind
    monkeypatch.setattr(O, "residual", planted("none"))
    assert _pins_pass()
    monkeypatch.setattr(O, "residual", real_residual)
