"""GPU rounding (tree_ot_round, tree_ot_round_plan) against the oracle's rounding.

The rounding algorithm of Sec. 3.1 and lemmas lem:round / lem:round_applied
(Sec. 3.2).  Tolerances:
* costs and the stopping sum of the GPU's own input plans against the oracle's
  evaluation of the same potentials: 1e-7 relative (double-float plan entries,
  ~1e-7 relative each and uncorrelated, summed in FP64);
* rounded plans written out by the GPU: every constraint of the unregularised
  problem met to 1e-13 (FP64 sums of the same entries the rounding used);
* rounded plans against the oracle's rounding of the same potentials: 1e-6 in
  L1 per plan (entry accuracy, plus the GPU taking k's marginal as the column
  target where the paper keeps B^T 1: the two differ by the iterate's own
  stopping terms, ~1e-7 for FP32 iterates);
* FP64 handles: 1e-10 relative on costs, 1e-12 on plans.
"""
import math

import numpy as np
import pytest

import gen
from gen.problems import TreeProblem
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


def random_tree(seed, J, n_range, eps, D=2, kind="sqeuclid"):
    rng = np.random.default_rng(seed)
    p = gen.random_tree_problem(rng, J, n_range=n_range, eps_range=(eps, eps), D=D, name=f"rt{seed}")
    p.cost_kind = kind
    return p


def zeros_and_free_leaf():
    """A 12-leaf star with a free leaf, an n = 1 leaf and zeros in some marginals."""
    rng = np.random.default_rng(37)
    L = 12
    edges = np.array([[0, l] for l in range(1, L + 1)], np.int32)
    n = np.concatenate([[40], rng.integers(1, 60, size=L)]).astype(np.int32)
    n[3] = 1
    fixed = np.ones(L + 1, bool)
    fixed[0] = False
    fixed[5] = False
    coords = [rng.random((int(n[j]), 2)).astype(np.float32) for j in range(L + 1)]
    marg = {}
    for j in range(1, L + 1):
        if fixed[j]:
            m = gen.dirichlet_marginal(int(n[j]), rng)
            if n[j] > 3:
                m[1] = 0.0
                m /= m.sum()
            marg[j] = m
    return TreeProblem(name="zeros", edges=edges, n=n, fixed=fixed, marginals=marg, eps=0.05, coords=coords,
                       cost_scale=1.0, cost_kind="sqeuclid")


CASES = {
    "chain_dense_n70": lambda: gen.chain_problem(seed=1001, n=70, eps=0.01),
    "tree9_unequal_3d": lambda: random_tree(11, 9, (37, 300), 0.02, D=3),
    "tree7_unequal_dense": lambda: random_tree(12, 7, (5, 400), 0.03, kind="dense"),
    "star5_grid12": lambda: gen.star_problem(seed=2003, leaves=5, side=12, eps=0.01),
    "star12_zeros_free_leaf": zeros_and_free_leaf,
}


def node_marginals_of(p, plans):
    """Marginals of every node from a set of plans keyed by edge index (rows on edges[e][0])."""
    out = {j: [] for j in range(p.num_nodes)}
    for e, (a, b) in enumerate(np.asarray(p.edges)):
        out[int(a)].append(plans[e].sum(axis=1))
        out[int(b)].append(plans[e].sum(axis=0))
    return out


def feasibility_gap(p, plans):
    """Largest L1 violation of the unregularised constraints: fixed nodes carry mu (at unit
    mass), a free node's plans share one marginal; every plan has mass 1."""
    worst = 0.0
    for j, qs in node_marginals_of(p, plans).items():
        ref = p.marginals[j] / p.marginals[j].sum() if p.fixed[j] else qs[0]
        for q in qs:
            worst = max(worst, float(np.abs(q - ref).sum()), abs(float(q.sum()) - 1.0))
    return worst


def oracle_by_edge(p, R):
    """The oracle's rounded plans keyed by edge index, rows on edges[e][0]."""
    out = {}
    for e, (a, b) in enumerate(np.asarray(p.edges)):
        a, b = int(a), int(b)
        out[e] = R[(a, b)] if (a, b) in R else R[(b, a)].T
    return out


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_round_parity_fp32(T, name, steps):
    p = CASES[name]()
    with T.Solver([p], T.options(precision="fp32")) as s:
        s.half_steps(steps)
        res = s.round()[0]
        got = s.potentials(0)
        plans = {e: s.round_plan(0, e).cpu().numpy() for e in range(p.num_edges)}
    side = O.mismatched_side(steps)
    assert res["side"] == side and res["half_steps"] == steps
    fc = O.final_check(p, got)
    R = oracle_by_edge(p, O.round_plans(p, got, side))
    tr = O.rounded_transport_cost(p, O.round_plans(p, got, side))
    # the side updated last matches its marginals only to the FP32 iterate's accuracy: its
    # stopping terms bound how far k's marginal (the GPU's column target) is from B^T 1 (the paper's)
    colour = O.bipartition(p.num_nodes, p.edges)
    r_k = sum(v for (j, _), v in fc["terms"].items() if colour[j] != side)
    cinf = O.c_infinity(p)
    assert abs(res["transport_cost"] - fc["transport_cost"]) <= 1e-7 * abs(fc["transport_cost"])
    assert abs(res["rounded_transport_cost"] - tr) <= 1e-7 * abs(tr) + 2 * cinf * r_k
    assert abs(res["residual_sum_l1"] - fc["residual"]) <= 1e-7 * max(1.0, fc["residual"])
    assert abs(res["c_inf"] - O.c_infinity(p)) <= 1e-6 * O.c_infinity(p)
    # the GPU's rounded plans: exactly feasible, and the oracle's rounding to the entries' accuracy
    assert feasibility_gap(p, plans) <= 1e-13
    for e in range(p.num_edges):
        assert np.all(plans[e] >= 0.0)
        assert float(np.abs(plans[e] - R[e]).sum()) <= 1e-6 + 4 * r_k, e
    # lemma lem:round on the GPU's numbers: the cost moves by at most 2 C_inf r
    assert abs(res["rounded_transport_cost"] - res["transport_cost"]) <= 2 * res["c_inf"] * res["residual_sum_l1"] + 1e-12


def test_round_parity_fp64_chain(T):
    p = gen.chain_problem(seed=1003, n=64, eps=0.01)
    with T.Solver([p], T.options(precision="fp64")) as s:
        s.half_steps(5)
        res = s.round()[0]
        got = s.potentials(0)
        plans = {e: s.round_plan(0, e).cpu().numpy() for e in range(p.num_edges)}
    R = O.round_plans(p, got, O.mismatched_side(5))
    tr = O.rounded_transport_cost(p, R)
    assert abs(res["rounded_transport_cost"] - tr) <= 1e-10 * abs(tr)
    assert feasibility_gap(p, plans) <= 1e-13
    Re = oracle_by_edge(p, R)
    for e in range(p.num_edges):
        assert float(np.abs(plans[e] - Re[e]).sum()) <= 1e-12, e


@pytest.mark.parametrize("seed,J", [(71, 4), (72, 5), (73, 6)])
def test_round_against_lp_optimum(T, seed, J):
    """Lemma lem:round_applied on tiny trees: OPT <= TC(B^) <= OPT + 2 eps |E| log d + 4 C_inf r,
    OPT from an LP solver; the lower bound holds because the rounded plans are feasible."""
    import textbook_ot as TB
    from test_oracle_pins import random_small_tree
    p = random_small_tree(seed, J, nmin=3, nmax=4, eps=0.05)
    costs = [O.cost(p, int(a), int(b)) for a, b in p.edges]
    opt = TB.lp_optimum(p.num_nodes, [tuple(map(int, e)) for e in p.edges], [int(x) for x in p.n],
                        p.fixed, p.marginals, costs)
    d = int(p.n.max())
    with T.Solver([p], T.options(precision="fp32")) as s:
        for steps in (1, 2, 5, 20):
            s.reset()
            s.half_steps(steps)
            res = s.round()[0]
            assert res["bound"] == pytest.approx(2 * p.eps * p.num_edges * math.log(d)
                                                 + 4 * res["c_inf"] * res["residual_sum_l1"], rel=1e-12)
            assert opt - 1e-7 <= res["rounded_transport_cost"] <= opt + res["bound"] + 1e-7, steps


def test_round_after_batched_solve(T):
    """A forest solved to 1e-6: each retired tree is rounded on the colour its last half-step
    missed, and the rounding moves the cost by at most 2 C_inf r (r <= a few 1e-6)."""
    rng = np.random.default_rng(4002)
    probs = [gen.random_tree_problem(rng, int(rng.integers(4, 9)), n_range=(64, 300), eps_range=(0.01, 0.05),
                                     name=f"f{i}") for i in range(6)]
    with T.Solver(probs, T.options(precision="fp32", tol=1e-6, tol_kind="max")) as s:
        rc, sol = s.solve()
        assert rc == 0
        res = s.round()
        for i in (0, 3, 5):
            got = s.potentials(i)
            side = O.mismatched_side(sol[i]["half_steps"])
            assert res[i]["side"] == side and res[i]["half_steps"] == sol[i]["half_steps"]
            tr = O.rounded_transport_cost(probs[i], O.round_plans(probs[i], got, side))
            fc = O.final_check(probs[i], got)
            colour = O.bipartition(probs[i].num_nodes, probs[i].edges)
            r_k = sum(v for (j, _), v in fc["terms"].items() if colour[j] != side)
            assert abs(res[i]["rounded_transport_cost"] - tr) <= 1e-7 * abs(tr) + 2 * res[i]["c_inf"] * r_k
    for r in res:
        assert abs(r["rounded_transport_cost"] - r["transport_cost"]) <= 2 * r["c_inf"] * r["residual_sum_l1"] + 1e-12


def test_round_state_errors(T):
    p = gen.chain_problem(seed=1001, n=20, eps=0.05)
    with T.Solver([p], T.options(precision="fp32")) as s:
        with pytest.raises(T.TreeOTError) as ei:
            s.round()                      # no half-step yet: no colour class is matched
        assert ei.value.kind == "STATE"
        s.half_steps(3)
        s.round()
        s.round_plan(0, 1)
        s.half_steps(1)
        with pytest.raises(T.TreeOTError) as ei:
            s.round_plan(0, 1)             # potentials changed since the rounding
        assert ei.value.kind == "STATE"
