"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (from the accuracy targets of this solver):
* iterate parity after T half-steps from u = 1: potentials within 1e-4 relative
  (max |df| <= 1e-4 max(|f_ref|_inf, eps)) and, stricter, the FP64 marginals of
  the GPU iterate within 1e-6 (L1) of the oracle iterate's;
* converged parity: max marginal L1 violation <= 1e-6 (FP32 path) checked by the
  oracle in FP64 on the GPU's potentials, relative objective error <= 1e-6,
  gauge-fixed potentials within 1e-4 relative;
* FP64 path: 1e-9 stopping sum, potentials within 1e-9 relative.
"""
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


def rel_err(got, ref, eps):
    """max over directed edges of max|got - ref| / max(|ref|_inf, eps); inf if got is not finite."""
    worst = 0.0
    for key in ref:
        if not np.all(np.isfinite(got[key])):
            return float("inf")
        scale = max(float(np.max(np.abs(ref[key]))), eps)
        worst = max(worst, float(np.max(np.abs(got[key] - ref[key]))) / scale)
    return worst


def marginal_gap(p, f_got, f_ref):
    """max over directed edges of || B 1 (got) - B 1 (ref) ||_1 in FP64."""
    worst = 0.0
    for a, b in np.asarray(p.edges):
        for j, k in ((int(a), int(b)), (int(b), int(a))):
            gap = float(np.abs(O.edge_marginal(p, f_got, j, k) - O.edge_marginal(p, f_ref, j, k)).sum())
            if not np.isfinite(gap):
                return float("inf")
            worst = max(worst, gap)
    return worst


def random_tree(seed, J, n_range, eps, D=2, kind="sqeuclid"):
    rng = np.random.default_rng(seed)
    p = gen.random_tree_problem(rng, J, n_range=n_range, eps_range=(eps, eps), D=D, name=f"rt{seed}")
    p.cost_kind = kind
    return p


ITERATE_CASES = {
    "chain_dense_n70": lambda: gen.chain_problem(seed=1001, n=70, eps=0.01),
    "prufer12_dense_n1100": lambda: gen.prufer_problem(seed=3001, J=12, n=1100, num_leaves=6, eps=0.01),
    "star5_grid20_sqeuclid": lambda: gen.star_problem(seed=2003, leaves=5, side=20, eps=0.005),
    "tree9_unequal_3d": lambda: random_tree(11, 9, (37, 1300), 0.02, D=3),
    "tree7_unequal_2d_dense": lambda: random_tree(12, 7, (5, 700), 0.03, D=2, kind="dense"),
    "chain_1d_sqeuclid_n300": lambda: gen.chain_problem(seed=1002, n=300, eps=0.004, cost_kind="sqeuclid"),
}


@pytest.mark.parametrize("name", sorted(ITERATE_CASES))
@pytest.mark.parametrize("steps", [1, 2, 9])
def test_iterate_parity_fp32(T, name, steps):
    p = ITERATE_CASES[name]()
    ref = O.run_half_steps(p, steps)
    with T.Solver([p], T.options(precision="fp32")) as s:
        s.half_steps(steps)
        got = s.potentials(0)
    assert rel_err(got, ref, p.eps) <= 1e-4
    assert marginal_gap(p, got, ref) <= 1e-6


@pytest.mark.parametrize("name", ["star5_grid20_sqeuclid", "tree9_unequal_3d", "chain_1d_sqeuclid_n300"])
@pytest.mark.parametrize("steps", [1, 9])
def test_iterate_parity_exact_distances(T, name, steps):
    """Recomputed costs with exactly formed squared distances (split coordinates)."""
    p = ITERATE_CASES[name]()
    ref = O.run_half_steps(p, steps)
    with T.Solver([p], T.options(precision="fp32", exact_dist=True)) as s:
        s.half_steps(steps)
        got = s.potentials(0)
    assert rel_err(got, ref, p.eps) <= 1e-4
    assert marginal_gap(p, got, ref) <= 1e-6


def test_exact_distances_lower_the_floor(T):
    """16x16 stars at eps = 0.005: with exact squared distances every star is
    certified at 2e-7 (max marginal L1) by the FP64-grade check."""
    probs = gen.warmstart_stars(9_100_000, 16, side=16, eps=0.005)
    with T.Solver(probs, T.options(tol=2e-7, tol_kind="max", max_half_steps=20000, exact_dist=True)) as s:
        rc, res = s.solve()
        fs = [s.potentials(i) for i in (0, 7)]
    assert rc == 0, [r["max_marginal_l1"] for r in res]
    for i, f in zip((0, 7), fs):
        assert O.final_check(probs[i], f)["max_marginal_l1"] <= 2.5e-7


@pytest.mark.parametrize("steps", [1, 2, 9])
def test_iterate_parity_fp64(T, steps):
    p = gen.chain_problem(seed=1003, n=64, eps=0.01)
    ref = O.run_half_steps(p, steps)
    with T.Solver([p], T.options(precision="fp64")) as s:
        s.half_steps(steps)
        got = s.potentials(0)
    assert rel_err(got, ref, p.eps) <= 1e-11


def test_chain_fp64_to_1e9(T):
    """Chain of 5 nodes, n=64 grid, eps=0.01, FP64, stop at stopping sum < 1e-9."""
    p = gen.chain_problem(seed=1000)
    with T.Solver([p], T.options(precision="fp64", tol=1e-9, tol_kind="sum", check_every=2)) as s:
        rc, res = s.solve()
        got = s.potentials(0)
    assert rc == 0
    fc = O.final_check(p, got)
    assert fc["residual"] < 1e-9 and res[0]["residual_sum_l1"] < 1e-9
    fo, _, _ = O.solve(p, tol=1e-12)
    ref = O.final_check(p, fo)
    assert abs(res[0]["primal"] - ref["primal"]) <= 1e-9 * abs(ref["primal"])
    assert abs(res[0]["transport_cost"] - ref["transport_cost"]) <= 1e-8 * abs(ref["transport_cost"])
    assert rel_err(O.gauge_fix(p, got), O.gauge_fix(p, fo), p.eps) <= 1e-7


CONVERGED_CASES = {
    "star6_grid16": lambda: gen.star_problem(seed=2004, leaves=6, side=16, eps=0.01),
    "prufer10_dense_n300": lambda: gen.prufer_problem(seed=3002, J=10, n=300, num_leaves=5, eps=0.02),
    "tree8_unequal_2d": lambda: random_tree(13, 8, (60, 400), 0.03),
}


@pytest.mark.parametrize("name", sorted(CONVERGED_CASES))
def test_converged_parity_fp32(T, name):
    p = CONVERGED_CASES[name]()
    with T.Solver([p], T.options(precision="fp32", tol=5e-7, tol_kind="max", max_half_steps=60000)) as s:
        rc, res = s.solve()
        got = s.potentials(0)
        marg_gpu = {j: s.marginal(0, j) for j in range(p.num_nodes)}
    assert rc == 0, res
    fc = O.final_check(p, got)
    # the FP64 oracle confirms the GPU solution's feasibility
    assert fc["max_marginal_l1"] <= 1e-6, fc["max_marginal_l1"]
    # the GPU's own check agrees with the oracle's evaluation of the same potentials
    assert abs(res[0]["max_marginal_l1"] - fc["max_marginal_l1"]) <= 1e-7
    for j in range(p.num_nodes):
        # the double-float check is accurate to a few 1e-8 in L1, far inside the 1e-6 it certifies
        assert np.abs(marg_gpu[j] - fc["marginals"][j]).sum() <= 5e-8
    assert abs(res[0]["transport_cost"] - fc["transport_cost"]) <= 1e-8 * abs(fc["transport_cost"])
    fo, _, _ = O.solve(p, tol=1e-11, tol_kind="max")
    ref = O.final_check(p, fo)
    assert abs(res[0]["primal"] - ref["primal"]) <= 1e-6 * abs(ref["primal"])
    assert abs(res[0]["transport_cost"] - ref["transport_cost"]) <= 1e-6 * abs(ref["transport_cost"])
    assert rel_err(O.gauge_fix(p, got), O.gauge_fix(p, fo), p.eps) <= 1e-4


def test_full_star_barycenter(T):
    """8 fixed leaves on a 32x32 grid, free centre, eps=0.005, cost recomputed in-kernel."""
    p = gen.star_problem(seed=2000)
    with T.Solver([p], T.options(precision="fp32", tol=5e-7, tol_kind="max", max_half_steps=100000)) as s:
        rc, res = s.solve()
        got = s.potentials(0)
    assert rc == 0, res
    fc = O.final_check(p, got)
    assert fc["max_marginal_l1"] <= 1e-6, fc["max_marginal_l1"]
    assert abs(res[0]["max_marginal_l1"] - fc["max_marginal_l1"]) <= 1e-7
    # duality certificate of the objective: both P and D bracket the optimum
    assert abs(fc["primal"] - fc["dual"]) <= 1e-6 * abs(fc["primal"])
    assert abs(res[0]["primal"] - fc["primal"]) <= 1e-7 * abs(fc["primal"])


def test_full_prufer_dense_sampled(T):
    """64-node Pruefer tree, n=4096 in [0,1]^3, dense FP32 costs on the device (4.2 GB):
    one half-step of the GPU checked node by node against the oracle."""
    p = gen.prufer_problem(seed=3000)
    dev = torch.device("cuda")
    costs = [gen.sqeuclid_cost_f32_torch(p.coords[a], p.coords[b], 1.0, dev) for a, b in p.edges]
    # the device-built costs are the same FP32 values the oracle reads
    for e in (0, 31, 62):
        rows = [0, 1, 4095]
        np.testing.assert_array_equal(costs[e][rows].cpu().numpy(),
                                      gen.sqeuclid_cost_f32(p.coords[p.edges[e][0]], p.coords[p.edges[e][1]], 1.0,
                                                            rows=rows))
    colour = O.bipartition(p.num_nodes, p.edges)
    with T.Solver([p], T.options(precision="fp32"), device_costs=[costs]) as s:
        s.half_steps(4)
        f4 = s.potentials(0)
        s.half_steps(1)   # half-step 5 updates colour 0
        f5 = s.potentials(0)
    nb = O.neighbours(p.num_nodes, p.edges)
    fixed_nodes = [j for j in range(p.num_nodes) if colour[j] == 0 and p.fixed[j]]
    free_nodes = sorted([j for j in range(p.num_nodes) if colour[j] == 0 and not p.fixed[j]],
                        key=lambda j: len(nb[j]))
    sample = fixed_nodes[:1] + free_nodes[:1] + free_nodes[-1:]
    assert sample
    for j in sample:
        upd, _ = O.update_node(p, f4, j, nb)
        for key, ref in upd.items():
            got = f5[key]
            scale = max(float(np.max(np.abs(ref))), p.eps)
            assert float(np.max(np.abs(got - ref))) <= 1e-4 * scale, (j, key)
    del costs
    torch.cuda.empty_cache()


def test_full_prufer_bf16_solve_certified_by_oracle(T):
    """The 64-node tree at full size (n = 4096, 4.2 GB of stored costs): the BF16
    absorbed phase + FP32 refinement solved to max marginal L1 <= 1e-6 (the timed
    time-to-1e-6 form), then every directed edge's marginal of the returned
    potentials evaluated by the FP64 oracle: the largest stopping term is within
    1e-6 and equals the GPU check's."""
    p = gen.prufer_problem(seed=3000)
    dev = torch.device("cuda")
    costs = [gen.sqeuclid_cost_f32_torch(p.coords[a], p.coords[b], 1.0, dev) for a, b in p.edges]
    with T.Solver([p], T.options(precision="fp32", apply_mode="bf16", tol=1e-6, tol_kind="max",
                                 max_half_steps=20000), device_costs=[costs]) as s:
        rc, res = s.solve()
        got = s.potentials(0)
    del costs
    torch.cuda.empty_cache()
    assert rc == 0, res
    assert res[0]["lowp_half_steps"] > 0
    r, m, _ = O.residual(p, got)
    assert m <= 1e-6, m
    assert abs(res[0]["max_marginal_l1"] - m) <= 5e-8, (res[0]["max_marginal_l1"], m)
    assert abs(res[0]["residual_sum_l1"] - r) <= 1e-7 * max(1.0, r), (res[0]["residual_sum_l1"], r)


def test_batched_forest(T):
    """A forest of uneven trees solved in one handle: iterate parity per tree, then
    each tree converges and retires on its own."""
    rng = np.random.default_rng(4001)
    probs = []
    for i in range(10):
        J = int(rng.integers(4, 11))
        probs.append(gen.random_tree_problem(rng, J, n_range=(128, 520), eps_range=(0.01, 0.05),
                                             name=f"f{i}"))
    with T.Solver(probs, T.options(precision="fp32", tol=5e-7, tol_kind="max", max_half_steps=40000)) as s:
        s.half_steps(5)
        for i in (0, 4, 9):
            ref = O.run_half_steps(probs[i], 5)
            assert rel_err(s.potentials(i), ref, probs[i].eps) <= 1e-4
        s.reset()
        rc, res = s.solve()
        assert rc == 0
        steps = [r["half_steps"] for r in res]
        assert len(set(steps)) > 1          # trees retired at different half-steps
        for i in (1, 5, 8):
            fc = O.final_check(probs[i], s.potentials(i))
            assert fc["max_marginal_l1"] <= 1e-6
            assert abs(res[i]["max_marginal_l1"] - fc["max_marginal_l1"]) <= 1e-7


def test_full_batched_512_sampled(T):
    """The 512-tree batch (4..32 nodes, n in 128..2048, eps log-uniform): two
    half-steps on the GPU; the largest tree, the tree holding the largest
    support, the tree with the smallest eps and a median tree re-run by the
    oracle (the kernels' multi-split reductions and 2048-point tasks)."""
    probs = gen.batched_problems(seed=4000)
    sizes = np.array([pp.elements_per_half_step() for pp in probs])
    pick = {int(np.argmax(sizes)), int(np.argmax([int(np.max(pp.n)) for pp in probs])),
            int(np.argmin([pp.eps for pp in probs])), int(np.argsort(sizes)[len(probs) // 2])}
    with T.Solver(probs, T.options(precision="fp32")) as s:
        s.half_steps(2)
        for i in sorted(pick):
            ref = O.run_half_steps(probs[i], 2)
            got = s.potentials(i)
            assert rel_err(got, ref, probs[i].eps) <= 1e-4, i
            assert marginal_gap(probs[i], got, ref) <= 1e-6, i


def _geometric_mean_residual(p, f):
    """The stopping sum with the update's geometric mean in place of the arithmetic qbar
    (a plausible mistake; used only to show the comparison below can tell them apart)."""
    nb = O.neighbours(p.num_nodes, p.edges)
    tot = 0.0
    for j in range(p.num_nodes):
        if p.fixed[j]:
            (k,) = nb[j]
            tot += float(np.abs(O.edge_marginal(p, f, j, k) - p.marginals[j]).sum())
            continue
        qs = [O.edge_marginal(p, f, j, k) for k in nb[j]]
        g = np.exp(sum(np.log(q) for q in qs) / len(qs))
        tot += sum(float(np.abs(q - g).sum()) for q in qs)
    return tot


def test_stopping_quantity_away_from_convergence(T):
    """The stopping sum and its largest term (the while-condition of the Bipartite Iterative
    Scaling algorithm) at non-converged iterates of a 12-node tree with free nodes of degree
    3 and 4.  (a) The FP32 quantity the half-step kernels accumulate -- the one problems
    retire on -- for iterates 1..4 against the oracle's on the oracle's iterates; (b) the
    FP64-grade check of iterate 5 against the oracle's evaluation of the same potentials."""
    rng = np.random.default_rng(11)
    p = gen.random_tree_problem(rng, 12, n_range=(40, 300), eps_range=(0.03, 0.03), D=2, name="stop")
    with T.Solver([p], T.options(precision="fp32")) as s:
        s.half_steps(5)
        sums, maxs = s.residual_history(0, 1, 4)
        res = s.check()[0]
        got = s.potentials(0)
    tol_fp32 = 1e-5   # FP32 q (~1e-7 relative per entry) summed over 22 directed edges, plus the iterates' gap
    discriminating = 0
    for i, t in enumerate(range(1, 5)):
        f_ref = O.run_half_steps(p, t)
        r, m, _ = O.residual(p, f_ref)
        assert abs(sums[i] - r) <= tol_fp32, (t, sums[i], r)
        assert abs(maxs[i] - m) <= tol_fp32, (t, maxs[i], m)
        if abs(_geometric_mean_residual(p, f_ref) - r) > 10 * tol_fp32:
            discriminating += 1
    assert discriminating >= 2   # a geometric-mean stopping sum would fail (a)
    r, m, _ = O.residual(p, got)
    # double-float check: each marginal within a few 1e-8 (L1) of the FP64 evaluation
    assert abs(res["residual_sum_l1"] - r) <= 1e-7, (res["residual_sum_l1"], r)
    assert abs(res["max_marginal_l1"] - m) <= 5e-8, (res["max_marginal_l1"], m)


def test_iteration_cap_reports_not_converged(T):
    """A cap far below what tol needs: TREE_OT_NOT_CONVERGED, every result finite, the
    reported stopping sum above tol and equal to the oracle's on the returned potentials."""
    p = gen.star_problem(seed=2005, leaves=4, side=12, eps=0.01)
    with T.Solver([p], T.options(precision="fp32", tol=1e-9, tol_kind="sum", max_half_steps=10,
                                 check_every=2)) as s:
        rc, res = s.solve()
        got = s.potentials(0)
    assert rc == T.NOT_CONVERGED and res[0]["status"] == T.NOT_CONVERGED
    for k in ("residual_sum_l1", "max_marginal_l1", "primal", "dual", "transport_cost"):
        assert np.isfinite(res[0][k]), k
    assert res[0]["half_steps"] == 10
    r, _, _ = O.residual(p, got)
    assert res[0]["residual_sum_l1"] > 1e-9 and abs(res[0]["residual_sum_l1"] - r) <= 1e-7


def test_infeasible_row_reports_nonfinite(T):
    """A fixed leaf point with mu > 0 whose cost row is all +inf has no admissible plan
    (K = 0 on its whole row): the solve stops with TREE_OT_ERR_NONFINITE (the node
    update's non-finite flag, read between chunks; no device fault), and a new handle
    on the same device then solves normally."""
    rng = np.random.default_rng(29)
    n = 24
    mu0 = gen.dirichlet_marginal(n, rng)
    mu2 = gen.dirichlet_marginal(n, rng)
    C01 = rng.random((n, n)).astype(np.float32)
    C01[5, :] = np.inf
    C12 = rng.random((n, n)).astype(np.float32)
    mk = lambda c: TreeProblem(name="inf", edges=np.array([[0, 1], [1, 2]], np.int32), n=np.full(3, n, np.int32),
                               fixed=np.array([True, False, True]), marginals={0: mu0, 2: mu2}, eps=0.1,
                               coords=[np.zeros((n, 1), np.float32)] * 3, cost_scale=1.0, cost_kind="dense",
                               dense_costs=[c, C12])
    assert mu0[5] > 0
    with T.Solver([mk(C01)], T.options(precision="fp32", tol=1e-7, check_every=2)) as s:
        with pytest.raises(T.TreeOTError) as ei:
            s.solve()
    assert ei.value.kind == "NONFINITE"
    C01[5, :] = 0.5
    with T.Solver([mk(C01)], T.options(precision="fp32", tol=1e-7, tol_kind="max")) as s:
        rc, res = s.solve()
    assert rc == 0 and res[0]["max_marginal_l1"] <= 1e-7


def test_identity_edge_chain_is_sinkhorn_on_gpu(T):
    """Dense costs with +inf entries: the fixed-free-fixed chain with an identity
    edge solves two-marginal entropic OT (checked against the textbook solver)."""
    import textbook_ot as TB
    rng = np.random.default_rng(17)
    n = 37
    mu1 = gen.dirichlet_marginal(n, rng)
    mu3 = gen.dirichlet_marginal(n, rng)
    C12 = rng.random((n, n)).astype(np.float32)
    C23 = np.full((n, n), np.inf, np.float32)
    np.fill_diagonal(C23, 0.0)
    p = TreeProblem(name="ident", edges=np.array([[0, 1], [1, 2]], np.int32), n=np.full(3, n, np.int32),
                    fixed=np.array([True, False, True]), marginals={0: mu1, 2: mu3}, eps=0.1,
                    coords=[np.zeros((n, 1), np.float32)] * 3, cost_scale=1.0, cost_kind="dense",
                    dense_costs=[C12, C23])
    with T.Solver([p], T.options(precision="fp32", tol=1e-7, tol_kind="max")) as s:
        rc, res = s.solve()
        f = s.potentials(0)
    assert rc == 0
    P = TB.sinkhorn(mu1, mu3, C12.astype(np.float64), 0.1)
    assert np.abs(O.plan(p, f, 0, 1) - P).sum() <= 2e-6


def test_edge_cases_small_supports_and_free_leaf(T):
    """n = 1 nodes, a free leaf, marginal zeros and a 40-leaf star (degree > 8)."""
    rng = np.random.default_rng(23)
    # star with 40 leaves, one free leaf, unequal supports including n=1
    L = 40
    edges = np.array([[0, l] for l in range(1, L + 1)], np.int32)
    n = np.concatenate([[33], rng.integers(1, 40, size=L)]).astype(np.int32)
    n[5] = 1
    fixed = np.ones(L + 1, bool)
    fixed[0] = False
    fixed[7] = False  # free leaf
    coords = [rng.random((int(n[j]), 2)).astype(np.float32) for j in range(L + 1)]
    marg = {}
    for j in range(1, L + 1):
        if fixed[j]:
            m = gen.dirichlet_marginal(int(n[j]), rng)
            if n[j] > 3:
                m[1] = 0.0
                m /= m.sum()
            marg[j] = m
    p = TreeProblem(name="edge", edges=edges, n=n, fixed=fixed, marginals=marg, eps=0.05, coords=coords,
                    cost_scale=1.0, cost_kind="sqeuclid")
    ref = O.run_half_steps(p, 7)
    with T.Solver([p], T.options(precision="fp32", tol=5e-7, tol_kind="max")) as s:
        s.half_steps(7)
        assert rel_err(s.potentials(0), ref, p.eps) <= 1e-4
        s.reset()
        rc, res = s.solve()
        got = s.potentials(0)
    assert rc == 0
    assert O.final_check(p, got)["max_marginal_l1"] <= 1e-6


def high_degree_star(L, seed=29, eps=0.05):
    """Star with L leaves (free centre) and small unequal supports."""
    rng = np.random.default_rng(seed)
    edges = np.array([[0, l] for l in range(1, L + 1)], np.int32)
    n = np.concatenate([[37], rng.integers(1, 9, size=L)]).astype(np.int32)
    fixed = np.ones(L + 1, bool)
    fixed[0] = False
    coords = [rng.random((int(n[j]), 2)).astype(np.float32) for j in range(L + 1)]
    marg = {j: gen.dirichlet_marginal(int(n[j]), rng) for j in range(1, L + 1)}
    return TreeProblem(name=f"star{L}", edges=edges, n=n, fixed=fixed, marginals=marg, eps=eps, coords=coords,
                       cost_scale=1.0, cost_kind="sqeuclid")


@pytest.mark.parametrize("precision,tol,mtol", [("fp32", 1e-4, 1e-5), ("fp64", 1e-11, 1e-9)])
def test_high_degree_node_update(T, precision, tol, mtol):
    """A 400-leaf star: the centre's chunks hold two points and 400 edges, so the
    node update's warps mix edges (per-lane stopping-term sums)."""
    p = high_degree_star(400)
    ref = O.run_half_steps(p, 5)
    with T.Solver([p], T.options(precision=precision)) as s:
        s.half_steps(5)
        got = s.potentials(0)
        res = s.check()
    assert rel_err(got, ref, p.eps) <= tol
    ref_res = O.final_check(p, ref)
    assert marginal_gap(p, got, ref) <= mtol
    assert abs(res[0]["max_marginal_l1"] - ref_res["max_marginal_l1"]) <= mtol


def test_degree_limit_is_reported(T):
    """A node of degree 2700 does not fit the node update's shared memory."""
    with pytest.raises(T.TreeOTError) as ei:
        T.Solver([high_degree_star(2700)], T.options())
    assert ei.value.kind == "ARG"


def test_nan_cost_is_rejected(T):
    p = gen.chain_problem(seed=1004, n=16)
    p.dense_cost(0)
    p.dense_costs[0] = p.dense_costs[0].copy()
    p.dense_costs[0][3, 4] = np.nan
    with pytest.raises(T.TreeOTError) as ei:
        T.Solver([p], T.options())
    assert ei.value.kind == "NONFINITE"


def test_split_launches_equal_half_steps(T):
    """tree_ot_apply + tree_ot_node_update equal one tree_ot_half_steps call (bitwise)."""
    p = gen.prufer_problem(seed=3003, J=8, n=600, num_leaves=4)
    with T.Solver([p], T.options()) as a, T.Solver([p], T.options()) as b:
        a.half_steps(3)
        for c in (0, 1, 0):
            b.apply(c)
            b.node_update(c)
        fa, fb = a.potentials(0), b.potentials(0)
    for key in fa:
        np.testing.assert_array_equal(fa[key], fb[key])


def test_graph_and_direct_launches_agree(T):
    p = gen.star_problem(seed=2005, leaves=4, side=12, eps=0.02)
    out = []
    for g in (True, False):
        with T.Solver([p], T.options(tol=1e-7, tol_kind="max", use_graph=g, check_every=8)) as s:
            rc, res = s.solve()
            out.append((res[0]["half_steps"], s.potentials(0)))
    assert out[0][0] == out[1][0]
    for key in out[0][1]:
        np.testing.assert_array_equal(out[0][1][key], out[1][1][key])


def test_warm_start_from_converged_potentials(T):
    """A checkpoint (converged potentials) resumes and stops within one check period."""
    p = gen.star_problem(seed=2006, leaves=3, side=10, eps=0.02)
    fo, _, _ = O.solve(p, tol=1e-12)
    with T.Solver([p], T.options(tol=1e-6, tol_kind="max", check_every=4)) as s:
        s.set_potentials(fo)
        rc, res = s.solve()
        assert rc == 0 and res[0]["half_steps"] <= 4
        assert O.final_check(p, s.potentials(0))["max_marginal_l1"] <= 1e-6


# ---------------------------------------------------------------------------
# absorbed BF16 phase + FP32 refinement (stored costs)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("transpose", [True, False])
def test_bf16_phase_then_fp32_refinement_reaches_tolerance(T, transpose):
    """BF16 absorbed kernel until the stopping quantity is below refine_tol, then
    the FP32 kernel: the result meets the FP32 parity bar (column node's apply on
    the transposed kernel, or down the columns)."""
    p = gen.prufer_problem(seed=3004, J=12, n=700, num_leaves=6, eps=0.01)
    opts = T.options(precision="fp32", tol=2e-7, tol_kind="max", apply_mode="bf16", refine_tol=1e-3,
                     absorb_tau=24, lowp_start=4, max_half_steps=40000, transpose=transpose)
    with T.Solver([p], opts) as s:
        rc, res = s.solve()
        got = s.potentials(0)
    assert rc == 0, res
    fc = O.final_check(p, got)
    assert fc["max_marginal_l1"] <= 1e-6
    fo, _, _ = O.solve(p, tol=1e-11, tol_kind="max")
    ref = O.final_check(p, fo)
    assert abs(res[0]["primal"] - ref["primal"]) <= 1e-6 * abs(ref["primal"])
    assert rel_err(O.gauge_fix(p, got), O.gauge_fix(p, fo), p.eps) <= 1e-4


def test_bf16_phase_alone_is_approximate(T):
    """Without refinement the absorbed BF16 kernel converges to its own fixed point,
    a few 1e-4 .. 1e-3 away in marginal L1 (evidence that the BF16 path runs)."""
    p = gen.prufer_problem(seed=3004, J=12, n=700, num_leaves=6, eps=0.01)
    opts = T.options(precision="fp32", tol=1e-7, tol_kind="max", apply_mode="bf16", refine_tol=0.0,
                     absorb_tau=24, lowp_start=4, max_half_steps=3000)
    with T.Solver([p], opts) as s:
        rc, res = s.solve()
        got = s.potentials(0)
    fc = O.final_check(p, got)
    assert np.isfinite(fc["max_marginal_l1"])
    assert 1e-6 < fc["max_marginal_l1"] < 2e-2


def test_bf16_iterate_close_to_oracle(T):
    """A few absorbed half-steps track the oracle's iterate to BF16 accuracy."""
    p = gen.prufer_problem(seed=3005, J=8, n=600, num_leaves=4, eps=0.02)
    opts = T.options(precision="fp32", apply_mode="bf16", lowp_start=2, absorb_tau=24)
    with T.Solver([p], opts) as s:
        s.half_steps(8)
        got = s.potentials(0)
    ref = O.run_half_steps(p, 8)
    assert marginal_gap(p, got, ref) <= 3e-2
    assert rel_err(got, ref, p.eps) <= 5e-2


def test_bf16_layouts_agree(T):
    """With and without the transposed FP32 costs (which also change the BF16
    column tasks' reduction split from 512 to 1024 rows) the BF16 iterates agree
    far inside the BF16 phase's own error (FP32 summation order differs, and with
    it the half-step at which an edge's drift crosses absorb_tau)."""
    p = gen.prufer_problem(seed=3006, J=10, n=1100, num_leaves=5, eps=0.01)
    out = {}
    for tr in (True, False):
        opts = T.options(precision="fp32", apply_mode="bf16", lowp_start=2, absorb_tau=24, transpose=tr)
        with T.Solver([p], opts) as s:
            s.half_steps(9)
            out[tr] = s.potentials(0)
    ref = O.run_half_steps(p, 9)
    assert rel_err(out[True], out[False], p.eps) <= 5e-4
    assert rel_err(out[True], ref, p.eps) <= 5e-2 and rel_err(out[False], ref, p.eps) <= 5e-2
