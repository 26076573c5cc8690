"""The persistent forest launch (TREE_OT_OPT_PERSISTENT): chunks of half-steps of a
batch of trees as one launch each, problems advancing on their own phase counters.

It runs the same per-task and per-chunk device code as the per-half-step
launches, in a different order across problems only, so iterates must equal
theirs bit for bit (potentials after T half-steps), and the oracle's within the
FP32 path's tolerances.  The failure path (a wait that runs out) is tested with
the TEST_STALL hook: node items never report completion, no GPU fault."""
import numpy as np
import pytest

import gen
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


def forest(seed, count, J_range=(4, 12), n_range=(64, 700), D=2):
    rng = np.random.default_rng(seed)
    return [gen.random_tree_problem(rng, int(rng.integers(J_range[0], J_range[1] + 1)), n_range=n_range,
                                    eps_range=(0.005, 0.05), D=D, name=f"pf{seed}_{i}") for i in range(count)]


def rel_err(got, ref, eps):
    worst = 0.0
    for key in ref:
        scale = max(float(np.max(np.abs(ref[key]))), eps)
        worst = max(worst, float(np.max(np.abs(got[key] - ref[key]))) / scale)
    return worst


@pytest.mark.parametrize("D", [1, 2, 3])
def test_persistent_iterates_equal_per_half_step_launches(T, D):
    probs = forest(5100 + D, 12, D=D)
    with T.Solver(probs, T.options(precision="fp32", persistent=True, autotune=False)) as sp, \
            T.Solver(probs, T.options(precision="fp32", autotune=False)) as sl:
        assert sp.plan_stats()["persistent"] == 2 and sl.plan_stats()["persistent"] == 0
        for steps in (1, 4, 9):   # 1 + 4 + 9 = 14 half-steps, chunks of odd and even length
            sp.half_steps(steps)
            sl.half_steps(steps)
        for i in range(len(probs)):
            a, b = sp.potentials(i), sl.potentials(i)
            for key in a:
                np.testing.assert_array_equal(a[key], b[key], err_msg=f"{i} {key}")
    for i in (0, 5, 11):
        ref = O.run_half_steps(probs[i], 14)
        with T.Solver([probs[i]], T.options(precision="fp32", persistent=True, autotune=False)) as s1:
            s1.half_steps(14)
            assert rel_err(s1.potentials(0), ref, probs[i].eps) <= 1e-4


def test_persistent_solve_certified(T):
    probs = forest(5200, 16)
    with T.Solver(probs, T.options(precision="fp32", tol=1e-6, tol_kind="max", max_half_steps=40000,
                                   persistent=True, autotune=False)) as s:
        rc, res = s.solve()
        assert rc == 0, [r["max_marginal_l1"] for r in res]
        steps = [r["half_steps"] for r in res]
        assert len(set(steps)) > 1           # trees retired at different half-steps
        for i in (2, 7, 13):
            fc = O.final_check(probs[i], s.potentials(i))
            assert fc["max_marginal_l1"] <= 1e-6
            assert abs(res[i]["max_marginal_l1"] - fc["max_marginal_l1"]) <= 1e-7


def test_persistent_full_batch_sampled(T):
    """The 512-tree batch in persistent launches: two half-steps, the largest, widest,
    smallest-eps and median trees re-run by the oracle; the timing at create picks a form."""
    probs = gen.batched_problems(seed=4000)
    sizes = np.array([pp.elements_per_half_step() for pp in probs])
    pick = {int(np.argmax(sizes)), int(np.argmax([int(np.max(pp.n)) for pp in probs])),
            int(np.argmin([pp.eps for pp in probs])), int(np.argsort(sizes)[len(probs) // 2])}
    with T.Solver(probs, T.options(precision="fp32", persistent=True, autotune=False)) as s:
        assert s.plan_stats()["persistent"] == 2
        s.half_steps(2)
        for i in sorted(pick):
            ref = O.run_half_steps(probs[i], 2)
            assert rel_err(s.potentials(i), ref, probs[i].eps) <= 1e-4, i
    with T.Solver(probs[:64], T.options(precision="fp32", persistent=True)) as s:
        assert s.plan_stats()["persistent"] in (0, 2, 3)


def test_persistent_wait_timeout_reports_error(T):
    """TEST_STALL: node items never report completion, so the next apply items' bounded
    waits run out (1 s); the launch ends, the solve returns TREE_OT_ERR_TIMEOUT, and a new
    handle on the same device solves normally."""
    probs = forest(5300, 4, n_range=(32, 64))
    with T.Solver(probs, T.options(precision="fp32", persistent=True, autotune=False, test_stall=True,
                                   tol=1e-6, tol_kind="max")) as s:
        assert s.plan_stats()["persistent"] == 2
        with pytest.raises(T.TreeOTError) as ei:
            s.solve()
    assert ei.value.kind == "TIMEOUT"
    with T.Solver(probs, T.options(precision="fp32", persistent=True, autotune=False, tol=1e-6,
                                   tol_kind="max")) as s:
        rc, _ = s.solve()
    assert rc == 0
