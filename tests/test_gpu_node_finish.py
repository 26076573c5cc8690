"""Where the node update's bookkeeping runs (TREE_OT_OPT_NODE_DEFER / _ARRIVE).

The normalisers Z_j, the per-edge stopping terms, the stopping quantity of the
iterate, phase control and retirement are finished either by the last chunk to
arrive or by one extra launch after the chunks.  The chunks' own arithmetic is
the same in both forms, so the potentials must be equal bit for bit; the
stopping quantity differs only in the order of its sums; and with defer
forced on a small tree the iterates meet the oracle's at the FP32 path's
tolerance."""
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


def forest(seed, count, n_range=(40, 600), D=2):
    rng = np.random.default_rng(seed)
    return [gen.random_tree_problem(rng, int(rng.integers(3, 11)), n_range=n_range, eps_range=(0.005, 0.05), D=D,
                                    name=f"nf{seed}_{i}") for i in range(count)]


def test_plan_stats_report_the_form(T):
    p = gen.chain_problem(seed=1001, J=5, n=70, eps=0.05)
    for finish, want in (("auto", 0), ("defer", 3), ("arrive", 0)):
        with T.Solver([p], T.options(precision="fp32", node_finish=finish)) as s:
            assert s.plan_stats()["node_defer"] == want, finish


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_deferred_iterates_equal_arrival(T, precision):
    probs = forest(7100, 14)
    kw = dict(precision=precision, autotune=False)
    with T.Solver(probs, T.options(node_finish="defer", **kw)) as sd, \
            T.Solver(probs, T.options(node_finish="arrive", **kw)) as sa:
        for steps in (1, 2, 6):
            sd.half_steps(steps)
            sa.half_steps(steps)
        for i in range(len(probs)):
            a, b = sd.potentials(i), sa.potentials(i)
            for key in a:
                np.testing.assert_array_equal(a[key], b[key], err_msg=f"{i} {key}")
            # a chunk's per-edge terms are FP32 sums whose warp contributions meet in
            # shared-memory atomics (any order, in either form): agreement to FP32 rounding
            ds, dm = sd.residual_history(i, 1, 8)
            as_, am = sa.residual_history(i, 1, 8)
            np.testing.assert_allclose(ds, as_, rtol=2e-6, atol=0.0)
            np.testing.assert_allclose(dm, am, rtol=2e-6, atol=0.0)


def test_deferred_iterates_match_oracle(T):
    p = gen.random_tree_problem(np.random.default_rng(7200), 9, n_range=(30, 1100), eps_range=(0.01, 0.01), D=2,
                                name="nf_oracle")
    for steps in (1, 2, 9):
        ref = O.run_half_steps(p, steps)
        with T.Solver([p], T.options(precision="fp32", node_finish="defer")) as s:
            s.half_steps(steps)
            got = s.potentials(0)
        for key in ref:
            scale = max(float(np.max(np.abs(ref[key]))), p.eps)
            assert float(np.max(np.abs(got[key] - ref[key]))) <= 1e-4 * scale, (steps, key)


def test_deferred_solve_retires_like_arrival(T):
    probs = forest(7300, 20)
    kw = dict(precision="fp32", tol=1e-6, tol_kind="max", max_half_steps=40000, autotune=False)
    out = {}
    for finish in ("defer", "arrive"):
        with T.Solver(probs, T.options(node_finish=finish, **kw)) as s:
            rc, res = s.solve()
            assert rc == 0, finish
            out[finish] = (res, [s.potentials(i) for i in range(len(probs))])
    (rd, pd), (ra, pa) = out["defer"], out["arrive"]
    assert len({r["half_steps"] for r in rd}) > 1       # retirements at different half-steps
    for i in range(len(probs)):
        assert rd[i]["half_steps"] == ra[i]["half_steps"], i
        assert rd[i]["max_marginal_l1"] <= 1e-6
        for key in pd[i]:
            np.testing.assert_array_equal(pd[i][key], pa[i][key])
    for i in (0, 9, 19):
        assert O.final_check(probs[i], pd[i])["max_marginal_l1"] <= 1e-6


def test_deferred_shared_kernel_phase(T):
    """Phase control (entering and leaving the BF16 phase, the stall detector) runs in
    the deferred launch too: same phase spans and half-steps as the arrival form."""
    probs = gen.warmstart_stars(9_100_000, 48, side=16, eps=0.005)
    kw = dict(apply_mode="bf16", lowp_start=0, refine_tol=1e-5, tol=1e-6, tol_kind="max", max_half_steps=20000)
    out = {}
    for finish in ("defer", "arrive"):
        with T.Solver(probs, T.options(node_finish=finish, **kw)) as s:
            rc, res = s.solve()
            assert rc == 0, finish
            out[finish] = res
    for a, b in zip(out["defer"], out["arrive"]):
        assert a["lowp_half_steps"] == b["lowp_half_steps"] > 0
        assert a["half_steps"] == b["half_steps"]
        assert a["max_marginal_l1"] <= 1e-6
