"""Shared-kernel BF16 phase (apply_mode "bf16" on squared-Euclidean problems
whose directed edges share one support pair, scale and eps): iterate parity
with the FP64 oracle, certified solves, and batches that mix shared, separately
shared and unshared problems in one handle."""
import numpy as np
import pytest

import gen
from oracle import tree_ot as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    return T


def rel_err(got, ref, eps):
    """max over directed edges of max|got - ref| / max(|ref|_inf, eps)."""
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
            worst = max(worst, gap if np.isfinite(gap) else float("inf"))
    return worst


def stars(count, side=16, eps=0.01, seed=7_000_000):
    return gen.warmstart_stars(seed, count, side=side, eps=eps)


@pytest.mark.parametrize("steps", [1, 2, 7])
def test_shared_kernel_iterates_match_oracle(T, steps):
    """Six 16x16 stars at eps 0.01 in the phase from the first half-step: the
    split-BF16 product keeps the iterate within FP32-path tolerances."""
    probs = stars(6)
    with T.Solver(probs, T.options(apply_mode="bf16", lowp_start=0, refine_tol=0.0)) as s:
        s.half_steps(steps)
        got = {i: s.potentials(i) for i in (0, 3, 5)}
    for i, f in got.items():
        ref = O.run_half_steps(probs[i], steps)
        assert rel_err(f, ref, probs[i].eps) <= 1e-4
        assert marginal_gap(probs[i], f, ref) <= 1e-5


def test_shared_kernel_ragged_support(T):
    """Six 11x11 stars (121 points: neither the four-point vectors of the
    envelope and operand builds nor the 64-point reduction padding divide it)
    follow the oracle for five half-steps in the phase."""
    probs = stars(6, side=11, eps=0.01, seed=7_050_000)
    with T.Solver(probs, T.options(apply_mode="bf16", lowp_start=0, refine_tol=0.0)) as s:
        s.half_steps(5)
        got = {i: s.potentials(i) for i in (0, 5)}
    with T.Solver(probs, T.options()) as s:  # the FP32 path, for contrast
        s.half_steps(5)
        fp32 = s.potentials(0)
    assert any(not np.array_equal(got[0][k], fp32[k]) for k in fp32)  # the phase ran
    for i, f in got.items():
        ref = O.run_half_steps(probs[i], 5)
        assert rel_err(f, ref, probs[i].eps) <= 1e-4
        assert marginal_gap(probs[i], f, ref) <= 1e-5


def test_shared_kernel_solve_is_certified(T):
    """Twelve 16x16 stars at eps 0.005: the phase runs until the stopping
    quantity is below refine_tol, FP32 sweeps finish, the FP64-grade check
    certifies every star at 1e-6, and the oracle agrees."""
    probs = stars(12, eps=0.005, seed=7_100_000)
    with T.Solver(probs, T.options(apply_mode="bf16", tol=1e-6, tol_kind="max", max_half_steps=20000)) as s:
        rc, res = s.solve()
        fs = {i: s.potentials(i) for i in (0, 11)}
    assert rc == 0, [r["max_marginal_l1"] for r in res]
    assert all(r["lowp_half_steps"] > 0 for r in res)
    assert all(r["max_marginal_l1"] <= 1e-6 for r in res)
    for i, f in fs.items():
        assert O.final_check(probs[i], f)["max_marginal_l1"] <= 1.5e-6


def test_mixed_batch(T):
    """One handle: four 12x12 stars at eps 0.01 (one shared kernel), two at
    eps 0.02 (another), a 5-leaf 20x20 star (its own, 10 columns) and a random
    tree with distinct supports (no sharing: FP32 throughout)."""
    rng = np.random.default_rng(41)
    tree = gen.random_tree_problem(rng, 7, n_range=(20, 90), eps_range=(0.03, 0.03), D=2, name="rt41")
    tree.cost_kind = "sqeuclid"
    probs = (stars(4, side=12, eps=0.01, seed=7_200_000) + stars(2, side=12, eps=0.02, seed=7_300_000)
             + [gen.star_problem(seed=2003, leaves=5, side=20, eps=0.005), tree])
    steps = 5
    with T.Solver(probs, T.options(apply_mode="bf16", lowp_start=0, refine_tol=0.0)) as s:
        s.half_steps(steps)
        got = [s.potentials(i) for i in range(len(probs))]
    for p, f in zip(probs, got):
        ref = O.run_half_steps(p, steps)
        assert rel_err(f, ref, p.eps) <= 1e-4, p.name
    with T.Solver(probs, T.options(apply_mode="bf16", tol=1e-6, tol_kind="max", max_half_steps=20000)) as s:
        rc, res = s.solve()
    assert rc == 0, [(p.name, r["status"], r["max_marginal_l1"], r["half_steps"], r["lowp_half_steps"])
                     for p, r in zip(probs, res)]
    assert [r["lowp_half_steps"] > 0 for r in res] == [True] * 7 + [False]


@pytest.mark.parametrize("side", [16, 19, 10])
def test_tensor_memory_product_matches_mma_sync(T, side):
    """The tcgen05 product over CTA pairs (256-row MMAs), the one over single CTAs
    (128-row MMAs) and the mma.sync product form the same split-BF16 sums, the
    last in a different order: 40 stars (320 columns per colour, a ragged third
    column tile whose second half lies wholly past the columns) agree after six
    half-steps.  Supports of 256, 361 and 100 points: rows padded to 256, 384
    and 128, so a pair tile is full, half past the padded rows, or wholly in the
    even CTA."""
    probs = stars(40, side=side, eps=0.01, seed=7_400_000 + side)
    got = {}
    for prod in ("auto", "one_cta", "mma"):
        with T.Solver(probs, T.options(apply_mode="bf16", lowp_start=0, refine_tol=0.0, sk_product=prod)) as s:
            assert s.plan_stats()["sk_product"] == {"auto": 3, "one_cta": 2, "mma": 1}[prod]
            s.half_steps(6)
            got[prod] = [s.potentials(i) for i in (0, 17, 39)]
    for i, a, b, c in zip((0, 17, 39), got["auto"], got["one_cta"], got["mma"]):
        assert rel_err(a, b, probs[i].eps) <= 1e-6
        assert rel_err(a, c, probs[i].eps) <= 1e-5


def test_large_support_two_pass_envelope(T):
    """Supports above 1024 points (33 x 33 = 1089) take the two-pass envelope
    kernel (the one-pass kernel holds at most 1024 points per CTA in registers):
    three stars follow the oracle for three half-steps in the phase."""
    probs = stars(3, side=33, eps=0.01, seed=7_500_000)
    with T.Solver(probs, T.options(apply_mode="bf16", lowp_start=0, refine_tol=0.0)) as s:
        s.half_steps(3)
        got = {i: s.potentials(i) for i in (0, 2)}
    for i, f in got.items():
        ref = O.run_half_steps(probs[i], 3)
        assert rel_err(f, ref, probs[i].eps) <= 1e-4
        assert marginal_gap(probs[i], f, ref) <= 1e-5
