"""GPU parity of the two stored-cost apply kernels (bulk-copy staged and plain
loads), each forced through options.flags, against the FP64 oracle.

Same bars as the other parity tests: potentials within 1e-4 relative and the
FP64 marginals of the GPU iterate within 1e-6 (L1) of the oracle iterate's;
converged solves certified by the oracle at 1e-6.
"""
import numpy as np
import pytest

import gen
from gen.problems import TreeProblem
from oracle import tree_ot as O

from test_gpu_parity import marginal_gap, random_tree, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    return T


def ragged_chain(seed=21, sizes=(3, 1, 2053, 4, 1030, 129), eps=0.02):
    """Chain with supports of 1..4 points next to 1030 and 2053: ragged ROW and COL tiles."""
    rng = np.random.default_rng(seed)
    J = len(sizes)
    edges = gen.chain_edges(J)
    fixed = gen.leaves_of(J, edges)
    coords = [rng.random((k, 2)).astype(np.float32) for k in sizes]
    marg = {j: gen.dirichlet_marginal(sizes[j], rng) for j in range(J) if fixed[j]}
    return TreeProblem(name="ragged_chain", edges=edges, n=np.asarray(sizes, np.int32), fixed=fixed,
                       marginals=marg, eps=eps, coords=coords, cost_scale=1.0, cost_kind="dense", meta={})


DENSE_CASES = {
    "chain_dense_n70": lambda: gen.chain_problem(seed=1001, n=70, eps=0.01),
    "prufer12_dense_n1100": lambda: gen.prufer_problem(seed=3001, J=12, n=1100, num_leaves=6, eps=0.01),
    "tree7_unequal_2d_dense": lambda: random_tree(12, 7, (5, 700), 0.03, D=2, kind="dense"),
    "ragged_chain_dense": ragged_chain,
}


@pytest.mark.parametrize("transpose", [True, False])
@pytest.mark.parametrize("kernel", ["tma", "ldg"])
@pytest.mark.parametrize("name", sorted(DENSE_CASES))
@pytest.mark.parametrize("steps", [1, 9])
def test_dense_kernel_iterate_parity(T, kernel, name, steps, transpose):
    """Both stored-cost kernels, with the column owner's apply on the transposed
    copy (rows) or on the given layout (columns)."""
    p = DENSE_CASES[name]()
    ref = O.run_half_steps(p, steps)
    with T.Solver([p], T.options(precision="fp32", dense_kernel=kernel, transpose=transpose)) as s:
        assert s.plan_stats()["dense_tma"] == (1 if kernel == "tma" else 0)
        s.half_steps(steps)
        got = s.potentials(0)
    assert rel_err(got, ref, p.eps) <= 1e-4
    assert marginal_gap(p, got, ref) <= 1e-6


@pytest.mark.parametrize("kernel", ["tma", "ldg"])
def test_dense_kernel_converged(T, kernel):
    p = DENSE_CASES["prufer12_dense_n1100"]()
    with T.Solver([p], T.options(precision="fp32", tol=5e-7, tol_kind="max", max_half_steps=60000,
                                 dense_kernel=kernel)) as s:
        rc, res = s.solve()
        f = s.potentials(0)
    assert rc == 0 and res[0]["status"] == 0
    chk = O.final_check(p, f)
    assert chk["max_marginal_l1"] <= 1e-6
    assert abs(res[0]["max_marginal_l1"] - chk["max_marginal_l1"]) <= 1e-7


def test_kernels_agree_on_a_batch(T):
    """A forest of dense trees: both kernels give the same iterate up to rounding
    order (the staged kernel splits column tiles across warps differently)."""
    probs = [random_tree(40 + i, 5 + i % 4, (16, 900), 0.01 + 0.005 * i, D=2, kind="dense") for i in range(6)]
    out = {}
    for kernel in ("tma", "ldg"):
        with T.Solver(probs, T.options(precision="fp32", dense_kernel=kernel)) as s:
            s.half_steps(6)
            out[kernel] = [s.potentials(i) for i in range(len(probs))]
    for i, p in enumerate(probs):
        assert rel_err(out["tma"][i], out["ldg"][i], p.eps) <= 2e-5
        ref = O.run_half_steps(p, 6)
        assert marginal_gap(p, out["tma"][i], ref) <= 1e-6


def test_staged_kernel_timeout_is_reported(T):
    """Failure path of the staged kernel, without a GPU fault: with the test hook
    its producer issues nothing, every consumer's bounded wait runs out (250 ms),
    the kernel returns, and the solve reports TREE_OT_ERR_TIMEOUT; the device
    stays usable for the next handle."""
    import time
    p = DENSE_CASES["chain_dense_n70"]()
    opts = T.options(precision="fp32", test_stall=True, use_graph=False, check_every=2, max_half_steps=2)
    with T.Solver([p], opts) as s:
        t0 = time.perf_counter()
        with pytest.raises(T.TreeOTError) as ei:
            s.solve()
        dt = time.perf_counter() - t0
    assert ei.value.code == -10, ei.value     # TREE_OT_ERR_TIMEOUT
    assert dt < 30.0
    with T.Solver([p], T.options(precision="fp32", dense_kernel="tma")) as s:
        s.half_steps(1)
        ref = O.run_half_steps(p, 1)
        assert rel_err(s.potentials(0), ref, p.eps) <= 1e-4
