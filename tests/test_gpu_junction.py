"""General graphs through modified junction trees (Sec. 4) on the GPU: the
Wasserstein least-squares problem (Sec. 2.3, the paper's second workload in
Sec. 5) reduced to its tree of separators and solved by the library's kernels,
against the junction-tree oracle (the general separator update of
prop:general_algo) on the same FP32 costs.

Tolerances: the FP32 path's (plans within 1e-6 in L1 per clique after T
half-steps; converged: max marginal L1 <= 1e-6 by the FP64 oracle)."""
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


@pytest.mark.parametrize("J,d", [(4, 8), (12, 10), (3, 33)])
@pytest.mark.parametrize("steps", [1, 2, 9])
def test_wls_iterates_match_the_junction_tree_oracle(T, J, d, steps):
    from paper_2406_10849_gb300 import junction as JR
    jt = fp32_costs(gen.wls_junction_tree(8000 + J + d, J, d))
    tr = JR.reduce_junction_tree(jt)
    with T.Solver([tr], T.options(precision="fp32")) as s:
        s.half_steps(steps)
        got = s.potentials(0)
    Bj = JT.plans(jt, JT.run_half_steps(jt, steps))
    for e, (a, b) in enumerate(np.asarray(tr.edges)):
        B = JR.clique_plan(tr, jt, e, O.plan(tr, got, int(a), int(b)))
        assert float(np.abs(B - Bj[tr.edge_clique[e]]).sum()) <= 1e-6, e


def test_wls_converged(T):
    from paper_2406_10849_gb300 import junction as JR
    jt = fp32_costs(gen.wls_junction_tree(8100, 6, 12))
    tr = JR.reduce_junction_tree(jt)
    with T.Solver([tr], T.options(precision="fp32", tol=1e-6, tol_kind="max", max_half_steps=200000)) as s:
        rc, res = s.solve()
        got = s.potentials(0)
    assert rc == 0, res
    fc = O.final_check(tr, got)
    assert fc["max_marginal_l1"] <= 1e-6
    du, _, r = JT.solve(jt, tol=1e-11, max_half_steps=500000)
    assert r < 1e-11
    for e, (a, b) in enumerate(np.asarray(tr.edges)):
        B = JR.clique_plan(tr, jt, e, O.plan(tr, got, int(a), int(b)))
        Bj = JT.plans(jt, du)[tr.edge_clique[e]]
        assert float(np.abs(B - Bj).sum()) <= 2e-5, e
    assert abs(res[0]["transport_cost"] - JT.transport_cost(jt, du)) <= 1e-5 * JT.transport_cost(jt, du)
