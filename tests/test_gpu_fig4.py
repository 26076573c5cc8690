"""The paper's numerical experiment (Sec. 5, Fig. 4(a)) on the GPU against the
oracle: log-normal barycenters with eps = delta / (4 |E| log d), stopping sum
below delta' = delta / (8 C_inf), solved as one batch.

* Half-steps: the GPU measures the stopping sum of iterate t during half-step
  t + 1 and retires there, so its count is the oracle's + 1; FP32 rounding may
  move the crossing of delta' by one half-step: |GPU - (oracle + 1)| <= 1.
* The GPU's rounding certifies every instance delta-approximate (its reported
  bound of lemma lem:round_applied is below delta) and, on the small ones, the
  rounded cost is within that bound of an LP optimum.
"""
import numpy as np
import pytest

import gen
from oracle import tree_ot as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(2, 10, 0), (3, 10, 1), (3, 40, 2), (3, 160, 3), (4, 10, 4), (6, 10, 5), (8, 12, 6), (12, 10, 7)]


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    return T


def test_fig4_half_steps_and_delta_approximation(T):
    import textbook_ot as TB
    delta = 0.2
    probs = [gen.lognormal_barycenter(7_000_000 + s, E, d, delta) for E, d, s in CASES]
    tol = probs[0].meta["tol"]
    with T.Solver(probs, T.options(precision="fp32", tol=tol, tol_kind="sum", max_half_steps=100000)) as s:
        rc, res = s.solve()
        rr = s.round()
    assert rc == 0
    for p, r, q in zip(probs, res, rr):
        _, t_oracle, _ = O.solve(p, tol=tol, tol_kind="sum", max_half_steps=100000)
        assert abs(r["half_steps"] - (t_oracle + 1)) <= 1, (p.name, r["half_steps"], t_oracle)
        assert r["residual_sum_l1"] < tol
        assert q["bound"] < delta, p.name
        if int(p.n[0]) <= 12 and p.num_edges <= 4:
            costs = [O.cost(p, int(a), int(b)) for a, b in p.edges]
            opt = TB.lp_optimum(p.num_nodes, [tuple(map(int, e)) for e in p.edges], [int(x) for x in p.n],
                                p.fixed, p.marginals, costs)
            assert opt - 1e-7 <= q["rounded_transport_cost"] <= opt + q["bound"] + 1e-7, p.name
