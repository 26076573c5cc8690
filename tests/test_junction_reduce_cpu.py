"""The reduction of a modified junction tree with trivial inclusion sequences to a
tree of separators (paper_2406_10849_gb300/junction.py), checked on the CPU:
the tree oracle on the reduced problem and the junction-tree oracle on the
original follow the same iterates (Wasserstein least squares, Sec. 2.3 / Sec. 5),
and junction trees with nested inclusion sequences are rejected."""
import numpy as np
import pytest

import gen
from oracle import junction_tree as JT
from oracle import tree_ot as O
from paper_2406_10849_gb300 import junction as JR


def fp32_costs(jt):
    """The junction tree with its costs rounded to FP32, as the reduced problem stores them."""
    jt.clique_costs = [np.asarray(C, np.float32).astype(np.float64) for C in jt.clique_costs]
    return jt


@pytest.mark.parametrize("J,d", [(3, 4), (5, 3)])
def test_wls_reduces_to_a_star_with_the_same_iterates(J, d):
    jt = fp32_costs(gen.wls_junction_tree(11, J, d))
    jt.eps = 0.1
    tr = JR.reduce_junction_tree(jt)
    assert tr.num_nodes == J + 1 and list(tr.n) == [d * d] + [d] * J
    assert not tr.fixed[0] and all(tr.fixed[1:])
    O.validate(tr)
    for T in (1, 2, 5):
        f = O.run_half_steps(tr, T)
        du = JT.run_half_steps(jt, T)
        Bj = JT.plans(jt, du)
        for e, (a, b) in enumerate(np.asarray(tr.edges)):
            B = JR.clique_plan(tr, jt, e, O.plan(tr, f, int(a), int(b)))
            np.testing.assert_allclose(B, Bj[tr.edge_clique[e]], rtol=1e-11, atol=1e-16)


def test_tree_round_trip():
    p = gen.chain_problem(seed=1004, n=5, eps=0.2)
    tr = JR.reduce_junction_tree(gen.tree_as_junction_tree(p))
    assert [tuple(map(int, e)) for e in tr.edges] == [tuple(map(int, e)) for e in p.edges]
    for e in range(p.num_edges):
        np.testing.assert_array_equal(tr.dense_cost(e), p.dense_cost(e))


def test_nested_inclusion_is_rejected():
    with pytest.raises(JR.NotReducible):
        JR.reduce_junction_tree(gen.nested_junction_tree(1))
