"""The allocation-free entry point (tree_ot_edge_apply_noalloc) against the
library's regular path, through the C ABI, on a GPU.

Callers that cannot allocate device memory (graph capture in progress,
pre-sized memory pools, real-time loops) use the allocation-free variant; its
messages must equal those the regular solver computes for the same edge.  The
regular path is read through a two-node problem: after one half-step the fixed
node's potential is f = -eps * m with m the message this entry point returns.
This file is collected last, and the test also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

import gen
from gen.problems import TreeProblem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _regular_message(T, C, g, eps):
    """m(x) = LSE_y(g(y) - C(x,y)/eps) via tree_ot_create/set_potentials/half_steps."""
    n_rows, n_cols = C.shape
    rng = np.random.default_rng(5)
    mu = gen.dirichlet_marginal(n_rows, rng)
    p = TreeProblem(name="edge", edges=np.array([[0, 1]], np.int32), n=np.array([n_rows, n_cols], np.int32),
                    fixed=np.array([True, False]), marginals={0: mu}, eps=eps,
                    coords=[np.zeros((n_rows, 1), np.float32), np.zeros((n_cols, 1), np.float32)],
                    cost_scale=1.0, cost_kind="dense", dense_costs=[C])
    with T.Solver([p], T.options(precision="fp32")) as s:
        s.set_potential(0, 1, eps * g)       # f_(1,0) = eps g (node 1 is free: log gamma = 0)
        s.half_steps(1)                      # colour 0 = the fixed node 0: f_(0,1) = -eps m
        return -s.potential(0, 0) / eps


def test_noalloc_matches_regular_path_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    rng = np.random.default_rng(11)
    n_rows, n_cols, eps = 1100, 2500, 0.02     # ragged rows and three 1024-column splits
    ld = 2504
    X = rng.random((n_rows, 3)).astype(np.float32)
    Y = rng.random((n_cols, 3)).astype(np.float32)
    C = gen.sqeuclid_cost_f32(X, Y, 1.0)
    C_pad = np.full((n_rows, ld), 7.0, np.float32)   # padding the entry point must ignore
    C_pad[:, :n_cols] = C
    dev = torch.device("cuda")
    cost = torch.from_numpy(C_pad).to(dev)
    m_out = torch.full((n_rows,), float("nan"), dtype=torch.float64, device=dev)
    for call in range(2):
        g = rng.normal(0.0, 3.0, size=n_cols) + np.log(rng.dirichlet(np.ones(n_cols)))
        T.treeot.edge_apply_noalloc(cost, torch.from_numpy(g).to(dev), eps, m_out, ld=ld)
        torch.cuda.synchronize()
        got = m_out.cpu().numpy()
        ref = _regular_message(T, C, g, eps)
        assert np.all(np.isfinite(got)), call
        # the potentials tolerance of the parity tests: 1e-4 relative
        scale = max(float(np.max(np.abs(ref))), 1.0)
        assert float(np.max(np.abs(got - ref))) <= 1e-4 * scale, call


def test_noalloc_rejects_oversize_request():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    dev = torch.device("cuda")
    n_rows, n_cols = 70000, 8192          # 2 * 70000 * 8 partial floats > 2^20
    cost = torch.zeros((1, 8192), dtype=torch.float32, device=dev).expand(n_rows, 8192)
    g = torch.zeros(n_cols, dtype=torch.float64, device=dev)
    m_out = torch.zeros(16, dtype=torch.float64, device=dev)
    with pytest.raises(T.TreeOTError) as ei:
        T.treeot.edge_apply_noalloc(cost, g, 0.1, m_out, ld=8192)
    assert ei.value.kind == "ARG"
