"""Warm-start MLP kernels (forward, backward, Adam) against the FP64 reference."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    return T


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("dims,batch", [((100, 64, 48), 37), ((1025, 512, 1024), 256)])
def test_forward_and_gradients_match_reference(T, dims, batch):
    i, h, o = dims
    net = T.MLP(i, h, o, max_batch=256, seed=3)
    rng = np.random.default_rng(1)
    p = net.get_params()
    P = {k: v.astype(np.float64) for k, v in net.tensors(p).items()}
    x = rng.normal(size=(batch, i)).astype(np.float32)
    t = rng.normal(size=(batch, o)).astype(np.float32)
    dev = torch.device("cuda")
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    y = torch.zeros(batch, o, device=dev)
    net.forward(xd, y)
    g = torch.zeros(net.num_params, device=dev)
    loss = net.backward(xd, td, g)
    torch.cuda.synchronize()
    y_ref, _ = M.forward(P, x, bf16=True)
    assert rel(y.cpu().numpy(), y_ref) <= 2e-3
    loss_ref, g_ref = M.loss_and_grads(P, x, t, bf16=True)
    assert abs(loss - loss_ref) <= 2e-3 * loss_ref
    G = net.tensors(g.cpu().numpy())
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert rel(G[name], g_ref[name]) <= 1e-2, name
    # and against the unrounded FP64 network: BF16 accuracy
    y64, _ = M.forward(P, x, bf16=False)
    assert rel(y.cpu().numpy(), y64) <= 3e-2


def test_training_reduces_loss(T):
    rng = np.random.default_rng(2)
    i, h, o, B = 33, 64, 16, 128
    A = rng.normal(size=(i, o)) / np.sqrt(i)
    x = rng.normal(size=(B, i)).astype(np.float32)
    t = np.tanh(x @ A).astype(np.float32)
    dev = torch.device("cuda")
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    net = T.MLP(i, h, o, max_batch=B, seed=5)
    first = net.train_step(xd, td, 3e-3)
    for _ in range(300):
        last = net.train_step(xd, td, 3e-3)
    assert last < 0.1 * first, (first, last)
