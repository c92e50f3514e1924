"""GPU rank-predictor kernels against the numpy oracle (FP64): forward
outputs, minibatch loss and gradient, one Adam step, and a short training
run.  The CUDA side computes in FP32, so the bars are FP32-level relative
errors (forward 1e-5, gradient 1e-4 of the largest entry, Adam 1e-5 of the
step, training losses 1e-3)."""
import numpy as np
import pytest

from oracle import mlp
from paper_1811_11248_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1811_11248_gb300 import build, hsolve
    build.build()
    hsolve.lib()
    assert torch.cuda.is_available()
    return hsolve


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def sample(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 8)).astype(np.float32)
    t = (np.maximum(X[:, 0], 0) + 0.3 * X[:, 1] * X[:, 2]).astype(np.float32)
    return X, t


@pytest.mark.parametrize("n", [1, 127, 1000])
def test_forward(hs, n):
    th = inputs.mlp_init_params(3).astype(np.float32)
    X, _ = sample(n, 1)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    hs.hs_mlp_forward(f32(th), f32(X), n, y)
    torch.cuda.synchronize()
    yo, _ = mlp.forward(th.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), yo, rtol=1e-5, atol=1e-5 * np.abs(yo).max())


@pytest.mark.parametrize("batch", [1, 37, 256])
def test_gradient(hs, batch):
    th = inputs.mlp_init_params(4).astype(np.float32)
    X, t = sample(600, 2)
    idx = np.random.default_rng(3).choice(600, batch, replace=False).astype(np.int32)
    g = torch.empty(mlp.NPARAM, dtype=torch.float32, device="cuda")
    L = torch.empty(1, dtype=torch.float32, device="cuda")
    hs.hs_mlp_grad(f32(th), f32(X), f32(t), torch.from_numpy(idx).cuda(), batch, g, L)
    torch.cuda.synchronize()
    Lo, go = mlp.loss_and_grad(th.astype(np.float64), X[idx].astype(np.float64), t[idx].astype(np.float64))
    assert abs(float(L.item()) - Lo) <= 1e-5 * max(1.0, Lo)
    gg = g.cpu().numpy()
    assert np.abs(gg - go).max() <= 1e-4 * np.abs(go).max(), np.abs(gg - go).max()


def test_adam_step(hs):
    th = inputs.mlp_init_params(5).astype(np.float32)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(mlp.NPARAM).astype(np.float32)
    m0 = (0.1 * rng.standard_normal(mlp.NPARAM)).astype(np.float32)
    v0 = (0.01 * rng.random(mlp.NPARAM)).astype(np.float32)
    dth, dm, dv = f32(th), f32(m0), f32(v0)
    hs.hs_mlp_adam(dth, f32(g), dm, dv, 7, 1e-3)
    torch.cuda.synchronize()
    tho, mo, vo = mlp.adam_step(th.astype(np.float64), g.astype(np.float64), m0.astype(np.float64),
                                v0.astype(np.float64), 7, 1e-3)
    np.testing.assert_allclose(dm.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)
    # 1 - beta2 rounds to 0.99998713e-3 in FP32: 1.3e-5 relative on the g^2 term
    np.testing.assert_allclose(dv.cpu().numpy(), vo, rtol=3e-5, atol=1e-9)
    step = np.abs(tho - th).max()
    assert np.abs(dth.cpu().numpy() - tho).max() <= 1e-5 * max(step, 1e-3) + 1e-6


def test_training_run_tracks_oracle(hs):
    """Same initial weights and batch order on both sides: per-step losses
    agree while both descend (FP32 vs FP64 trajectories drift slowly)."""
    X, t = sample(2048, 7)
    th0 = inputs.mlp_init_params(8)
    order = inputs.mlp_batch_order(2048, 128, 3, seed=9)
    thg, lg = hs.hs_mlp_train(th0, X, t, order, 128, 3e-3)
    tho, lo = mlp.train_steps(th0.copy(), X.astype(np.float64), t.astype(np.float64), order, 128, 3e-3)
    assert len(lg) == len(lo) == 48
    np.testing.assert_allclose(lg, lo, rtol=1e-3)
    assert lg[-8:].mean() < 0.5 * lg[:8].mean()
