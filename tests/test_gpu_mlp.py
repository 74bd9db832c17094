"""Perceptron kernels against the FP64 CPU oracle (needs a GPU).

Forward: the bf16 weights widened to FP32 with FP32 accumulation and tanhf
versus FP64 on the same bf16-rounded weights: |dy| <= 1e-5 (1 + |y|).
Gradient: FP32 sums over rows versus FP64: <= 1e-4 of the largest gradient
component.  Adam: the FP32 update versus FP64 on the same gradient."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1206_1199_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch  # noqa: F401
    L.load()
    from paper_1206_1199_gb300 import mlp
    return mlp


def data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 6)).astype(np.float32)
    t = (np.sin(x[:, 0]) - 0.5 * x[:, 5] + 0.1 * x[:, 1] * x[:, 2]).astype(np.float32)
    return x, t


def test_forward_matches_oracle(M):
    net = M.ThetaNet(M.init_weights(3))
    x, _ = data(3000, 1)
    y = net.predict(x)
    wb = omlp.bf16_round(net.weights())
    np.testing.assert_array_equal(net.weights_bf16().astype(np.uint32) << 16,
                                  wb.astype(np.float32).view(np.uint32))
    yr = omlp.forward(wb, net.scale(x).astype(np.float64))
    assert np.all(np.abs(y - yr) <= 1e-5 * (1 + np.abs(yr)))


@pytest.mark.parametrize("n", [1, 127, 128, 129, 5000])
def test_gradient_matches_oracle(M, n):
    net = M.ThetaNet(M.init_weights(4))
    x, t = data(n, 2)
    g, loss = net.grad(x, t)
    wb = omlp.bf16_round(net.weights())
    xs = net.scale(x).astype(np.float64)
    gr = omlp.grad(wb, xs, t)
    assert np.abs(g - gr).max() <= 1e-4 * np.abs(gr).max()
    assert abs(loss - omlp.loss(wb, xs, t)) <= 1e-4 * omlp.loss(wb, xs, t)
    g2, _ = net.grad(x, t)
    np.testing.assert_array_equal(g, g2)  # fixed summation order


def test_adam_step_matches_oracle(M):
    net = M.ThetaNet(M.init_weights(5))
    x, t = data(1000, 3)
    w0 = net.weights().astype(np.float64)
    g, _ = net.grad(x, t)
    net.train(x, t, steps=1, lr=1e-2)
    w1, m1, v1 = omlp.adam(w0, np.zeros(omlp.NP), np.zeros(omlp.NP), g.astype(np.float64), 1, 1e-2)
    np.testing.assert_allclose(net.weights(), w1, rtol=0, atol=1e-6)
    np.testing.assert_array_equal(net.weights_bf16().astype(np.uint32) << 16,
                                  omlp.bf16_round(net.weights()).astype(np.float32).view(np.uint32))


def test_training_reduces_loss(M):
    net = M.ThetaNet(M.init_weights(6))
    x, t = data(8192, 4)
    net.fit_scaler(x)
    hist = net.train(x, t, steps=600, lr=3e-3, log_every=100)
    assert hist[-1] < 0.05 * hist[0]
    xv, tv = data(2048, 5)
    assert np.mean((net.predict(xv) - tv) ** 2) < 0.05 * np.var(tv)


def test_select_theta_matches_oracle(M):
    net = M.ThetaNet(M.init_weights(7))
    rng = np.random.default_rng(8)
    feats = rng.normal(size=(500, 5)).astype(np.float32)
    grid = np.linspace(0.3, 0.9, 13).astype(np.float32)
    out = net.select_theta(feats, grid, -0.05)
    rows = np.concatenate([np.repeat(feats, 13, 0), np.tile(grid, 500)[:, None]], 1)
    wb = omlp.bf16_round(net.weights())
    ref, y = omlp.select_theta(wb, net.scale(rows).astype(np.float64).reshape(500, 13, 6), grid.astype(np.float64),
                               -0.05, 0.5)
    # decisions are compared where no prediction sits within rounding of the target
    clear = np.all(np.abs(y + 0.05) > 1e-4, axis=1)
    assert clear.sum() > 400
    np.testing.assert_array_equal(out[clear], ref[clear].astype(np.float32))
    # a non-finite prediction falls back
    bad = feats.copy()
    bad[0, 0] = np.nan
    assert net.select_theta(bad, grid, -0.05, fallback=0.5)[0] == np.float32(0.5)
