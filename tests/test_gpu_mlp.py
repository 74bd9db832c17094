"""Perceptron kernels against the FP64 CPU oracle (needs a GPU).

Forward: the bf16 weights widened to FP32 with FP32 accumulation and tanhf
versus FP64 on the same bf16-rounded weights: |dy| <= 1e-5 (1 + |y|).
Gradient: FP32 sums over rows versus FP64: <= 1e-4 of the largest gradient
component.  Adam: the FP32 update versus FP64 on the same gradient.
Selection (otoo_select_theta, otoo_learned_theta): decisions equal to the
oracle's wherever no prediction lies within 1e-4 of its target (the two
sides round differently), targets within 1e-5 in log10."""
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


def std_rows(net, x):
    """The oracle's standardisation of rows (FP64)."""
    return (np.asarray(x, np.float64) - net.mean.astype(np.float64)) / net.std.astype(np.float64)


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
    yr = omlp.forward(wb, std_rows(net, x))
    assert np.all(np.abs(y - yr) <= 1e-5 * (1 + np.abs(yr)))


@pytest.mark.parametrize("n", [1, 127, 128, 129, 5000])
def test_gradient_matches_oracle(M, n):
    net = M.ThetaNet(M.init_weights(4))
    x, t = data(n, 2)
    g, loss = net.grad(x, t)
    wb = omlp.bf16_round(net.weights())
    xs = std_rows(net, x)
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
    ref, y = omlp.select_theta(wb, std_rows(net, rows).reshape(500, 13, 6), grid.astype(np.float64),
                               -0.05, 0.5)
    # decisions are compared where no prediction sits within rounding of the target
    clear = np.all(np.abs(y + 0.05) > 1e-4, axis=1)
    assert clear.sum() > 400
    np.testing.assert_array_equal(out[clear], ref[clear].astype(np.float32))
    # a non-finite prediction falls back
    bad = feats.copy()
    bad[0, 0] = np.nan
    assert net.select_theta(bad, grid, -0.05, fallback=0.5)[0] == np.float32(0.5)


def test_standardise_matches_oracle(M):
    rng = np.random.default_rng(9)
    net = M.ThetaNet(M.init_weights(8), mean=rng.normal(size=6), std=rng.uniform(0.2, 3.0, 6))
    x = rng.normal(size=(777, 6)).astype(np.float32) * 3
    got = net.scaled(x).cpu().numpy().astype(np.float64)
    ref = std_rows(net, x)
    assert np.all(np.abs(got - ref) <= 2.0 ** -22 * (np.abs(ref) + np.abs(x) / net.std + 1e-30))


def test_learned_theta_matches_oracle(M):
    # the whole selection from raw statistics: range check, standardisation,
    # budgeted targets (both exponents, a calibration), the choice
    rng = np.random.default_rng(10)
    g = 3000
    feats = np.column_stack([rng.uniform(6, 13, g), rng.normal(0.5, 0.2, g), rng.normal(1, 0.5, g),
                             rng.uniform(0, 1, g), rng.normal(-1.5, 0.5, g)]).astype(np.float32)
    count = rng.integers(1, 65, g).astype(np.int32)
    grid = np.round(np.arange(0.3, 1.61, 0.1), 2).astype(np.float32)
    net = M.ThetaNet(M.init_weights(11), mean=np.r_[feats.mean(0), 0.9], std=np.r_[feats.std(0), 0.4],
                     xmin=np.percentile(feats, 1, axis=0), xmax=np.percentile(feats, 99, axis=0), alpha=1.0 / 3,
                     beta=1.0 / 3, calib=1.2)
    feats[5, 2] = np.nan
    th, tg = net.learned_theta(feats, count, grid, 1e-3, theta0=0.5, fallback=0.55)
    wb = omlp.bf16_round(net.weights())
    ref, rtg = omlp.learned_theta(wb, net.mean, net.std, net.xmin, net.xmax, feats, count, grid.astype(np.float64),
                                  0.5, 1e-3, 1.2, 1.0 / 3, 1.0 / 3, 0.55)
    out = ~np.isfinite(rtg)
    assert out.sum() > 50 and th[5] == np.float32(0.55)
    np.testing.assert_array_equal(th[out], np.float32(0.55))
    assert np.all(np.isnan(tg[out]))
    assert np.abs(tg[~out] - rtg[~out]).max() <= 1e-5
    rows = np.concatenate([np.repeat(feats[~out], len(grid), 0), np.tile(grid, (~out).sum())[:, None]], 1)
    y = omlp.forward(wb, std_rows(net, rows)).reshape(-1, len(grid))
    clear = np.all(np.abs(y - rtg[~out][:, None]) > 1e-4, axis=1)
    assert clear.sum() > 0.9 * (~out).sum()
    np.testing.assert_array_equal(th[~out][clear], ref[~out][clear].astype(np.float32))
    # equal targets: every group in range aims at the target itself
    th2, tg2 = net.learned_theta(feats, count, grid, 1e-3, fallback=0.55, mode="equal")
    np.testing.assert_allclose(tg2[~out], -3.0, atol=1e-6)


def test_group_rms_error_matches_definition(M):
    import ctypes

    import torch
    rng = np.random.default_rng(12)
    sizes = rng.integers(1, 70, 300)
    off = np.r_[0, np.cumsum(sizes)].astype(np.int64)
    n = int(off[-1])
    ref = rng.normal(size=(n, 3))
    acc = ref * (1 + rng.normal(scale=1e-3, size=(n, 3)))
    acc[off[0]:off[1]] = ref[off[0]:off[1]]  # a group with no error floors at 1e-9
    d = torch.from_numpy(acc).cuda(), torch.from_numpy(ref).cuda(), torch.from_numpy(off).cuda()
    out = torch.empty(300, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.call("otoo_group_rms_error", d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), 300, 1e-9, out.data_ptr(),
           st.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    rel2 = (np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1)) ** 2
    want = np.log10(np.maximum(np.sqrt(np.add.reduceat(rel2, off[:-1]) / sizes), 1e-9))
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=1e-6)
    assert int(st.item()) == 0
