"""FP64 reference of the 6-32-32-1 perceptron (tanh, tanh, linear), its
loss gradient and the Adam update.  TEST INFRASTRUCTURE ONLY.

Parameter vector layout (1313 values): W1 [32][6], b1 [32], W2 [32][32],
b2 [32], w3 [32], b3.  Loss: mean squared residual.  Adam: Kingma & Ba,
"Adam: A Method for Stochastic Optimization", ICLR 2015 (Algorithm 1, bias
corrected).  The gradient is written out by the chain rule, one layer at a
time; it is pinned against central finite differences in the tests.
"""
import numpy as np

NI, NH = 6, 32
NP = NH * NI + NH + NH * NH + NH + NH + 1


def unpack(w):
    w = np.asarray(w, np.float64)
    o = 0
    W1 = w[o:o + NH * NI].reshape(NH, NI); o += NH * NI
    b1 = w[o:o + NH]; o += NH
    W2 = w[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = w[o:o + NH]; o += NH
    w3 = w[o:o + NH]; o += NH
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def forward(w, x):
    """y [n] for rows x [n][6]."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    x = np.asarray(x, np.float64)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss(w, x, t):
    r = forward(w, x) - np.asarray(t, np.float64)
    return float(np.mean(r * r))


def grad(w, x, t):
    """d loss / d w by the chain rule (layer by layer)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    x = np.asarray(x, np.float64)
    n = x.shape[0]
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ w3 + b3
    dy = 2.0 * (y - np.asarray(t, np.float64)) / n          # d loss / d y
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, w3) * (1.0 - h2 * h2)                 # d loss / d z2
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)                        # d loss / d z1
    g_W1 = d1.T @ x
    g_b1 = d1.sum(0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


def adam(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step; returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(w):
    """Round FP32 values to the nearest bf16 (ties to even), returned as FP64."""
    a = np.asarray(w, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def choose_theta(y, grid, log10_target, fallback):
    """Per group g (row of the prediction table y [g][k], one column per grid
    angle, grid increasing): the largest grid[k] whose prediction y[g, k] is
    at most the group's target (a prediction equal to the target passes);
    grid[0] when no angle passes; fallback when any of the group's
    predictions is not finite.  log10_target: one value or one per group."""
    y = np.asarray(y, np.float64)
    g, k = y.shape
    tg = np.broadcast_to(np.asarray(log10_target, np.float64), (g,))
    out = np.empty(g, np.float64)
    for a in range(g):
        if not np.all(np.isfinite(y[a])):
            out[a] = fallback
            continue
        passing = [grid[j] for j in range(k) if y[a, j] <= tg[a]]
        out[a] = max(passing) if passing else grid[0]
    return out


def select_theta(w, feats, grid, log10_target, fallback):
    """choose_theta on the network's predictions for rows feats [g][k][6]
    (group g's features with angle grid[k]); returns (angles, predictions)."""
    g, k, _ = feats.shape
    y = forward(w, feats.reshape(g * k, NI)).reshape(g, k)
    return choose_theta(y, grid, log10_target, fallback), y


def budget_targets(y0, log2_len, count, target_rms, alpha, beta):
    """Per-group error targets e_g = lambda w_g with w_g = 10^(alpha y0_g +
    beta log10 L_g) (y0: predicted log10 error at theta0, L = 2^log2_len the
    list length at theta0) and lambda fixing the particle-weighted RMS of
    the targets: sum_g n_g e_g^2 / sum_g n_g = target_rms^2.  Returns
    log10 e_g.  (With a group error c theta^k and a list length a theta^-3,
    minimising sum n a theta^-3 at fixed sum n c^2 theta^(2k) gives
    e ~ c^(3/(2k+3)) a^(k/(2k+3)): alpha = 3/(2k+3), beta = k/(2k+3).)"""
    y0 = np.asarray(y0, np.float64)
    n = np.asarray(count, np.float64)
    w = 10.0 ** (alpha * y0 + beta * np.asarray(log2_len, np.float64) * np.log10(2.0))
    lam = target_rms / np.sqrt(np.sum(n * w * w) / np.sum(n))
    return np.log10(lam * w)


def learned_theta(w, mean, std, lo, hi, feats, count, grid, theta0, target_rms, calib, alpha, beta, fallback):
    """The learned per-group angle from raw list statistics feats [g][5]:
    groups with a non-finite statistic or one outside [lo, hi] take the
    fallback; the others get budget_targets (aimed at calib * target_rms,
    from the prediction at theta0 on the standardised row (x - mean) / std)
    and choose_theta over the grid (a non-finite prediction: fallback).
    Returns (angles, log10 targets with NaN where out of range)."""
    f = np.asarray(feats, np.float64)
    g = f.shape[0]
    ok = np.all(np.isfinite(f), axis=1)
    if lo is not None:
        ok &= np.all((f >= np.asarray(lo, np.float64)) & (f <= np.asarray(hi, np.float64)), axis=1)
    mean = np.asarray(mean, np.float64)
    std = np.asarray(std, np.float64)

    def rows(th):
        return (np.concatenate([f, np.full((g, 1), th)], 1) - mean) / std

    y0 = forward(w, rows(theta0))
    ok &= np.isfinite(y0)
    out = np.full(g, fallback, np.float64)
    tg = np.full(g, np.nan)
    if ok.any():
        tg[ok] = budget_targets(y0[ok], f[ok, 0], np.asarray(count)[ok], calib * target_rms, alpha, beta)
        y = np.stack([forward(w, rows(th))[ok] for th in grid], 1)
        out[ok] = choose_theta(y, grid, tg[ok], fallback)
    return out, tg
