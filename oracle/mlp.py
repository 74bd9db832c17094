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
