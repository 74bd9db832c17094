"""Device-side perceptron for the learned opening angle (argument
marshalling over the otoo_mlp_* and otoo_learned_theta C ABI; the
arithmetic runs in mlp.cu).

ThetaNet holds FP32 master weights, their bf16 copy and the Adam moments as
device tensors, with the input statistics of its training rows (mean, std,
the range of the list statistics) and the selection rule's constants
(budget exponents, calibration).  Rows are standardised on the device."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

NP = L.MLP_NPARAM
NI = L.MLP_IN


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def init_weights(seed=0):
    """Glorot-uniform weights, zero biases (FP32 master copy)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.zeros(NP, np.float32)
    o = 0
    for fan_in, fan_out in ((NI, 32), (32, 32), (32, 1)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        w[o:o + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
        o += fan_in * fan_out + fan_out
    return w


class ThetaNet:
    def __init__(self, w=None, device="cuda", mean=None, std=None, xmin=None, xmax=None, alpha=1.0 / 3.0,
                 beta=1.0 / 3.0, calib=1.0, theta0=0.9, grid=None):
        import torch
        self.device = device
        w = init_weights() if w is None else np.asarray(w, np.float32)
        self.w = torch.tensor(w, dtype=torch.float32, device=device)
        self.wbf16 = torch.empty(NP, dtype=torch.int16, device=device)
        self.m = torch.zeros(NP, dtype=torch.float32, device=device)
        self.v = torch.zeros(NP, dtype=torch.float32, device=device)
        self.t = 0
        self.mean = np.zeros(NI, np.float32) if mean is None else np.asarray(mean, np.float32)
        self.std = np.ones(NI, np.float32) if std is None else np.asarray(std, np.float32)
        self.xmin = None if xmin is None else np.asarray(xmin, np.float32)
        self.xmax = None if xmax is None else np.asarray(xmax, np.float32)
        self.alpha, self.beta, self.calib = float(alpha), float(beta), float(calib)
        # the base walk's angle and the angle grid the network was trained on
        self.theta0 = float(theta0)
        self.grid = None if grid is None else tuple(float(g) for g in grid)
        L.call("otoo_mlp_to_bf16", _vp(self.w), _vp(self.wbf16), NP, _stream(device))

    def fit_scaler(self, x):
        """Input statistics of the training rows (the range of the list
        statistics too: selection falls back outside it)."""
        x = np.asarray(x, np.float32)
        self.mean = x.mean(0).astype(np.float32)
        self.std = np.maximum(x.std(0), 1e-6).astype(np.float32)
        self.xmin = x[:, :NI - 1].min(0)
        self.xmax = x[:, :NI - 1].max(0)

    def _dev(self, a):
        import torch
        return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(self.device)

    def scaled(self, x):
        """Rows x [n][6] (host) standardised on the device."""
        xs = self._dev(x)
        n = xs.shape[0]
        # device copies of the statistics held until the launch is enqueued
        # (freed earlier, their memory could be handed to the next copy)
        mean, std = self._dev(self.mean), self._dev(self.std)
        L.call("otoo_mlp_standardise", _vp(xs), n, _vp(mean), _vp(std), _vp(xs), _stream(self.device))
        return xs

    def predict_scaled(self, xs_dev):
        import torch
        n = xs_dev.shape[0]
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        L.call("otoo_mlp_predict", _vp(self.wbf16), _vp(xs_dev), _vp(y), n, _stream(self.device))
        return y

    def predict(self, x):
        return self.predict_scaled(self.scaled(x)).cpu().numpy()

    def grad(self, x, t):
        import torch
        xs, ts = self.scaled(x), self._dev(t)
        n = xs.shape[0]
        scratch = torch.empty(int(L.load().otoo_mlp_scratch_floats(n)), dtype=torch.float32, device=self.device)
        g = torch.empty(NP, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        L.call("otoo_mlp_grad", _vp(self.wbf16), _vp(xs), _vp(ts), n, _vp(scratch), _vp(g), _vp(loss),
               _stream(self.device))
        return g.cpu().numpy(), float(loss.item())

    def train(self, x, t, steps, lr=3e-3, batch=None, seed=0, b1=0.9, b2=0.999, eps=1e-8, log_every=0):
        """Adam on (standardised x, t); full batch unless batch is set.
        Returns the loss history (one value per logged step)."""
        import torch
        xs, ts = self.scaled(x), self._dev(t)
        n = xs.shape[0]
        nb = n if batch is None else min(batch, n)
        scratch = torch.empty(int(L.load().otoo_mlp_scratch_floats(nb)), dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        rng = np.random.Generator(np.random.PCG64(seed))
        hist = []
        st = _stream(self.device)
        for k in range(steps):
            if nb < n:
                sel = torch.from_numpy(rng.choice(n, nb, replace=False)).to(self.device)
                xb, tb = xs.index_select(0, sel).contiguous(), ts.index_select(0, sel).contiguous()
            else:
                xb, tb = xs, ts
            self.t += 1
            L.call("otoo_mlp_train_step", _vp(self.w), _vp(self.wbf16), _vp(self.m), _vp(self.v), _vp(scratch),
                   _vp(xb), _vp(tb), nb, lr, b1, b2, eps, self.t, _vp(loss), st)
            if log_every and (k % log_every == 0 or k == steps - 1):
                hist.append(float(loss.item()))
        return hist

    def select_theta(self, feats, grid, log10_target, fallback=0.5, log10_target_per_group=None):
        """otoo_select_theta: feats [g][5] (list statistics); rows (g, k) =
        feats[g] + grid[k], standardised on the device."""
        import torch
        g = feats.shape[0]
        k = len(grid)
        rows = np.concatenate([np.repeat(feats, k, axis=0), np.tile(np.asarray(grid, np.float32), g)[:, None]], 1)
        xs = self.scaled(rows)
        gd = self._dev(np.asarray(grid, np.float32))
        tg = None if log10_target_per_group is None else self._dev(log10_target_per_group)
        out = torch.empty(g, dtype=torch.float32, device=self.device)
        L.call("otoo_select_theta", _vp(self.wbf16), _vp(xs), _vp(gd), k, g, float(log10_target),
               _vp(tg) if tg is not None else None, float(fallback), _vp(out), _stream(self.device))
        return out.cpu().numpy()

    def learned_theta(self, feats, count, grid, target_rms, theta0=0.5, fallback=0.5, mode="budget"):
        """otoo_learned_theta: one angle per group from its raw list
        statistics feats [g][5] (base walk at theta0) and particle count;
        mode "budget" uses the network's exponents and calibration, "equal"
        aims every group at target_rms.  Returns (angles, log10 targets)."""
        import torch
        g = int(feats.shape[0])
        net = L.ThetaNet()
        keep = [self._dev(self.mean), self._dev(self.std)]
        net.wbf16, net.mean, net.std = self.wbf16.data_ptr(), keep[0].data_ptr(), keep[1].data_ptr()
        if self.xmin is not None:
            keep += [self._dev(self.xmin), self._dev(self.xmax)]
            net.lo, net.hi = keep[2].data_ptr(), keep[3].data_ptr()
        rule = L.ThetaRule(theta0=float(theta0), target_rms=float(target_rms),
                           calib=self.calib if mode == "budget" else 1.0,
                           alpha=self.alpha if mode == "budget" else 0.0, beta=self.beta if mode == "budget" else 0.0,
                           fallback=float(fallback))
        f = self._dev(feats)
        c = torch.from_numpy(np.ascontiguousarray(count, np.int32)).to(self.device)
        gd = self._dev(np.asarray(grid, np.float32))
        scratch = torch.empty(max(int(L.load().otoo_learned_theta_scratch_floats(g)), 2), dtype=torch.float32,
                              device=self.device)
        tg = torch.empty(max(g, 1), dtype=torch.float32, device=self.device)
        out = torch.empty(max(g, 1), dtype=torch.float32, device=self.device)
        L.call("otoo_learned_theta", ctypes.byref(net), ctypes.byref(rule), _vp(f), _vp(c), g, _vp(gd), len(grid),
               _vp(scratch), _vp(tg), _vp(out), _stream(self.device))
        return out[:g].cpu().numpy(), tg[:g].cpu().numpy()

    def weights(self):
        return self.w.cpu().numpy()

    def weights_bf16(self):
        return self.wbf16.cpu().numpy().view(np.uint16)

    def save(self, path):
        extra = {}
        if self.xmin is not None:
            extra = dict(xmin=self.xmin, xmax=self.xmax)
        if self.grid is not None:
            extra["grid"] = np.asarray(self.grid, np.float32)
        np.savez(path, w=self.weights(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(), t=self.t,
                 mean=self.mean, std=self.std, alpha=self.alpha, beta=self.beta, calib=self.calib,
                 theta0=self.theta0, **extra)

    @classmethod
    def load(cls, path, device="cuda"):
        d = np.load(path)
        rule = {k: float(d[k]) for k in ("alpha", "beta", "calib", "theta0") if k in d}
        net = cls(d["w"], device, d["mean"], d["std"], d["xmin"][:NI - 1] if "xmin" in d else None,
                  d["xmax"][:NI - 1] if "xmax" in d else None, grid=d["grid"] if "grid" in d else None, **rule)
        import torch
        net.m = torch.tensor(d["m"], device=device)
        net.v = torch.tensor(d["v"], device=device)
        net.t = int(d["t"])
        return net
