"""FP64 reference of the learned bound proposer -- TEST INFRASTRUCTURE ONLY.

Plain numpy, float64, written from the network's definition (the paper has
no learned component; the definition is the project's):

    x_v   = [1, log1p(d_v)/8, log1p(a_v)/8, min(d_v/delta - 1, 8)/8,
             log1p(mean neighbour degree)/8, log1p(min neighbour degree)/8,
             q1_v, q2_v]
            d = weighted degree, a = number of neighbours, delta = min d,
            h = splitmix64(FEAT_SEED ^ splitmix64(v)),
            r1 = 2 U(h) - 1, r2 = 2 U(splitmix64(h)) - 1,
            U(h) = ((h >> 40) & (2^24 - 1)) / 2^24;
            q = r after SMOOTH steps of the lazy random walk
                s <- (s + D^-1 A s) / 2   (D^-1 A s = 0 where d = 0),
            centred by its degree-weighted mean (sum d s / sum d) and scaled
            by its largest magnitude (when that is > 0): a sparse cut's two
            sides drift apart under the walk while each side evens out
    h0    = ReLU(x W_in + b_in)
    g_l   = D^-1 A h_l
    h_l+1 = ReLU([h_l, g_l] W_l + b_l),  l = 0, 1, 2
    s     = h_3 w_out + b_out
    L     = min(sum BCE(p, y), sum BCE(p, 1 - y)) / n,  p = sigmoid(s)

The network's precision is part of its definition: with ``bf16=True`` the
dense weights W_l, the stored activations h_l and g_l, and the gradient
dZ_l entering the dense products are rounded to BF16 (round to nearest
even) where the CUDA kernels round them; every sum is exact otherwise
(float64 here, float32 on the GPU).  ``bf16=False`` is the unrounded network,
whose analytic gradient `numeric_grad` (central differences) pins.

Parameter vector layout (floats): W_in (8 x 64 row-major), b_in (64), then
for each layer W_l (128 x 64 row-major) and b_l (64), then w_out (64), b_out.

Only the test-suite may import this module.
"""
from __future__ import annotations

import numpy as np

import oracle

F, H, L, K = 8, 64, 3, 128
P_WIN, P_BIN = 0, 8 * 64
P_W0 = P_BIN + 64
P_LAYER = K * H + H
P_WOUT = P_W0 + L * P_LAYER
P_BOUT = P_WOUT + H
P_TOTAL = P_BOUT + 1
FEAT_SEED = 0x51ED270B27A4BB1D
SMOOTH = 32
EPS = 1e-7


def bf16(x):
    """Round to the nearest BF16 value (ties to even), via float32."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _canon(rp, col, w):
    """Canonical graph (parallel arcs summed, no self-loops), via the oracle's
    contraction with identity labels."""
    n = len(rp) - 1
    crp, ccol, cw = oracle.contract(rp, col, w, np.arange(n, dtype=np.int32), n)
    return n, crp.astype(np.int64), ccol.astype(np.int64), cw.astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    W_in = p[P_WIN:P_WIN + F * H].reshape(F, H)
    b_in = p[P_BIN:P_BIN + H]
    layers = []
    for l in range(L):
        o = P_W0 + l * P_LAYER
        layers.append((p[o:o + K * H].reshape(K, H), p[o + K * H:o + K * H + H]))
    return W_in, b_in, layers, p[P_WOUT:P_WOUT + H], p[P_BOUT]


def features(rp, col, w):
    n, crp, ccol, cw = _canon(rp, col, w)
    src = np.repeat(np.arange(n), np.diff(crp))
    d = np.zeros(n)
    np.add.at(d, src, cw)
    a = np.diff(crp).astype(np.float64)
    delta = d.min()
    X = np.zeros((n, F))
    X[:, 0] = 1.0
    X[:, 1] = np.log1p(d) / 8
    X[:, 2] = np.log1p(a) / 8
    rel = d / delta - 1.0 if delta > 0 else np.zeros(n)
    X[:, 3] = np.minimum(rel, 8.0) / 8
    nbr = d[ccol]
    ssum = np.zeros(n)
    np.add.at(ssum, src, nbr)
    mn = np.full(n, np.inf)
    np.minimum.at(mn, src, nbr)
    X[:, 4] = np.log1p(np.where(a > 0, ssum / np.maximum(a, 1), 0.0)) / 8
    X[:, 5] = np.log1p(np.where(a > 0, mn, 0.0)) / 8
    R = np.zeros((n, 2))
    for v in range(n):
        h = oracle.splitmix64(FEAT_SEED ^ oracle.splitmix64(v))
        h2 = oracle.splitmix64(h)
        R[v, 0] = 2 * (((h >> 40) & 0xFFFFFF) / 16777216.0) - 1
        R[v, 1] = 2 * (((h2 >> 40) & 0xFFFFFF) / 16777216.0) - 1
    G = (n, crp, ccol, cw, src, d)
    for _ in range(SMOOTH):
        R = (R + _aggregate(G, R)) / 2
    if d.sum() > 0:
        R = R - (d @ R) / d.sum()
    for j in range(2):
        mx = np.abs(R[:, j]).max() if n else 0.0
        if mx > 0:
            R[:, j] /= mx
    X[:, 6:8] = R
    return X, G


def _aggregate(G, h):
    n, crp, ccol, cw, src, d = G
    out = np.zeros_like(h)
    np.add.at(out, src, cw[:, None] * h[ccol])
    return out / np.where(d > 0, d, 1.0)[:, None]


def _aggregate_t(G, dg):
    # transpose of D^-1 A: out[u] = sum_v (w_uv / d_v) dg[v]
    n, crp, ccol, cw, src, d = G
    out = np.zeros_like(dg)
    coef = cw / np.where(d[ccol] > 0, d[ccol], 1.0)
    np.add.at(out, src, coef[:, None] * dg[ccol])
    return out


def forward(params, rp, col, w, bf16_round=False):
    X, G = features(rp, col, w)
    rnd = bf16 if bf16_round else (lambda x: x)
    W_in, b_in, layers, w_out, b_out = unpack(params)
    Z0 = X @ W_in + b_in
    hs, gs, zs = [rnd(np.maximum(Z0, 0))], [], [Z0]
    for W, b in layers:
        g = rnd(_aggregate(G, hs[-1]))
        z = np.concatenate([hs[-1], g], axis=1) @ rnd(W) + b
        gs.append(g)
        zs.append(z)
        hs.append(rnd(np.maximum(z, 0)))
    s = hs[-1] @ w_out + b_out
    return s, (X, G, hs, gs, zs)


def _bce(p, y):
    p = np.clip(p, EPS, 1 - EPS)
    return np.where(y == 1, -np.log(p), -np.log(1 - p))


def loss_and_grad(params, rp, col, w, side, bf16_round=False):
    side = np.asarray(side, dtype=np.int64)
    s, (X, G, hs, gs, zs) = forward(params, rp, col, w, bf16_round)
    rnd = bf16 if bf16_round else (lambda x: x)
    n = len(s)
    p = 1 / (1 + np.exp(-s))
    l0, l1 = _bce(p, side).sum(), _bce(p, 1 - side).sum()
    y = side if l0 <= l1 else 1 - side
    loss = min(l0, l1) / n
    W_in, b_in, layers, w_out, b_out = unpack(params)
    grad = np.zeros(P_TOTAL)
    ds = (p - y) / n  # clip is inactive away from p in {0, 1}
    grad[P_WOUT:P_WOUT + H] = hs[-1].T @ ds
    grad[P_BOUT] = ds.sum()
    dh = np.outer(ds, w_out)
    for l in range(L - 1, -1, -1):
        W, b = layers[l]
        dz = dh * (zs[l + 1] > 0)
        dzr = rnd(dz)
        Xl = np.concatenate([hs[l], gs[l]], axis=1)
        o = P_W0 + l * P_LAYER
        grad[o:o + K * H] = (Xl.T @ dzr).reshape(-1)
        grad[o + K * H:o + K * H + H] = dz.sum(axis=0)
        dX = dzr @ rnd(W).T
        dh = dX[:, :H] + _aggregate_t(G, dX[:, H:])
    dz0 = dh * (zs[0] > 0)
    grad[P_WIN:P_WIN + F * H] = (X.T @ dz0).reshape(-1)
    grad[P_BIN:P_BIN + H] = dz0.sum(axis=0)
    return loss, grad


def loss_only(params, rp, col, w, side):
    side = np.asarray(side, dtype=np.int64)
    s, _ = forward(params, rp, col, w)
    p = 1 / (1 + np.exp(-s))
    return min(_bce(p, side).sum(), _bce(p, 1 - side).sum()) / len(s)


def numeric_grad(params, rp, col, w, side, idx, h=1e-6):
    params = np.asarray(params, dtype=np.float64).copy()
    out = []
    for i in idx:
        old = params[i]
        params[i] = old + h
        lp = loss_only(params, rp, col, w, side)
        params[i] = old - h
        lm = loss_only(params, rp, col, w, side)
        params[i] = old
        out.append((lp - lm) / (2 * h))
    return np.array(out)


def glorot(seed: int) -> np.ndarray:
    """A float64 parameter vector with Glorot-uniform weights (for tests)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(P_TOTAL)

    def fill(off, fi, fo):
        a = np.sqrt(6.0 / (fi + fo))
        p[off:off + fi * fo] = rng.uniform(-a, a, size=fi * fo)
    fill(P_WIN, F, H)
    for l in range(L):
        fill(P_W0 + l * P_LAYER, K, H)
        p[P_W0 + l * P_LAYER + K * H:P_W0 + (l + 1) * P_LAYER] = rng.uniform(-0.1, 0.1, H)
    fill(P_WOUT, H, 1)
    p[P_BIN:P_BIN + H] = rng.uniform(-0.1, 0.1, H)
    return p
