"""FP64 reference of the ranked-LoD helpers: per-Gaussian features, the
per-template ranking, and the 48-64-64-1 ranking MLP (forward, gradient,
Adam).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only the
tests, the smoke check and the benchmark's baseline legs use it.  Plain
numpy, one step per line of the definitions; nothing is shared with the
CUDA library.

The paper has no learned LoD (CrowdSplat Sec. 2 fits one template per
distance band); the definitions followed here are the library's own
(``include/crowdsplat_lod.h``): the feature list, the parameter layout, the
rounding points of the BF16 kernels, mean-squared error, and Adam as
published (Kingma and Ba, ICLR 2015, Algorithm 1, with bias correction).
Pinned by ``tests/test_oracle_lod_pins.py``.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_FEAT, N_BANDS = 48, 64, 32, 4
N_PARAMS = N_IN * N_H + N_H + N_H * N_H + N_H + N_H + 1


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

def unpack(p):
    """(W1 [48,64], b1 [64], W2 [64,64], b2 [64], w3 [64], b3) views of the
    flat parameter vector."""
    p = np.asarray(p, np.float64)
    assert p.shape == (N_PARAMS,)
    o = 0
    W1 = p[o:o + N_IN * N_H].reshape(N_IN, N_H); o += N_IN * N_H
    b1 = p[o:o + N_H]; o += N_H
    W2 = p[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = p[o:o + N_H]; o += N_H
    w3 = p[o:o + N_H]; o += N_H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


# ---------------------------------------------------------------------------
# BF16 rounding (round to nearest, ties to even, of the float32 value)
# ---------------------------------------------------------------------------

def bf16(x) -> np.ndarray:
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(x):
    return np.asarray(x, np.float64)


# ---------------------------------------------------------------------------
# the MLP
# ---------------------------------------------------------------------------

def inputs(feat, band) -> np.ndarray:
    """x [n, 48]: the 32 features, the one-hot band (bands outside 0..3: all
    zero), zeros."""
    feat = np.asarray(feat, np.float32).astype(np.float64)
    band = np.asarray(band, np.int64)
    n = feat.shape[0]
    x = np.zeros((n, N_IN))
    x[:, :N_FEAT] = feat
    ok = (band >= 0) & (band < N_BANDS)
    x[np.nonzero(ok)[0], N_FEAT + band[ok]] = 1.0
    return x


def forward(params, feat, band, rounding: bool = True):
    """Scores y [n] and the intermediate values.  rounding=True rounds to
    BF16 where the kernels do: x, W1, W2 and the first hidden activation."""
    r = bf16 if rounding else _ident
    W1, b1, W2, b2, w3, b3 = unpack(params)
    x = r(inputs(feat, band))
    W1r, W2r = r(W1), r(W2)
    z1 = x @ W1r + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2r + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, dict(x=x, W1r=W1r, W2r=W2r, z1=z1, h1=h1, z2=z2, h2=h2)


def loss_and_grad(params, feat, band, target, rounding: bool = True):
    """Mean squared error L = (1/n) sum (y - t)^2 and dL/dparams by the chain
    rule through the network (ReLU derivative 0 at 0).  rounding=True also
    rounds the back-propagated pre-activation gradients to BF16 where they
    enter a matrix product, as the kernels do."""
    r = bf16 if rounding else _ident
    W1, b1, W2, b2, w3, b3 = unpack(params)
    y, c = forward(params, feat, band, rounding)
    t = np.asarray(target, np.float32).astype(np.float64)
    n = y.shape[0]
    e = y - t
    L = float(np.mean(e * e))
    dy = 2.0 * e / n
    dw3 = c["h2"].T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, w3) * (c["z2"] > 0)
    db2 = dz2.sum(0)
    dz2r = r(dz2)
    dW2 = c["h1"].T @ dz2r
    dh1 = dz2r @ c["W2r"].T
    dz1 = dh1 * (c["z1"] > 0)
    db1 = dz1.sum(0)
    dW1 = c["x"].T @ r(dz1)
    return L, pack(dW1, db1, dW2, db2, dw3, db3)


def adam(params, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns new (params, m, v)."""
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# features and ranking
# ---------------------------------------------------------------------------

Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi))


def features(t) -> np.ndarray:
    """The 32 ranking features of every Gaussian of template t (attributes
    as uploaded: scales, quaternions, opacity, SH, skinning, rest joints,
    parents; or, when the template carries ``cov`` [n, 6], its canonical
    covariance instead of scales and quaternions), [n, 32] in FP64."""
    s = np.asarray(t.scales, np.float32).astype(np.float64)
    qt = np.asarray(t.quats, np.float32).astype(np.float64)
    o = np.asarray(t.opacity, np.float32).astype(np.float64)
    mu = np.asarray(t.means, np.float32).astype(np.float64)
    sh = np.asarray(t.sh, np.float32).astype(np.float64)
    w = np.asarray(t.skin_w, np.float32).astype(np.float64)
    idx = np.asarray(t.skin_idx).astype(np.int64)
    rest = np.asarray(t.rest_joints, np.float32).astype(np.float64)
    parents = np.asarray(t.parents)
    n = s.shape[0]
    f = np.zeros((n, N_FEAT))
    cov6 = getattr(t, "cov", None)
    if cov6 is not None:
        # covariance given directly: principal deviations from its eigenvalues
        c = np.asarray(cov6, np.float32).astype(np.float64).reshape(n, 6)
        Cg = np.stack([c[:, 0], c[:, 1], c[:, 2], c[:, 1], c[:, 3], c[:, 4], c[:, 2], c[:, 4], c[:, 5]], 1).reshape(n, 3, 3)
        ss = np.sqrt(np.maximum(np.linalg.eigvalsh(Cg)[:, ::-1], 1e-20))
    else:
        # principal standard deviations: the scales, largest first
        ss = -np.sort(-s, axis=1)
    ls = np.log(ss / 0.01)
    f[:, 0:3] = ls
    f[:, 3] = ls.mean(1)
    f[:, 4] = ls[:, 0] - ls[:, 2]
    f[:, 5] = o
    oc = np.clip(o, 1e-6, 1 - 1e-6)
    f[:, 6] = np.clip(np.log(oc / (1 - oc)) / 4.0, -2.0, 2.0)
    f[:, 7] = (np.log(np.maximum(o, 1e-12)) + ls[:, 0] + ls[:, 1]) / 4.0
    dc = np.maximum(0.0, Y00 * sh[:, 0, :] + 0.5)
    f[:, 8:11] = dc
    f[:, 11] = dc.mean(1)
    for l in (1, 2, 3):
        if l <= t.sh_degree:
            block = sh[:, l * l:(l + 1) * (l + 1), :]
            f[:, 11 + l] = np.sqrt(np.mean(block ** 2, axis=(1, 2))) / 0.3
    f[:, 15:18] = mu
    f[:, 18] = np.hypot(mu[:, 0] - rest[0, 0], mu[:, 2] - rest[0, 2])
    # skinning weights, largest first (stable for ties)
    order = np.argsort(-w, axis=1, kind="stable")
    ws = np.take_along_axis(w, order, 1)
    f[:, 19:23] = ws
    j0 = np.take_along_axis(idx, order[:, :1], 1)[:, 0]
    f[:, 23] = j0 / 23.0
    depth = np.zeros(len(parents), np.int64)
    for j in range(1, len(parents)):
        depth[j] = depth[parents[j]] + 1
    f[:, 24] = depth[j0] / depth.max() if depth.max() > 0 else 0.0
    f[:, 25] = 10.0 * np.linalg.norm(mu - rest[j0], axis=1)
    # covariance R diag(s^2) R^T from the normalised quaternion (or as given)
    if cov6 is not None:
        cov = Cg
    else:
        qn = qt / np.linalg.norm(qt, axis=1, keepdims=True)
        qw, qx, qy, qz = qn.T
        R = np.stack([1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                      2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                      2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)],
                     1).reshape(n, 3, 3)
        cov = np.einsum("nik,nk,njk->nij", R, s * s, R)
    tr = np.trace(cov, axis1=1, axis2=2)
    f[:, 26] = cov[:, 0, 0] / tr
    f[:, 27] = cov[:, 1, 1] / tr
    f[:, 28] = cov[:, 2, 2] / tr
    f[:, 29] = np.log(tr / 3e-4)
    f[:, 30] = o * ss[:, 0] / 0.01
    f[:, 31] = dc.max(1) - dc.min(1)
    return f


def targets(contrib, sizes, floor: float = 1e-3) -> np.ndarray:
    """ln(c / m + floor) per (band, Gaussian), m the mean of c over the
    Gaussian's template in that band.  contrib [n_bands, n_total]."""
    c = np.asarray(contrib, np.float32).astype(np.float64)
    out = np.empty_like(c)
    off = 0
    for n in sizes:
        seg = c[:, off:off + n]
        m = np.maximum(seg.mean(1, keepdims=True), 1e-30)
        out[:, off:off + n] = np.log(seg / m + floor)
        off += n
    return out


def rank(scores, sizes) -> np.ndarray:
    """Concatenated per-template orders: for each template (sizes in upload
    order), its local indices by descending score, ties by lower index."""
    scores = np.asarray(scores, np.float32)
    out, off = [], 0
    for n in sizes:
        seg = scores[off:off + n].astype(np.float64)
        out.append(np.lexsort((np.arange(n), -seg)).astype(np.uint32))
        off += n
    return np.concatenate(out) if out else np.zeros(0, np.uint32)
