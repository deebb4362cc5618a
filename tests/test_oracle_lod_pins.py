"""Pins of the ranked-LoD reference (oracle/lod_ref.py): finite differences,
closed forms, library routines and properties.  CPU only."""
import math

import numpy as np
import pytest

from oracle import lod_ref as R
from paper_2501_17792_gb300 import scene as S
from tests import scene_util as U


def _random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (48, 64)) * math.sqrt(6 / 36) * scale
    W1[36:] = 0.0
    W2 = rng.uniform(-1, 1, (64, 64)) * math.sqrt(6 / 64) * scale
    return R.pack(W1, rng.normal(0, 0.1, 64), W2, rng.normal(0, 0.1, 64),
                  rng.uniform(-1, 1, 64) * math.sqrt(3 / 64), 0.05)


def _random_batch(seed, n):
    rng = np.random.default_rng(seed)
    feat = rng.normal(0, 1, (n, 32)).astype(np.float32)
    band = rng.integers(0, 4, n)
    target = rng.normal(0, 1, n).astype(np.float32)
    return feat, band, target


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000) * 1e-30,
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -1 - 2 ** -8, 3 * 2 ** -8 + 1, 0.0, -0.0]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(R.bf16(x), ref)
    assert R.bf16([1 + 2 ** -8])[0] == 1.0            # tie to even
    assert R.bf16([1 + 3 * 2 ** -8])[0] == 1 + 2 ** -6  # tie to even (upwards)


def test_gradient_matches_central_differences():
    p = _random_params(2)
    feat, band, target = _random_batch(3, 40)
    L, g = R.loss_and_grad(p, feat, band, target, rounding=False)
    rng = np.random.default_rng(4)
    # a sample of every block: W1 (live rows), b1, W2, b2, w3, b3
    idx = np.concatenate([rng.choice(36 * 64, 60, replace=False), 3072 + rng.choice(64, 10, replace=False),
                          3136 + rng.choice(4096, 60, replace=False), 7232 + rng.choice(64, 10, replace=False),
                          7296 + rng.choice(64, 10, replace=False), [7360]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (R.loss_and_grad(p + e, feat, band, target, False)[0] -
              R.loss_and_grad(p - e, feat, band, target, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])
    # padding rows of W1 see zero input
    assert np.all(g[36 * 64:48 * 64] == 0.0)


def test_permutation_network_closed_form():
    """W1, W2 permutation embeddings, zero biases, non-negative inputs:
    y = sum_j w3[j] x[pi(j)] + b3 (exact in BF16 for dyadic inputs)."""
    rng = np.random.default_rng(5)
    p1 = rng.permutation(64)          # hidden unit k <- input p1[k] (inputs 0..47 only)
    W1 = np.zeros((48, 64))
    for k in range(64):
        if p1[k] < 36:
            W1[p1[k], k] = 1.0
    p2 = rng.permutation(64)
    W2 = np.zeros((64, 64))
    W2[p2, np.arange(64)] = 1.0       # unit j of layer 2 copies unit p2[j] of layer 1
    w3 = rng.integers(-8, 9, 64) / 8.0
    params = R.pack(W1, np.zeros(64), W2, np.zeros(64), w3, 0.25)
    feat = (rng.integers(0, 64, (20, 32)) / 64.0).astype(np.float32)
    band = rng.integers(0, 4, 20)
    x = R.inputs(feat, band)
    want = np.zeros(20)
    for j in range(64):
        src = p1[p2[j]]
        if src < 36:
            want += w3[j] * x[:, src]
    want += 0.25
    for rounding in (False, True):
        y, _ = R.forward(params, feat, band, rounding)
        assert np.array_equal(y, want)


def test_inputs_one_hot_and_padding():
    feat = np.arange(64, dtype=np.float32).reshape(2, 32)
    x = R.inputs(feat, [2, 7])
    assert np.array_equal(x[:, :32], feat)
    assert list(x[0, 32:36]) == [0, 0, 1, 0] and np.all(x[1, 32:] == 0) and np.all(x[:, 36:] == 0)


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(6)
    p = rng.normal(0, 1, R.N_PARAMS)
    g = rng.normal(0, 1, R.N_PARAMS) * 10.0 ** rng.uniform(-6, 1, R.N_PARAMS)
    g[:5] = 0.0
    q, m, v = R.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    assert np.allclose(q - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
    assert np.all(q[:5] == p[:5])
    # constant gradient: every step moves by lr g/(|g| + eps) (bias correction)
    for t in range(2, 6):
        q2, m, v = R.adam(q, g, m, v, t, 1e-3)
        assert np.allclose(q2 - q, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-6, atol=1e-12)
        q = q2


def test_training_fits_a_teacher_network():
    teacher = _random_params(7, scale=1.5)
    feat, band, _ = _random_batch(8, 512)
    target, _ = R.forward(teacher, feat, band, rounding=False)
    p = _random_params(9)
    m = v = np.zeros_like(p)
    L0 = R.loss_and_grad(p, feat, band, target, False)[0]
    for t in range(1, 401):
        L, g = R.loss_and_grad(p, feat, band, target, False)
        p, m, v = R.adam(p, g, m, v, t, 3e-3)
    L1 = R.loss_and_grad(p, feat, band, target, False)[0]
    assert L1 < L0 / 10, (L0, L1)


def test_rounded_gradient_is_close_to_exact():
    p = _random_params(10)
    feat, band, target = _random_batch(11, 300)
    _, ge = R.loss_and_grad(p, feat, band, target, rounding=False)
    _, gr = R.loss_and_grad(p, feat, band, target, rounding=True)
    # BF16 keeps 8 significant bits: relative error of a few 2^-8 per block
    for a, b in ((0, 3072), (3136, 7232), (7296, 7360)):
        assert np.linalg.norm(gr[a:b] - ge[a:b]) <= 0.05 * np.linalg.norm(ge[a:b])


def test_features_closed_forms():
    # axis-aligned Gaussian: principal sigmas are the scales
    t = U.template_from([[0.1, 1.0, 0.2]], [[0.005, 0.02, 0.01]], [[1, 0, 0, 0]], [0.8],
                        np.full((1, 4, 3), 0.3, np.float32), skin_idx=[[3, 0, 5, 1]],
                        skin_w=[[0.2, 0.5, 0.25, 0.05]])
    f = R.features(t)[0]
    s = np.array([0.02, 0.01, 0.005], np.float32).astype(np.float64)
    assert np.allclose(f[0:3], np.log(s / 0.01), atol=1e-12)
    assert np.isclose(f[4], math.log(4.0))
    assert np.isclose(f[5], np.float32(0.8)) and np.isclose(f[6], math.log(np.float32(0.8) / (1 - np.float32(0.8))) / 4)
    dc = max(0.0, R.Y00 * np.float32(0.3) + 0.5)
    assert np.allclose(f[8:11], dc) and np.isclose(f[31], 0.0)
    assert np.isclose(f[12], np.float32(0.3) / 0.3)       # degree 1 rms
    assert f[13] == 0.0 and f[14] == 0.0                   # degree 1 template
    assert np.allclose(f[19:23], np.float32([0.5, 0.25, 0.2, 0.05]))
    assert np.isclose(f[23], 0 / 23.0)                     # joint 0 carries the largest weight
    var = np.array([0.005, 0.02, 0.01], np.float32).astype(np.float64) ** 2
    assert np.allclose(f[26:29], var / var.sum())
    assert np.isclose(f[29], math.log(var.sum() / 3e-4))
    # a rotation about y swaps the x and z variances, keeps the sigmas
    c = math.cos(math.pi / 4)
    t2 = U.template_from([[0.1, 1.0, 0.2]], [[0.005, 0.02, 0.01]], [[c, 0, c, 0]], [0.8],
                         np.full((1, 4, 3), 0.3, np.float32))
    f2 = R.features(t2)[0]
    assert np.allclose(f2[0:3], f[0:3]) and np.allclose(f2[[26, 27, 28]], f[[28, 27, 26]], atol=1e-7)


def test_features_of_generated_template_are_finite_and_scaled():
    t = S.make_template(77, 2000, 3)
    f = R.features(t)
    assert f.shape == (2000, 32) and np.isfinite(f).all()
    assert np.all(f[:, 0] >= f[:, 1]) and np.all(f[:, 1] >= f[:, 2])
    assert np.all(np.abs(f[:, 26:29].sum(1) - 1) < 1e-12)
    assert np.all((f[:, 24] >= 0) & (f[:, 24] <= 1))


def test_rank_orders_by_descending_score_with_index_ties():
    s = np.array([0.5, 2.0, 0.5, -1.0, 3.0, 3.0, 0.0], np.float32)
    o = R.rank(s, [4, 3])
    assert list(o[:4]) == [1, 0, 2, 3]
    assert list(o[4:]) == [0, 1, 2]


def test_targets_closed_form():
    c = np.array([[1.0, 3.0, 0.0, 2.0, 2.0], [0.0, 0.0, 0.0, 5.0, 1.0]], np.float32)
    t = R.targets(c, [3, 2], floor=1e-3)
    assert np.allclose(t[0, :3], np.log(np.array([0.75, 2.25, 0.0]) + 1e-3))
    assert np.allclose(t[0, 3:], np.log(1.0 + 1e-3))
    assert np.allclose(t[1, :3], np.log(1e-3))                    # a template that never contributed
    assert np.allclose(t[1, 3:], np.log(np.array([5 / 3, 1 / 3]) + 1e-3))


def test_features_from_a_direct_covariance_match_scales():
    import dataclasses
    t = S.make_template(78, 500, 1)
    q = t.quats.astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    import oracle as O
    Rq = np.stack([O.quat_to_rot(x) for x in q])
    C = np.einsum("nik,nk,njk->nij", Rq, t.scales.astype(np.float64) ** 2, Rq)
    t2 = dataclasses.replace(t)
    t2.cov = np.stack([C[:, 0, 0], C[:, 0, 1], C[:, 0, 2], C[:, 1, 1], C[:, 1, 2], C[:, 2, 2]], 1).astype(np.float32)
    a, b = R.features(t), R.features(t2)
    assert np.abs(a - b).max() < 1e-4
