"""GPU parity of the ranked-LoD kernels through the C ABI: per-Gaussian
features, the per-template ranking sort, and the BF16 tensor-core MLP
(forward, gradient, Adam) against the FP64 reference in oracle/lod_ref.py."""
import math

import numpy as np
import pytest

from oracle import lod_ref as R
from paper_2501_17792_gb300 import scene as S
from tests.test_gpu_parity import built, make  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mlp(seed=0):
    from paper_2501_17792_gb300 import binding
    return binding.Mlp(device=0, seed=seed)


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (48, 64)) * math.sqrt(6 / 36) * scale
    W1[36:] = 0.0
    W2 = rng.uniform(-1, 1, (64, 64)) * math.sqrt(6 / 64) * scale
    p = R.pack(W1, rng.normal(0, 0.1, 64), W2, rng.normal(0, 0.1, 64),
               rng.uniform(-1, 1, 64) * math.sqrt(3 / 64), 0.05)
    return p.astype(np.float32)


def _batch(seed, n, bad_bands=False):
    rng = np.random.default_rng(seed)
    feat = rng.normal(0, 1, (n, 32)).astype(np.float32)
    band = rng.integers(0, 4, n).astype(np.int32)
    if bad_bands and n > 4:
        band[:2] = [-1, 5]
    target = rng.normal(0, 1, n).astype(np.float32)
    return feat, band, target


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _forward_bound(p, feat, band):
    """Per-row bound of |y_gpu - y_ref|: one BF16 step (2^-7 relative) in
    any first-layer activation, plus FP32 accumulation."""
    y, c = R.forward(p, feat, band, rounding=True)
    W1, b1, W2, b2, w3, b3 = R.unpack(p)
    flip = (2.0 ** -7) * (np.abs(c["h1"]) @ np.abs(c["W2r"])) @ np.abs(w3)
    fp32 = 1e-5 * ((np.abs(c["h1"]) @ np.abs(c["W2r"]) + np.abs(b2)) @ np.abs(w3) + abs(b3) + 1.0)
    return y, flip + fp32


def test_features_match_reference():
    tpls = [S.make_template(500 + t, 3000 + 517 * t, d) for t, d in enumerate((3, 1, 0))]
    sc = S.Scene(tpls, S.Instances(np.zeros(1, np.int32), np.tile(np.eye(3, 4, dtype=np.float32), (1, 1, 1)),
                                   np.zeros((1, 24, 3), np.float32)),
                 S.look_camera((0, 1, 0), 0, 32, 32), S.single_lod(), "features")
    r = make(sc)
    f = r.lod_features().cpu().numpy().astype(np.float64)
    ref = np.concatenate([R.features(t) for t in tpls])
    assert f.shape == ref.shape
    d = np.abs(f - ref)
    tol = 2e-5 + 2e-5 * np.abs(ref)
    worst = np.unravel_index(np.argmax(d / tol), d.shape)
    print(f"\n[features] n={f.shape[0]} max|d|={d.max():.2e} worst (row, feature)={worst}")
    assert np.all(d <= tol), (worst, f[worst], ref[worst])


def test_rank_matches_reference():
    sizes = [4096, 1000, 2500, 1]
    tpls = [S.make_template(600 + t, n, 0) for t, n in enumerate(sizes)]
    sc = S.Scene(tpls, S.Instances(np.zeros(1, np.int32), np.tile(np.eye(3, 4, dtype=np.float32), (1, 1, 1)),
                                   np.zeros((1, 24, 3), np.float32)),
                 S.look_camera((0, 1, 0), 0, 32, 32), S.single_lod(), "rank")
    r = make(sc)
    rng = np.random.default_rng(3)
    s = np.round(rng.normal(0, 1, sum(sizes)) * 8) / 8           # many ties
    s[:10] = [0.0, -0.0, 1e-30, -1e-30, 3.5, 3.5, -7.0, np.float32(1e30), -np.float32(1e30), 0.125]
    s = s.astype(np.float32)
    assert (np.signbit(s) & (s == 0)).sum() > 10      # -0.0 ties with 0.0
    o = r.lod_rank(_cuda(s)).cpu().numpy().view(np.uint32)
    ref = R.rank(s, sizes)
    assert np.array_equal(o, ref)


def test_targets_match_reference():
    sizes = [3000, 517, 4096]
    tpls = [S.make_template(700 + t, n, 0) for t, n in enumerate(sizes)]
    sc = S.Scene(tpls, S.Instances(np.zeros(1, np.int32), np.tile(np.eye(3, 4, dtype=np.float32), (1, 1, 1)),
                                   np.zeros((1, 24, 3), np.float32)),
                 S.look_camera((0, 1, 0), 0, 32, 32), S.single_lod(), "targets")
    r = make(sc)
    rng = np.random.default_rng(4)
    c = (rng.exponential(1.0, (3, sum(sizes))) * (rng.random((3, sum(sizes))) < 0.7)).astype(np.float32)
    c[2, :3000] = 0.0
    t = r.lod_targets(_cuda(c)).cpu().numpy().astype(np.float64)
    ref = R.targets(c, sizes)
    assert np.abs(t - ref).max() < 1e-5


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 40000])
def test_mlp_forward_matches_reference(n):
    m = _mlp()
    p = _params(1)
    m.set_params(p)
    assert np.array_equal(m.params(), p)
    feat, band, _ = _batch(2 + n, n, bad_bands=True)
    y = m.forward(_cuda(feat), _cuda(band)).cpu().numpy().astype(np.float64)
    ref, bound = _forward_bound(p.astype(np.float64), feat, band)
    d = np.abs(y - ref)
    print(f"\n[mlp forward n={n}] max|d|={d.max():.2e} median={np.median(d):.2e} max d/bound={np.max(d / bound):.3f}")
    assert np.all(d <= bound)
    assert np.median(d) <= 1e-4


def test_mlp_empty_and_errors():
    from paper_2501_17792_gb300 import binding
    m = _mlp()
    out = m.forward(torch.zeros((0, 32), device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert out.shape == (0,)
    feat, band, tgt = _batch(5, 10)
    with pytest.raises(binding.CrowdSplatError):
        m.train_step(_cuda(feat), _cuda(band), _cuda(tgt), lr=0.0)
    with pytest.raises(binding.CrowdSplatError):
        m.grad()  # before the first step
    bad = np.zeros(binding.MLP_PARAMS, np.float32)
    bad[7] = np.nan
    with pytest.raises(binding.CrowdSplatError):
        m.set_params(bad)


def test_mlp_gradient_and_adam_match_reference():
    m = _mlp()
    p = _params(7)
    m.set_params(p)
    feat, band, tgt = _batch(8, 3001, bad_bands=True)
    lr = 1e-3
    loss = m.train_step(_cuda(feat), _cuda(band), _cuda(tgt), lr)
    g = m.grad().astype(np.float64)
    L, gr = R.loss_and_grad(p.astype(np.float64), feat, band, tgt, rounding=True)
    assert abs(loss - L) <= 1e-4 * L
    blocks = dict(W1=(0, 3072), b1=(3072, 3136), W2=(3136, 7232), b2=(7232, 7296), w3=(7296, 7360), b3=(7360, 7361))
    for name, (a, b) in blocks.items():
        rel = np.linalg.norm(g[a:b] - gr[a:b]) / max(np.linalg.norm(gr[a:b]), 1e-30)
        print(f"[grad {name}] rel err {rel:.2e}")
        assert rel <= 2e-2, name
    assert np.all(g[36 * 64:48 * 64] == 0.0)         # padding inputs
    # Adam's first step moves each weight by about lr sign(g) where the
    # gradient is clearly non-zero
    q = m.params().astype(np.float64)
    qr, _, _ = R.adam(p.astype(np.float64), gr, np.zeros(R.N_PARAMS), np.zeros(R.N_PARAMS), 1, lr)
    err = np.abs(g - gr)
    sure = np.abs(gr) > 20 * np.maximum(err, 1e-7)
    assert sure.mean() > 0.5
    assert np.allclose(q[sure], qr[sure], rtol=0, atol=2e-6)


def test_mlp_training_fits_a_teacher():
    teacher = _params(11, scale=1.5).astype(np.float64)
    feat, band, _ = _batch(12, 8192)
    target, _ = R.forward(teacher, feat, band, rounding=False)
    m = _mlp(seed=5)
    f, b, t = _cuda(feat), _cuda(band), _cuda(target.astype(np.float32))
    L0 = m.train_step(f, b, t, 3e-3)
    for _ in range(400):
        m.train_step(f, b, t, 3e-3, want_loss=False)
    L1 = m.train_step(f, b, t, 3e-3)
    print(f"\n[mlp training] loss {L0:.4f} -> {L1:.4f}")
    assert L1 < L0 / 10
    # the trained weights predict through the reference too
    y_ref, _ = R.forward(m.params().astype(np.float64), feat, band, rounding=True)
    y = m.forward(f, b).cpu().numpy()
    assert np.mean((y_ref - target) ** 2) < L0 / 10
    assert np.abs(y - y_ref).max() < 0.05 * (np.abs(y_ref).max() + 1)
