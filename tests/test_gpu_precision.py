"""GPU tests of the precision variant (CS_STORE_BF16): BF16 template
attributes, FP16 SH, the skinning blend as a split-BF16 tensor-core product.

Parity: the oracle is fed the attributes exactly as the library stores them
(rounded here the same way), so the same image tolerances as the FP32 path
apply.  Precision cost: the same frames against the oracle on the original
FP32 attributes, reported as per-pixel error, PSNR and the mean 3D position
error of the posed Gaussians (m)."""
import dataclasses

import numpy as np
import pytest

import oracle
from oracle import lod_ref as R
from paper_2501_17792_gb300 import scene as S
from tests import parity_util as PU
from tests.test_gpu_parity import built, make, render  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BF16 = 1  # CS_STORE_BF16


def quantized(t):
    """The template as the BF16 storage holds it: the skinning slot of the
    joint nearest to the mean first, the mean as that joint's rest position
    plus a BF16 offset (added in FP32), BF16 opacity and canonical
    covariance (FP64 -> FP32 -> BF16), BF16 weights divided by their sum (the
    kernel normalises the blend), FP16 SH."""
    m = t.means.astype(np.float64)
    rest = t.rest_joints.astype(np.float32)
    idx = t.skin_idx.astype(np.int64).copy()
    w = t.skin_w.astype(np.float32).copy()
    n = m.shape[0]
    d = np.empty((n, 4))
    for k in range(4):
        e = m - rest[idx[:, k]].astype(np.float64)
        d[:, k] = e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1] + e[:, 2] * e[:, 2]
    best = np.argmin(d, axis=1)
    rows = np.arange(n)
    for arr in (idx, w):
        first = arr[:, 0].copy()
        arr[:, 0] = arr[rows, best]
        arr[rows, best] = first
    anchor = rest[idx[:, 0]]
    off = R.bf16((m - anchor.astype(np.float64)).astype(np.float32)).astype(np.float32)
    means = (anchor + off).astype(np.float32)
    q = t.quats.astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    Rq = np.stack([oracle.quat_to_rot(x) for x in q])
    s2 = t.scales.astype(np.float64) ** 2
    C = np.einsum("nik,nk,njk->nij", Rq, s2, Rq)
    cov = np.stack([C[:, 0, 0], C[:, 0, 1], C[:, 0, 2], C[:, 1, 1], C[:, 1, 2], C[:, 2, 2]], 1).astype(np.float32)
    out = dataclasses.replace(
        t, means=means, opacity=R.bf16(t.opacity).astype(np.float32), skin_idx=idx.astype(np.uint8),
        skin_w=(R.bf16(w) / R.bf16(w).sum(1, keepdims=True)).astype(np.float32),
        sh=t.sh.astype(np.float16).astype(np.float32))
    out.cov = R.bf16(cov).astype(np.float32)
    return out


def qscene(sc):
    return dataclasses.replace(sc, templates=[quantized(t) for t in sc.templates])


def _check_parity(sc, label, max_boundary=0.08):
    r = make(sc, template_storage=BF16)
    img, st = render(r, sc, stats=True)
    os_q = oracle.OracleScene(qscene(sc))
    errs = PU.compare_splats(r, sc, os_q)
    ref = oracle.render(os_q, PU.eps_from(errs))
    rep = PU.compare_images(img, ref)
    print(f"\n[{label}] splats={st['splats']} duv={errs['duv']:.2e} conic_rel={errs['conic_rel']:.2e} "
          f"depth_rel={errs['depth_rel']:.2e} drgb={errs['drgb']:.2e} live_mismatch={errs['live_mismatch']} | "
          f"max_abs={rep['max_abs']:.2e} psnr={rep['psnr']:.1f} boundary={100 * rep['boundary_frac']:.2f}%")
    assert rep["nonfinite"] == 0
    assert errs["radius_boundary"] == 0
    assert errs["live_mismatch"] <= max(2, errs["n"] // 2000)
    assert rep["max_abs"] <= PU.TOL_MAX_ABS, rep
    assert rep["psnr"] >= PU.TOL_PSNR_DB, rep
    assert rep["boundary_frac"] <= max_boundary
    return r, img, st


def _cam_xyz(cam, uv, z):
    return np.stack([(uv[:, 0] - cam.cx) / cam.fx * z, (uv[:, 1] - cam.cy) / cam.fy * z, z], 1)


def _rounding_bound(sc, os_, i, g, depth):
    """Largest position error the BF16 storage of Gaussians g of instance i
    can cause, from the rounding of the stored values alone (not from the
    library's upload transform, which the quantiser above mirrors): the mean
    is kept as a BF16 offset from its nearest skinning joint, off by at most
    the BF16 unit roundoff 2^-8 of that offset (a rigid transform keeps the
    error's length); the four BF16 weights are each off by at most 2^-8
    relative and renormalised, so by at most 2^-7 w_k, and as they still sum
    to one they move the point by at most 2^-7 sum_k w_k |P_k - P| (P_k the
    point under joint k's transform alone, P the blend).  The skinning
    transforms enter the tensor-core blend as BF16 hi + lo parts, off by
    2^-16 relative of the local coordinates (about 2 m): 2^-14 m with
    margin.  Plus FP32 rounding of the projection (1e-5 m + 1e-6 of the
    depth)."""
    t = sc.templates[int(sc.instances.template_id[i])]
    B = oracle.fk(os_, i)
    mh = np.c_[t.means[g].astype(np.float64), np.ones(len(g))]
    idx = t.skin_idx[g].astype(np.int64)
    w = t.skin_w[g].astype(np.float64)
    Pk = np.stack([np.einsum("nij,nj->ni", B[idx[:, k]], mh) for k in range(4)], 1)
    P = np.einsum("nk,nki->ni", w, Pk)
    spread = np.einsum("nk,nk->n", w, np.linalg.norm(Pk - P[:, None, :], axis=2))
    rest = t.rest_joints.astype(np.float64)
    offset = np.min(np.stack([np.linalg.norm(t.means[g] - rest[idx[:, k]], axis=1) for k in range(4)], 1), axis=1)
    return 2.0 ** -8 * offset + 1.01 * 2.0 ** -7 * spread + 2.0 ** -14 + 1e-5 + 1e-6 * np.abs(depth)


def _precision_cost(r, sc, img, label, lattice=None, max_instances=None):
    """Errors of the BF16 frame against the oracle on the FP32 attributes."""
    os_ = oracle.OracleScene(sc)
    rec = r.debug("records").astype(np.float64)
    inst, gau, _ = PU.splat_ids(r)
    live = PU.gpu_live(r, rec.shape[0])
    cam = sc.camera
    insts = np.unique(inst[live])
    if max_instances:
        insts = insts[:: max(1, len(insts) // max_instances)]
    errs, over = [], 0
    for i in insts:
        p = oracle.project_instance(os_, int(i))
        m = np.nonzero((inst == i) & live)[0]
        g = gau[m]
        ok = p["valid"][g] == 1
        m, g = m[ok], g[ok]
        xg = _cam_xyz(cam, rec[m, 0:2], rec[m, 7])
        xo = _cam_xyz(cam, p["uv"][g], p["depth"][g])
        e = np.linalg.norm(xg - xo, axis=1)
        errs.append(e)
        over += int((e > _rounding_bound(sc, os_, int(i), g, p["depth"][g])).sum())
    pos = np.concatenate(errs)
    ref = oracle.render(os_, lattice=lattice)
    if lattice is None:
        got = img
    else:
        ox, oy, sx, sy, nx, ny = lattice
        got = img[oy::sy, ox::sx][:ny, :nx]
    d = np.abs(got.astype(np.float64) - ref["rgba"])
    mse = float(np.mean(d[..., :3] ** 2))
    psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
    out = dict(mean_pos_m=float(pos.mean()), max_pos_m=float(pos.max()), max_abs=float(d.max()),
               mean_abs=float(d.mean()), psnr=float(psnr), splats_checked=int(pos.size), over_bound=over)
    print(f"[{label} vs FP32 attributes] mean position error {out['mean_pos_m'] * 1e3:.3f} mm "
          f"(max {out['max_pos_m'] * 1e3:.2f} mm over {pos.size} splats, {over} above the rounding bound) | "
          f"pixel max-abs {out['max_abs']:.3e} "
          f"mean-abs {out['mean_abs']:.2e} PSNR {out['psnr']:.1f} dB")
    return out


def test_bf16_single_avatar_parity_and_cost():
    sc = S.single_avatar()
    r, img, st = _check_parity(sc, "bf16 single_avatar")
    cost = _precision_cost(r, sc, img, "bf16 single_avatar")
    assert cost["mean_pos_m"] < 1e-3 and cost["over_bound"] == 0 and cost["psnr"] > 35.0


def test_bf16_small_crowd_lod_parity():
    lod = S.LodConfig(thresholds=np.array([5.0, 8.0], np.float32),
                      fractions=np.array([1.0, 0.25, 0.06], np.float32),
                      scale_mult=(np.array([1.0, 0.25, 0.06]) ** -0.5).astype(np.float32))
    sc = S.crowd(n_templates=3, n_gauss=4096, sh_degree=3, cols=8, rows=6, width=320, height=180, lod=lod)
    r, img, st = _check_parity(sc, "bf16 small_crowd_lod")
    assert all(n > 0 for n in st["instances_per_level"][:3])
    cost = _precision_cost(r, sc, img, "bf16 small_crowd_lod")
    assert cost["mean_pos_m"] < 1e-3 and cost["over_bound"] == 0 and cost["psnr"] > 35.0


def test_bf16_paper_scale_cost_and_memory():
    """The paper-scale frame (3,500 instances, 1920x1080) in BF16 storage:
    sampled pixels against the oracle on the FP32 attributes, template
    memory halved."""
    sc = S.crowd()
    r32 = make(sc)
    render(r32, sc)
    m32 = r32.memory_stats()["template_bytes"]
    r32.close()
    r = make(sc, template_storage=BF16)
    img, st = render(r, sc, stats=True)
    m16 = r.memory_stats()["template_bytes"]
    lat = (5, 3, 37, 29, (1920 - 5 + 36) // 37, (1080 - 3 + 28) // 29)
    cost = _precision_cost(r, sc, img, "bf16 paper scale", lattice=lat, max_instances=40)
    print(f"[bf16 paper scale] template bytes {m16 / 2**20:.1f} MiB vs FP32 {m32 / 2**20:.1f} MiB; "
          f"splats={st['splats']} pairs={st['pairs']}")
    n = sum(t.means.shape[0] for t in sc.templates)
    assert m16 <= n * 128 + 65536 and m32 >= n * 250
    assert cost["mean_pos_m"] < 1e-3 and cost["over_bound"] == 0 and cost["psnr"] > 30.0


def test_bf16_features_follow_the_stored_values():
    sc = S.crowd(n_templates=2, n_gauss=2048, sh_degree=3, cols=2, rows=1, width=64, height=48)
    r = make(sc, template_storage=BF16)
    f = r.lod_features().cpu().numpy().astype(np.float64)
    qs = qscene(sc)
    ref = np.concatenate([R.features(t) for t in qs.templates])
    # the kernel reports the stored (unnormalised) BF16 weights
    weights = [19, 20, 21, 22]
    other = [c for c in range(32) if c not in weights]
    assert np.abs(f[:, weights] - ref[:, weights]).max() < 0.01
    d = np.abs(f[:, other] - ref[:, other])
    assert d.max() < 1e-4, (np.unravel_index(np.argmax(d), d.shape), d.max())
