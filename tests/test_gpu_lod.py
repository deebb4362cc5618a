"""GPU parity of the ranked-LoD support: chosen Gaussian subsets per
(template, level) and the per-Gaussian contribution sums of
cs_render_contrib, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_17792_gb300 import scene as S
from tests import parity_util as PU
from tests.test_gpu_parity import built, full_check, make, render  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _crowd(width=256, height=144):
    lod = S.LodConfig(thresholds=np.array([5.0, 8.0], np.float32),
                      fractions=np.array([1.0, 0.25, 0.06], np.float32),
                      scale_mult=(np.array([1.0, 0.25, 0.06]) ** -0.5).astype(np.float32))
    return S.crowd(n_templates=3, n_gauss=4096, sh_degree=1, cols=8, rows=6, width=width, height=height,
                   lod=lod)


def _random_subsets(sc, seed):
    rng = np.random.default_rng(seed)
    out = {}
    for t, tpl in enumerate(sc.templates):
        n = tpl.means.shape[0]
        for l, f in enumerate(sc.lod.fractions):
            if (t + l) % 2 == 0:
                k = max(1, int(round(float(f) * n * rng.uniform(0.5, 1.0))))
                out[(t, l)] = rng.permutation(n)[:k].astype(np.uint32)
    return out


def test_lod_subsets_match_oracle():
    sc = _crowd()
    sub = _random_subsets(sc, 3)
    r, img, ref, errs, st = full_check(sc, subsets=sub, label="lod_subsets")
    assert all(n > 0 for n in st["instances_per_level"][:3]), st
    # the level sizes follow the subsets
    groups = r.debug("groups")
    for tpl, lv, _s0, _ns, ng, _sp, _b in groups:
        want = len(sub[(int(tpl), int(lv))]) if (int(tpl), int(lv)) in sub else \
            oracle.level_count(oracle.OracleScene(sc), int(lv), sc.templates[int(tpl)].means.shape[0])
        assert int(ng) == want


def test_subset_errors_and_clear():
    from paper_2501_17792_gb300 import binding
    sc = _crowd(160, 96)
    r = make(sc)
    base = render(r, sc)
    n = sc.templates[0].means.shape[0]
    for bad in ([0, 0], [n], [5, n + 3]):
        with pytest.raises(binding.CrowdSplatError) as e:
            r.set_lod_subset(0, 0, np.asarray(bad, np.uint32))
        assert e.value.code == binding.CS_ERR_ARG
    with pytest.raises(binding.CrowdSplatError):
        r.set_lod_subset(7, 0, [1])
    with pytest.raises(binding.CrowdSplatError):
        r.set_lod_subset(0, 4, [1])
    # a subset equal to the prefix, then cleared: the image does not change
    k = int(round(0.25 * n))
    r.set_lod_subset(0, 1, np.arange(k, dtype=np.uint32))
    assert np.array_equal(render(r, sc), base)
    r.set_lod_subset(0, 1, [5, 9, 11])
    changed = render(r, sc)
    r.set_lod_subset(0, 1, np.zeros(0, np.uint32))
    assert np.array_equal(render(r, sc), base)
    assert not np.array_equal(changed, base)


def _contrib_gpu(r, sc):
    n_total = sum(t.means.shape[0] for t in sc.templates)
    c = torch.zeros(n_total, dtype=torch.float32, device="cuda:0")
    img, st = r.render_contrib(sc.camera, c, stats=True)
    torch.cuda.synchronize()
    return img.cpu().numpy(), c.cpu().numpy().astype(np.float64), st


def _check_contrib(sc, subsets=None, label=""):
    """Per-Gaussian contribution sums against the oracle.  Per pixel the two
    compositing weights agree to the image tolerance, so a Gaussian whose
    support boxes (over all instances) hold no boundary pixel must agree to
    TOL_MAX_ABS x the number of pixels in those boxes."""
    r = make(sc)
    for (t, l), idx in (subsets or {}).items():
        r.set_lod_subset(t, l, idx)
    plain = render(r, sc)
    img, c, st = _contrib_gpu(r, sc)
    os_ = oracle.OracleScene(sc, subsets=subsets)
    errs = PU.compare_splats(r, sc, os_)
    ref = oracle.render(os_, PU.eps_from(errs), contrib=True)
    co = ref["contrib"]
    W, H = sc.camera.width, sc.camera.height
    # the image of the statistics pass is the plain image (up to rounding order)
    assert np.abs(img - plain).max() <= 1e-5
    # sum of all contributions = sum of the alpha channel
    assert abs(c.sum() - img[..., 3].astype(np.float64).sum()) <= 1e-4 * max(1.0, c.sum())
    assert c.min() >= 0.0
    # boundary pixels: integral image of the oracle's flags
    bnd = np.pad((ref["flags"] != 0).astype(np.int64), ((1, 0), (1, 0))).cumsum(0).cumsum(1)
    g_off = np.concatenate([[0], np.cumsum([t.means.shape[0] for t in sc.templates])])
    npx = np.zeros(c.shape[0])
    nbnd = np.zeros(c.shape[0])
    touched = np.zeros(c.shape[0], bool)
    for i, p in errs["ref"].items():
        t = int(sc.instances.template_id[i])
        lv = p["level"]
        key = (t, lv)
        gidx = np.asarray(subsets[key], np.int64) if subsets and key in subsets else np.arange(p["count"])
        ok = p["valid"] == 1
        u, v, rr = p["uv"][:, 0], p["uv"][:, 1], p["radius"]
        x0 = np.clip(np.ceil(u - rr - 0.5), 0, W).astype(np.int64)
        x1 = np.clip(np.floor(u + rr - 0.5) + 1, 0, W).astype(np.int64)
        y0 = np.clip(np.ceil(v - rr - 0.5), 0, H).astype(np.int64)
        y1 = np.clip(np.floor(v + rr - 0.5) + 1, 0, H).astype(np.int64)
        x1, y1 = np.maximum(x1, x0), np.maximum(y1, y0)
        area = np.where(ok, (x1 - x0) * (y1 - y0), 0)
        nb = bnd[y1, x1] - bnd[y0, x1] - bnd[y1, x0] + bnd[y0, x0]
        np.add.at(npx, g_off[t] + gidx, area)
        np.add.at(touched, g_off[t] + gidx, ok & (nb > 0))
        np.add.at(nbnd, g_off[t] + gidx, np.where(ok, nb, 0))
    clean = ~touched
    d = np.abs(c - co)
    tol = PU.TOL_MAX_ABS * npx + 1e-6
    bad = clean & (d > tol)
    print(f"\n[{label}] gaussians={c.size} contributing={(co > 0).sum()} clean={clean.sum()} "
          f"max|d|={d[clean].max():.2e} max rel={(d[clean] / np.maximum(co[clean], 1e-3)).max():.2e} "
          f"sum gpu={c.sum():.3f} oracle={co.sum():.3f}")
    assert not bad.any(), (np.nonzero(bad)[0][:5], d[bad][:5], tol[bad][:5])
    # a boundary pixel moves a weight by at most 1
    assert np.all(d <= tol + nbnd)
    assert clean.sum() > 1000
    assert np.abs(c - co).sum() <= 1e-3 * co.sum()
    # Gaussians outside every rendered level receive nothing
    assert np.all(c[npx == 0] == 0.0)
    return c, co


def test_contrib_single_avatar():
    sc = S.single_avatar(n_gauss=8192, size=192)
    c, co = _check_contrib(sc, label="contrib_single")
    assert (co > 0).sum() > 4000


def test_contrib_crowd_with_subsets():
    sc = _crowd()
    sub = _random_subsets(sc, 5)
    c, co = _check_contrib(sc, subsets=sub, label="contrib_crowd_subsets")
    # a Gaussian outside its template's subsets on every level gets nothing
    assert (c == 0).sum() > 0


def test_contrib_accumulates_across_calls():
    sc = S.single_avatar(n_gauss=2048, size=96)
    r = make(sc)
    _, c1, _ = _contrib_gpu(r, sc)
    n_total = c1.size
    c = torch.zeros(n_total, dtype=torch.float32, device="cuda:0")
    r.render_contrib(sc.camera, c)
    r.render_contrib(sc.camera, c)
    torch.cuda.synchronize()
    assert np.allclose(c.cpu().numpy(), 2 * c1, rtol=1e-5, atol=1e-6)
