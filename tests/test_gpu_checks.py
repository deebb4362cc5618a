"""The frames of the parity tests once more through the debug build with
bounds checks in the kernels (libcrowdsplat_checks.so, CS_CHECKS=1): every
checked index (splat records, pairs, tiles, splat ids, sort positions,
compositing slots) stays inside its buffer, and the checks change no pixel
beyond rounding.  Stands in for compute-sanitizer, which this GPU pool does
not offer."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2501_17792_gb300 import binding, build
from paper_2501_17792_gb300 import scene as S
from tests import scene_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked():
    return build.build(checks=True)


def _pair(sc, checked):
    out = []
    for lib in (None, checked):
        r = binding.Renderer(device=0, library=lib)
        r.upload_templates(sc.templates)
        r.set_lod(sc.lod)
        r.set_instances(sc.instances.template_id, sc.instances.root, sc.instances.pose)
        out.append(r)
    return out


def _frames():
    lod = S.LodConfig(thresholds=np.array([5.0, 8.0], np.float32), fractions=np.array([1.0, 0.25, 0.06], np.float32),
                      scale_mult=(np.array([1.0, 0.25, 0.06]) ** -0.5).astype(np.float32))
    yield "crowd", S.crowd(n_templates=3, n_gauss=4096, sh_degree=3, cols=8, rows=6, width=320, height=180, lod=lod)
    # lists past the 32,768-pair pass-1 budget (split compositing), within the static call's limits
    rng = np.random.default_rng(5)
    n, w, h, f = 60000, 32, 16, 60.0
    z = rng.uniform(2.0, 6.0, n)
    px, py = rng.uniform(0, w, n), rng.uniform(0, h, n)
    s = (1.5 * z / f)[:, None] * np.exp(rng.normal(0, 0.3, (n, 3)))
    tpl = U.template_from(np.stack([(px - w / 2) * z / f, (py - h / 2) * z / f, z], 1), s, rng.standard_normal((n, 4)),
                          rng.uniform(0.006, 0.016, n), 0.3 * rng.standard_normal((n, 4, 3)))
    yield "deep", U.scene_of([tpl], U.instances(1), U.identity_camera(w, h, f))


def _same(a, b, what):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape and np.abs(a - b).max() <= 1e-6, (what, float(np.abs(a - b).max()))


def test_checked_build_reports_no_out_of_range_index(checked):
    for name, sc in _frames():
        rel, chk = _pair(sc, checked)
        assert chk.debug_checks() == (0, True)
        assert rel.debug_checks() == (0, False)
        # plain frames under every compositing schedule
        for mode in (binding.CS_BLEND_ITEMS_AUTO, binding.CS_BLEND_ITEMS_TILES, binding.CS_BLEND_ITEMS_BLOCKS):
            rel.debug_blend_items(mode)
            chk.debug_blend_items(mode)
            imgs = [r.render(sc.camera).cpu().numpy() for r in (rel, chk)]
            assert chk.debug_checks() == (0, True), (name, mode)
            _same(*imgs, (name, mode))
        if name == "deep":
            ranges = chk.debug("tile_ranges").astype(np.int64)
            assert (ranges[:, 1] - ranges[:, 0]).max() > 32768  # the split passes ran
        # statistics frame (one pass, per-splat contribution sums) and training frame
        ctr = [torch.zeros(r.n_gauss_total, dtype=torch.float32, device="cuda") for r in (rel, chk)]
        imgs = [r.render_contrib(sc.camera, c).cpu().numpy() for r, c in zip((rel, chk), ctr)]
        assert chk.debug_checks() == (0, True), name
        _same(*imgs, (name, "contrib image"))
        assert torch.allclose(ctr[0], ctr[1], rtol=1e-5, atol=1e-7), name
        imgs = [r.render_train(sc.camera).cpu().numpy() for r in (rel, chk)]
        assert chk.debug_checks() == (0, True), name
        _same(*imgs, (name, "train image"))
        # the allocation-free call and its static scratch
        if name == "deep":
            cam = binding.camera_struct(sc.camera)
            imgs = []
            for r in (rel, chk):
                out = torch.empty((sc.camera.height, sc.camera.width, 4), dtype=torch.float32, device="cuda")
                assert r.L.cs_render_static(r.h, C.byref(cam), C.c_void_p(out.data_ptr()), None) == binding.CS_OK
                imgs.append(out.cpu().numpy())
            assert chk.debug_checks() == (0, True), name
            _same(*imgs, (name, "static image"))
        rel.close()
        chk.close()
