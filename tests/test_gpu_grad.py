"""GPU gradients (cs_render_train + cs_backward) against central finite
differences of the FP64 oracle.

The loss is L = sum over pixels and RGBA channels of a fixed random weight
times the rendered value; dL/d(image) is that weight.  Pixels the oracle
flags as boundary cases get weight 0, so the loss is smooth in the
parameters up to the discrete decisions of the forward.  Each finite
difference perturbs the float32 inputs by a power of two, so the oracle sees
exactly the perturbed value, and divides by the actual difference of the
inputs.  A step can still move a splat's support-box edge or its 1/255
alpha threshold across a pixel: such a jump shows as a disagreement between
the differences at h and h/4, and that parameter is set aside (counted).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2501_17792_gb300 import scene as S
from tests.test_gpu_parity import built, make  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# finite-difference steps (powers of two) per parameter kind
H = dict(means=2.0 ** -17, scales=2.0 ** -19, quats=2.0 ** -15, opacity=2.0 ** -14, sh=2.0 ** -10,
         pose=2.0 ** -19)


def grad_scene(n_gauss=384, n_inst=3, size=96, sh_degree=3, seed=0, lod=None):
    tpl = S.make_template(2000 + seed, n_gauss, sh_degree)
    rng = np.random.default_rng(seed)
    roots = np.stack([S.yaw_root(rng.uniform(0, 2 * math.pi), x, 0.0, 3.0 + rng.uniform(-0.3, 0.3))
                      for x in np.linspace(-0.7, 0.7, n_inst)]).astype(np.float32)
    inst = S.Instances(np.zeros(n_inst, np.int32), roots, S.random_poses(seed + 50, n_inst))
    cam = S.look_camera((0.0, 0.9, 0.0), 0.0, size, size, vfov_deg=50.0)
    return S.Scene([tpl], inst, cam, lod if lod is not None else S.single_lod(), "grad")


def loss_weights(sc, seed=1, stride=1):
    """Random dL/d(RGBA), zero at oracle boundary pixels (and off the
    lattice of the given stride)."""
    Hh, Ww = sc.camera.height, sc.camera.width
    wt = np.random.default_rng(seed).normal(0, 1, (Hh, Ww, 4)).astype(np.float32)
    lat = (0, 0, stride, stride, (Ww + stride - 1) // stride, (Hh + stride - 1) // stride)
    ref = oracle.render(oracle.OracleScene(sc), lattice=lat)
    mask = np.zeros((Hh, Ww), bool)
    mask[::stride, ::stride] = ref["flags"] == 0
    wt[~mask] = 0.0
    return wt, lat


def oracle_loss(sc, wt, lat):
    ox, oy, sx, sy, nx, ny = lat
    rgba = oracle.render(oracle.OracleScene(sc), lattice=lat)["rgba"]
    return float(np.sum(wt[oy::sy, ox::sx][:ny, :nx].astype(np.float64) * rgba))


def gpu_grads(sc, wt, **kw):
    r = make(sc, **kw)
    r.render_train(sc.camera)
    g = r.backward(torch.from_numpy(wt).cuda(), sc.instances.n)
    torch.cuda.synchronize()
    return r, {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def perturbed(sc, kind, index, delta):
    """Copy of the scene with one float32 input moved by delta; returns the
    scene and the actual change of that input."""
    t = sc.templates[0]
    if kind == "pose":
        pose = sc.instances.pose.copy()
        old = pose.reshape(-1)[index]
        pose.reshape(-1)[index] = np.float32(old + delta)
        new = pose.reshape(-1)[index]
        return dataclasses.replace(sc, instances=dataclasses.replace(sc.instances, pose=pose)), float(new) - float(old)
    name = {"means": "means", "scales": "scales", "quats": "quats", "opacity": "opacity", "sh": "sh"}[kind]
    arr = getattr(t, name).copy()
    flat = arr.reshape(-1)
    old = flat[index]
    flat[index] = np.float32(old + delta)
    new = flat[index]
    t2 = dataclasses.replace(t, **{name: arr})
    return dataclasses.replace(sc, templates=[t2]), float(new) - float(old)


def input_value(sc, kind, index):
    if kind == "pose":
        return float(sc.instances.pose.reshape(-1)[index])
    return float(getattr(sc.templates[0], kind).reshape(-1)[index])


def step_scale(sc, kind, index, h_min):
    """Power of two by which a step of h_min must grow to move the float32
    input at all: one unit in the last place of its value at least."""
    ulp = float(np.spacing(np.float32(abs(input_value(sc, kind, index)))))
    return max(1.0, ulp / h_min)


def fd(sc, wt, lat, kind, index, h):
    sp, dp = perturbed(sc, kind, index, h)
    sm, dm = perturbed(sc, kind, index, -h)
    return (oracle_loss(sp, wt, lat) - oracle_loss(sm, wt, lat)) / (dp - dm)


def flat_grad(g, kind):
    if kind == "sh":
        return g["sh"].reshape(g["sh"].shape[0], -1)  # [N, 48], oracle sh is [N, K, 3]
    return g[kind].reshape(g[kind].shape[0], -1) if g[kind].ndim > 1 else g[kind][:, None]


def check_kind(sc, wt, lat, g, kind, n_pick=10, seed=0, steps=None):
    steps = steps or H
    t = sc.templates[0]
    rng = np.random.default_rng(seed)
    if kind == "pose":
        gv = g["pose"].reshape(-1)
        cand = np.nonzero(np.abs(gv) > 0)[0]
        gidx = list(cand[np.argsort(-np.abs(gv[cand]))[:n_pick // 2]]) + list(rng.choice(cand, n_pick // 2, replace=False))
        pairs = [(int(i), gv[i], int(i)) for i in gidx]
    elif kind == "sh":
        K = (t.sh_degree + 1) ** 2
        gs = g["sh"][:, :K, :]
        flat = gs.reshape(-1)
        cand = np.nonzero(np.abs(flat) > 0)[0]
        pick = list(cand[np.argsort(-np.abs(flat[cand]))[:n_pick // 2]]) + list(rng.choice(cand, n_pick // 2, replace=False))
        pairs = [(int(i), flat[i], int(i)) for i in pick]  # [N, K, 3] flat == the oracle's sh flat
    else:
        G = flat_grad(g, kind)
        flat = G.reshape(-1)
        cand = np.nonzero(np.abs(flat) > 0)[0]
        pick = list(cand[np.argsort(-np.abs(flat[cand]))[:n_pick // 2]]) + list(rng.choice(cand, n_pick // 2, replace=False))
        pairs = [(int(i), flat[i], int(i)) for i in pick]
    res = []
    for idx, gval, oidx in pairs:
        h = steps[kind] * step_scale(sc, kind, oidx, steps[kind] / 4)
        f = fd(sc, wt, lat, kind, oidx, h)
        f4 = fd(sc, wt, lat, kind, oidx, h / 4)
        res.append((idx, gval, f, f4))
    res = np.array(res)
    gpu, ref, ref4 = res[:, 1], res[:, 2], res[:, 3]
    scale = np.sqrt(np.mean(ref ** 2)) + 1e-12
    smooth = np.abs(ref - ref4) <= 1e-3 * np.abs(ref) + 1e-4 * scale  # no jump inside the step
    err = np.abs(gpu - ref)
    ok = ~smooth | (err <= 1e-2 * np.abs(ref) + 1e-3 * scale)
    rel = err / (np.abs(ref) + 1e-3 * scale)
    print(f"[grad {kind}] n={len(res)} smooth={int(smooth.sum())} max rel err (smooth) "
          f"{np.max(rel[smooth]) if smooth.any() else float('nan'):.2e} median {np.median(rel[smooth]):.2e} "
          f"mismatches {int((~ok).sum())}")
    assert smooth.sum() >= 0.6 * len(res), res
    return ok, res


@pytest.fixture(scope="module")
def small():
    sc = grad_scene()
    wt, lat = loss_weights(sc)
    r, g = gpu_grads(sc, wt)
    return sc, wt, lat, g


@pytest.mark.parametrize("kind", ["means", "scales", "quats", "opacity", "sh", "pose"])
def test_gradient_matches_finite_differences(small, kind):
    sc, wt, lat, g = small
    ok, res = check_kind(sc, wt, lat, g, kind)
    assert ok.all(), res[~ok]


def test_gradient_with_lod_multiplier_and_world_frame_sh():
    lod = S.LodConfig(thresholds=np.zeros(0, np.float32), fractions=np.ones(1, np.float32),
                      scale_mult=np.array([1.7], np.float32))
    sc = grad_scene(n_gauss=256, seed=3, lod=lod)
    wt, lat = loss_weights(sc, seed=4)
    r = make(sc, sh_frame=1)
    r.render_train(sc.camera)
    g = r.backward(torch.from_numpy(wt).cuda(), sc.instances.n)
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}

    os_cls = oracle.OracleScene

    class World(os_cls):  # the oracle in the same SH frame
        def __init__(self, scene, **kw):
            super().__init__(scene, sh_frame=1, **kw)

    oracle.OracleScene = World
    try:
        for kind in ("means", "scales", "pose", "sh"):
            ok, res = check_kind(sc, wt, lat, g, kind, n_pick=6, seed=5)
            assert ok.all(), (kind, res[~ok])
    finally:
        oracle.OracleScene = os_cls


def test_training_frame_state_and_errors():
    from paper_2501_17792_gb300 import binding
    sc = grad_scene(n_gauss=128)
    r = make(sc)
    wt = torch.zeros((sc.camera.height, sc.camera.width, 4), device="cuda")
    with pytest.raises(binding.CrowdSplatError) as e:
        r.backward(wt, sc.instances.n)  # no training frame yet
    assert e.value.code == binding.CS_ERR_STATE
    img_t = r.render_train(sc.camera).cpu().numpy()
    img = r.render(sc.camera).cpu().numpy()
    assert np.abs(img_t - img).max() < 1e-5
    with pytest.raises(binding.CrowdSplatError):
        r.backward(wt, sc.instances.n)  # a plain render replaced the training frame
    r.render_train(sc.camera)
    g = r.backward(wt, sc.instances.n)
    assert all(float(v.abs().max()) == 0.0 for v in g.values())  # zero loss, zero gradient
    rb = make(sc, template_storage=binding.CS_STORE_BF16)
    with pytest.raises(binding.CrowdSplatError):
        rb.render_train(sc.camera)


def test_gradient_at_scale():
    """1 template of 65,536 Gaussians (SH degree 3), 64 instances, 512x512,
    loss on every 4th pixel in x and y: per-parameter central differences of
    the oracle for the largest gradients of each kind.  One template
    Gaussian moves 64 splats and one joint thousands, so the steps are
    smaller than for the small scene, to keep support-box edges and alpha
    thresholds from crossing a pixel inside a step."""
    tpl = S.make_template(2100, 65536, 3)
    rng = np.random.default_rng(9)
    roots = [S.yaw_root(rng.uniform(0, 2 * math.pi), (col - 3.5) * 0.9, 0.0, 3.0 + row * 0.9)
             for row in range(8) for col in range(8)]
    inst = S.Instances(np.zeros(64, np.int32), np.stack(roots).astype(np.float32), S.random_poses(77, 64))
    cam = S.look_camera((0.0, 1.4, 0.0), 12.0, 512, 512, vfov_deg=60.0)
    sc = S.Scene([tpl], inst, cam, S.single_lod(), "grad_scale")
    wt, lat = loss_weights(sc, seed=2, stride=4)
    r, g = gpu_grads(sc, wt)
    steps = dict(means=2.0 ** -22, scales=2.0 ** -24, quats=2.0 ** -20, opacity=2.0 ** -18, sh=2.0 ** -12,
                 pose=2.0 ** -24)
    for kind in ("means", "scales", "quats", "opacity", "sh", "pose"):
        ok, res = check_kind(sc, wt, lat, g, kind, n_pick=4, seed=11, steps=steps)
        assert ok.all(), (kind, res[~ok])


def test_autograd_function_and_a_fit():
    """The torch.autograd wrapper gives the library's gradients, and a few
    Adam steps on the template means pull a rendered crowd towards a target
    rendered from shifted means."""
    from paper_2501_17792_gb300 import autograd as AG
    from paper_2501_17792_gb300 import binding
    sc = grad_scene(n_gauss=256, seed=6)
    t = sc.templates[0]
    wt, lat = loss_weights(sc, seed=7)
    _, g_ref = gpu_grads(sc, wt)
    r = binding.Renderer(device=0)
    params = [torch.tensor(a, requires_grad=True) for a in (t.means, t.scales, t.quats, t.opacity, t.sh)]
    pose = torch.tensor(sc.instances.pose, requires_grad=True)
    img = AG.render(r, sc.camera, sc.instances, t, *params, pose)
    (img * torch.from_numpy(wt).cuda()).sum().backward()
    def close(a, b):  # float32 atomics: the summation order varies between runs
        return np.allclose(a, b, rtol=1e-4, atol=1e-5 * np.abs(b).max())

    for name, p in zip(("means", "scales", "quats", "opacity"), params[:4]):
        assert close(p.grad.numpy(), g_ref[name].reshape(p.shape)), name
    K = t.sh.shape[1]
    assert close(params[4].grad.numpy(), g_ref["sh"][:, :K, :])
    assert close(pose.grad.numpy(), g_ref["pose"])
    # fit: target from means shifted by 5 mm
    shift = np.float32(0.005)
    with torch.no_grad():
        target = AG.render(r, sc.camera, sc.instances, t, params[0] + shift, *params[1:], pose).clone()
    means = torch.tensor(t.means, requires_grad=True)
    opt = torch.optim.Adam([means], lr=5e-4)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        img = AG.render(r, sc.camera, sc.instances, t, means, *params[1:], pose)
        loss = ((img - target) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    print(f"\n[grad fit] loss {losses[0]:.4f} -> {losses[-1]:.4f}; mean shift recovered "
          f"{float((means.detach() - torch.tensor(t.means)).mean()):.5f} m of {shift}")
    assert losses[-1] < 0.2 * losses[0]
