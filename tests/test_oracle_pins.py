"""Pins of the FP64 oracle against facts outside itself.

Each test compares the oracle with a library routine (scipy's expm,
Rotation, complex spherical harmonics), a closed form (analytic splat
footprint, two-layer compositing, a kinematic chain written as rotations
about rest joint centres), Monte-Carlo sampling, brute force on tiny
scenes, an invariance of the definition, or a value the paper prints
(tests/golden/paper_lod.json).  Together they are chosen so that a dropped
term, a wrong sign or index, or a transposed operand anywhere in the oracle
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation
import scipy.special as sps

import oracle
from paper_2501_17792_gb300 import scene as S
from tests import scene_util as U

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]], dtype=np.float64)


# ---------------------------------------------------------------------------
# rotations
# ---------------------------------------------------------------------------

def test_rodrigues_equals_matrix_exponential():
    rng = np.random.default_rng(0)
    vs = [rng.normal(0, 1, 3) for _ in range(30)]
    vs += [np.array([1e-10, -2e-10, 3e-11]), np.zeros(3), np.array([math.pi, 0, 0]),
           np.array([0.0, 3.0, 1.0]), np.array([1e-7, 0, 0])]
    for v in vs:
        assert np.abs(oracle.rodrigues(v) - expm(skew(v))).max() < 1e-13, v


def test_quaternion_matches_scipy_rotation():
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.normal(size=4) * rng.uniform(0.1, 5.0)  # unnormalised (w,x,y,z)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.abs(oracle.quat_to_rot(q) - ref).max() < 1e-14


# ---------------------------------------------------------------------------
# spherical harmonics
# ---------------------------------------------------------------------------

def _sh_ref(l, m, d):
    """Real SH in the 3DGS convention from scipy's complex SH (which carry
    the Condon-Shortley phase): sqrt(2) Im Y_l^|m| for m < 0, Y_l^0, and
    sqrt(2) Re Y_l^m for m > 0."""
    theta = np.arccos(np.clip(d[..., 2], -1, 1))
    phi = np.arctan2(d[..., 1], d[..., 0])
    if m < 0:
        return math.sqrt(2) * np.imag(sps.sph_harm_y(l, -m, theta, phi))
    if m == 0:
        return np.real(sps.sph_harm_y(l, 0, theta, phi))
    return math.sqrt(2) * np.real(sps.sph_harm_y(l, m, theta, phi))


def test_sh_basis_matches_scipy_complex_harmonics():
    rng = np.random.default_rng(2)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            assert np.abs(Y[:, k] - _sh_ref(l, m, d)).max() < 1e-12, (l, m)
    # degree-1 sign convention of the 3DGS rasteriser: C1 (-y, z, -x)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[:, 1:4], c1 * np.stack([-d[:, 1], d[:, 2], -d[:, 0]], 1), atol=1e-14)


def test_sh_basis_orthonormal_by_quadrature():
    n = 40000
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    phi = math.pi * (1 + 5 ** 0.5) * i
    rxy = np.sqrt(1 - z * z)
    d = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], 1)
    Y = oracle.sh_basis(3, d)
    G = (Y.T @ Y) * (4 * math.pi / n)
    assert np.abs(G - np.eye(16)).max() < 1e-3


def test_sh_lower_degrees_are_prefixes():
    d = np.array([[0.3, -0.5, 0.81]])
    d /= np.linalg.norm(d)
    full = oracle.sh_basis(3, d)
    for deg in range(3):
        assert np.array_equal(oracle.sh_basis(deg, d), full[:, :(deg + 1) ** 2])


# ---------------------------------------------------------------------------
# forward kinematics and LBS
# ---------------------------------------------------------------------------

def _chain(j):
    out = []
    while j >= 0:
        out.append(j)
        j = int(S.PARENTS[j])
    return out[::-1]  # root ... j


def _posed_by_chain(x, j, pose, rest, root):
    """Rigid motion of a point attached to joint j: rotate about each rest
    joint centre from j up to the root (A_j(x) = J_j + R_j (x - J_j)), then
    apply the root transform."""
    y = np.asarray(x, np.float64)
    for k in reversed(_chain(j)):
        Rk = expm(skew(pose[k].astype(np.float64)))
        y = rest[k] + Rk @ (y - rest[k])
    return root[:, :3] @ y + root[:, 3]


def _one_instance_scene(tpl, root, pose):
    return U.scene_of([tpl], U.instances(1, root[None], pose[None]),
                      U.identity_camera(64, 64, 80.0))


def test_fk_identity_and_rigid_root():
    sc = S.single_avatar(n_gauss=64)
    sc.instances.pose[:] = 0
    eye = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32)
    sc.instances.root[0] = eye
    B = oracle.fk(oracle.OracleScene(sc), 0)
    assert np.abs(B - eye[None]).max() < 1e-15
    root = S.yaw_root(0.7, 1.0, -2.0, 3.5).astype(np.float32)
    sc.instances.root[0] = root
    B = oracle.fk(oracle.OracleScene(sc), 0)
    assert np.abs(B - root.astype(np.float64)[None]).max() < 1e-15


def test_fk_matches_rotations_about_rest_joints():
    sc = S.single_avatar(n_gauss=64)
    rng = np.random.default_rng(3)
    pose = rng.normal(0, 0.5, (24, 3)).astype(np.float32)
    root = S.yaw_root(1.3, 0.5, 0.1, 4.0).astype(np.float32)
    sc.instances.pose[0] = pose
    sc.instances.root[0] = root
    B = oracle.fk(oracle.OracleScene(sc), 0)
    rest = sc.templates[0].rest_joints.astype(np.float64)
    for j in range(24):
        for _ in range(3):
            x = rng.normal(0, 0.5, 3) + rest[j]
            ref = _posed_by_chain(x, j, pose, rest, root.astype(np.float64))
            got = B[j][:, :3] @ x + B[j][:, 3]
            assert np.abs(got - ref).max() < 1e-12, j


def _tpl_single(mu, skin_idx, skin_w, scales=(0.02, 0.005, 0.01), quat=(1, 0, 0, 0), rest=None):
    return U.template_from([mu], [scales], [quat], [0.8], np.zeros((1, 1, 3)),
                           skin_idx=[skin_idx], skin_w=[skin_w], rest_joints=rest)


def test_lbs_one_hot_weight_moves_rigidly_with_its_joint():
    rng = np.random.default_rng(4)
    rest = S._REST.astype(np.float32)
    pose = rng.normal(0, 0.4, (24, 3)).astype(np.float32)
    root = S.yaw_root(0.4, 0.2, 0.0, 3.0).astype(np.float32)
    quat = np.array([0.9, 0.1, -0.3, 0.2], np.float32).astype(np.float64)
    for j in (0, 4, 7, 15, 20):
        mu = rest[j] + np.array([0.05, -0.02, 0.03], np.float32)
        tpl = _tpl_single(mu, [j, (j + 1) % 24, 2, 3], [1.0, 0.0, 0.0, 0.0], quat=quat, rest=rest)
        p = oracle.project_instance(oracle.OracleScene(_one_instance_scene(tpl, root, pose)), 0)
        ref = _posed_by_chain(mu, j, pose, rest.astype(np.float64), root.astype(np.float64))
        assert np.abs(p["mu"][0] - ref).max() < 1e-12
        # covariance of a rigidly moved Gaussian: R Sigma R^T, with R the
        # rotation of the chain (read off by moving three unit offsets)
        Rch = np.stack([_posed_by_chain(mu + e, j, pose, rest.astype(np.float64),
                                        root.astype(np.float64)) - ref for e in np.eye(3)], 1)
        Rq = Rotation.from_quat([quat[1], quat[2], quat[3], quat[0]]).as_matrix()
        Sig = Rq @ np.diag(np.array([0.02, 0.005, 0.01], np.float32).astype(np.float64) ** 2) @ Rq.T
        ref_cov = Rch @ Sig @ Rch.T
        c = p["cov3"][0]
        got = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        assert np.abs(got - ref_cov).max() < 1e-15


def test_lbs_weights_partition_of_unity_and_pairing():
    rng = np.random.default_rng(5)
    rest = S._REST.astype(np.float32)
    root = S.yaw_root(2.0, -0.3, 0.0, 2.0).astype(np.float32)
    mu = np.array([0.1, 1.0, 0.05], np.float32)
    w = np.array([0.5, 0.25, 0.125, 0.125], np.float32)  # exact sum 1
    idx = [3, 6, 9, 12]
    # identical joint transforms (zero pose): result is root . mu for any weights
    tpl = _tpl_single(mu, idx, w, rest=rest)
    p = oracle.project_instance(oracle.OracleScene(_one_instance_scene(tpl, root, np.zeros((24, 3), np.float32))), 0)
    ref = root[:, :3].astype(np.float64) @ mu + root[:, 3]
    assert np.abs(p["mu"][0] - ref).max() < 1e-12
    # permuting the (joint, weight) pairs leaves the result unchanged
    pose = rng.normal(0, 0.4, (24, 3)).astype(np.float32)
    base = oracle.project_instance(oracle.OracleScene(_one_instance_scene(tpl, root, pose)), 0)
    perm = [2, 0, 3, 1]
    tpl2 = _tpl_single(mu, [idx[k] for k in perm], w[perm], rest=rest)
    p2 = oracle.project_instance(oracle.OracleScene(_one_instance_scene(tpl2, root, pose)), 0)
    assert np.abs(p2["mu"][0] - base["mu"][0]).max() < 1e-12
    assert np.abs(p2["cov3"][0] - base["cov3"][0]).max() < 1e-14
    # a joint outside the four has no influence; a joint inside does
    pose_b = pose.copy()
    pose_b[20] += 0.5
    p3 = oracle.project_instance(oracle.OracleScene(_one_instance_scene(tpl, root, pose_b)), 0)
    assert np.abs(p3["mu"][0] - base["mu"][0]).max() < 1e-15
    pose_c = pose.copy()
    pose_c[9] += 0.5  # joint 9 is in the list (and an ancestor of 12)
    p4 = oracle.project_instance(oracle.OracleScene(_one_instance_scene(tpl, root, pose_c)), 0)
    assert np.abs(p4["mu"][0] - base["mu"][0]).max() > 1e-4


def test_canonical_covariance_closed_form():
    a, b, c = 0.02, 0.005, 0.01
    q = (math.cos(math.pi / 8), 0.0, 0.0, math.sin(math.pi / 8))  # +45 deg about z
    tpl = _tpl_single([0.0, 0.0, 3.0], [0, 1, 2, 3], [1, 0, 0, 0], scales=(a, b, c), quat=q)
    eye = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32)
    p = oracle.project_instance(oracle.OracleScene(_one_instance_scene(tpl, eye, np.zeros((24, 3), np.float32))), 0)
    a, b, c = (float(np.float32(x)) for x in (a, b, c))
    qq = np.array(q, np.float32).astype(np.float64)
    # the float32 quaternion is not exactly 45 deg: build its angle exactly
    ang = 2 * math.atan2(qq[3], qq[0])
    cs, sn = math.cos(ang), math.sin(ang)
    ref = np.array([a * a * cs * cs + b * b * sn * sn, (a * a - b * b) * cs * sn, 0.0,
                    a * a * sn * sn + b * b * cs * cs, 0.0, c * c])
    assert np.abs(p["cov3"][0] - ref).max() < 1e-17
    assert p["cov3"][0][1] > 0  # long axis along (1, 1): positive xy term


def test_means_only_mode_keeps_covariance_under_pose():
    sc = S.single_avatar(n_gauss=256)
    rng = np.random.default_rng(6)
    sc.instances.root[0] = S.yaw_root(0.9, 0.0, 0.0, 0.0).astype(np.float32)
    sc.instances.pose[0] = 0
    a = oracle.project_instance(oracle.OracleScene(sc, skin_mode=1), 0)
    sc.instances.pose[0] = rng.normal(0, 0.5, (24, 3)).astype(np.float32)
    b = oracle.project_instance(oracle.OracleScene(sc, skin_mode=1), 0)
    f = oracle.project_instance(oracle.OracleScene(sc, skin_mode=0), 0)
    assert np.abs(a["cov3"] - b["cov3"]).max() < 1e-15
    assert np.abs(a["mu"] - b["mu"]).max() > 1e-2
    assert np.abs(f["cov3"] - b["cov3"]).max() > 1e-7  # full LBS does rotate them


# ---------------------------------------------------------------------------
# level of detail
# ---------------------------------------------------------------------------

def test_paper_lod_bands_and_counts():
    g = json.load(open(os.path.join(GOLDEN, "paper_lod.json")))
    counts = g["template_counts"]
    frac = np.array([c / counts[0] for c in counts], np.float32)
    lod = S.LodConfig(thresholds=np.array(g["thresholds_m"], np.float32), fractions=frac,
                      scale_mult=np.ones(3, np.float32))
    # camera away from the origin, instance along an oblique direction
    cam = S.look_camera((1.0, 2.0, -3.0), 20.0, 16, 16, yaw_deg=30.0)
    centre = cam.center
    direction = np.array([0.36, -0.48, 0.8])
    for case in g["cases"]:
        d = case["distance_m"]
        tpl = _tpl_single([0, 0, 0], [0, 1, 2, 3], [1, 0, 0, 0])
        pos = centre + d * direction
        root = np.array([[1, 0, 0, pos[0]], [0, 1, 0, pos[1]], [0, 0, 1, pos[2]]], np.float32)
        sc = U.scene_of([tpl], U.instances(1, root[None]), cam, lod)
        os_ = oracle.OracleScene(sc)
        lvl, dist, _ = oracle.instance_level(os_, 0)
        assert abs(dist - d) < 1e-5, case
        assert lvl == case["level"], case
        assert oracle.level_count(os_, lvl, counts[0]) == case["count"], case


def test_lod_threshold_goes_to_coarser_band():
    lod = S.LodConfig(thresholds=np.array([5.0, 10.0], np.float32), fractions=np.array([1, 0.5, 0.25], np.float32),
                      scale_mult=np.ones(3, np.float32))
    for d, want in ((5.0, 1), (10.0, 2), (np.nextafter(np.float32(5.0), np.float32(0)), 0)):
        tpl = _tpl_single([0, 0, 0], [0, 1, 2, 3], [1, 0, 0, 0])
        root = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, d]], np.float32)
        sc = U.scene_of([tpl], U.instances(1, root[None]), U.identity_camera(16, 16, 10.0), lod)
        assert oracle.instance_level(oracle.OracleScene(sc), 0)[0] == want


def test_lod_level_equals_truncated_inflated_template():
    base = S.make_template(1234, 512, 1)
    lod = S.LodConfig(thresholds=np.array([10.0, 30.0], np.float32),
                      fractions=np.array([1.0, 0.25, 0.06], np.float32),
                      scale_mult=np.array([1.0, 2.0, 4.0], np.float32))
    cam = S.look_camera((0.0, 1.0, 0.0), 0.0, 96, 96, vfov_deg=8.0)
    root = S.yaw_root(0.3, 0.0, 0.0, 15.0).astype(np.float32)
    pose = np.random.default_rng(7).normal(0, 0.3, (1, 24, 3)).astype(np.float32)
    sc = U.scene_of([base], U.instances(1, root[None], pose), cam, lod)
    img = oracle.render(oracle.OracleScene(sc))["rgba"]
    n1 = 128
    t2 = S.Template(means=base.means[:n1], scales=base.scales[:n1] * np.float32(2.0),
                    quats=base.quats[:n1], opacity=base.opacity[:n1], sh=base.sh[:n1],
                    skin_idx=base.skin_idx[:n1], skin_w=base.skin_w[:n1],
                    rest_joints=base.rest_joints, parents=base.parents, sh_degree=1)
    sc2 = U.scene_of([t2], U.instances(1, root[None], pose), cam)
    img2 = oracle.render(oracle.OracleScene(sc2))["rgba"]
    assert img[..., 3].max() > 0.5
    assert np.abs(img - img2).max() < 1e-14


# ---------------------------------------------------------------------------
# projection
# ---------------------------------------------------------------------------

def _single_gauss_scene(mu, scales, quat, opacity=0.9, sh=None, size=64, f=80.0, cam=None):
    sh = np.zeros((1, 1, 3)) if sh is None else sh
    tpl = U.template_from([mu], [scales], [quat], [opacity], sh)
    eye = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32)
    cam = cam if cam is not None else U.identity_camera(size, size, f)
    return U.scene_of([tpl], U.instances(1, eye[None]), cam)


def _pinhole(cam, X):
    """Exact pinhole projection of world points X [n,3]."""
    R = np.asarray(cam.R, np.float32).astype(np.float64)
    t = np.asarray(cam.t, np.float32).astype(np.float64)
    Xc = X @ R.T + t
    fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    return np.stack([fx * Xc[:, 0] / Xc[:, 2] + cam.cx, fy * Xc[:, 1] / Xc[:, 2] + cam.cy], 1)


def _tilted_camera():
    return S.look_camera((0.3, 1.2, -0.5), 12.0, 200, 120, vfov_deg=50.0, yaw_deg=9.0)


def test_ewa_covariance_matches_sampled_projection():
    cam = _tilted_camera()
    mu = np.array([0.9, 0.7, 2.8])
    sc = _single_gauss_scene(mu, (0.004, 0.0015, 0.0025), (0.8, 0.3, -0.4, 0.2), cam=cam)
    p = oracle.project_instance(oracle.OracleScene(sc), 0)
    cov3 = p["cov3"][0]
    Sig = np.array([[cov3[0], cov3[1], cov3[2]], [cov3[1], cov3[3], cov3[4]], [cov3[2], cov3[4], cov3[5]]])
    rng = np.random.default_rng(8)
    X = rng.multivariate_normal(p["mu"][0], Sig, size=400000)
    uv = _pinhole(cam, X)
    emp = np.cov(uv.T)
    a, b, c = p["cov2"][0]
    ref = np.array([[a - 0.3, b], [b, c - 0.3]])
    assert np.abs(emp - ref).max() < 0.02 * np.abs(ref).max()
    assert np.abs(p["uv"][0] - _pinhole(cam, p["mu"][0][None])[0]).max() < 1e-9


def _fd_jacobian(cam, X, h=1e-6):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (_pinhole(cam, (X + e)[None])[0] - _pinhole(cam, (X - e)[None])[0]) / (2 * h)
    return J


@pytest.mark.parametrize("where", ["inside", "clamped_x", "clamped_y"])
def test_ewa_covariance_is_linearised_projection(where):
    cam = _tilted_camera()
    R = np.asarray(cam.R, np.float32).astype(np.float64)
    t = np.asarray(cam.t, np.float32).astype(np.float64)
    z = 3.0
    limx = 1.3 * (cam.width / 2) / float(np.float32(cam.fx))
    limy = 1.3 * (cam.height / 2) / float(np.float32(cam.fy))
    xc = {"inside": np.array([0.4 * z, -0.2 * z, z]), "clamped_x": np.array([2.0 * limx * z, 0.1 * z, z]),
          "clamped_y": np.array([0.2 * z, -1.8 * limy * z, z])}[where]
    mu = R.T @ (xc - t)
    scales = (0.05, 0.02, 0.03) if where == "inside" else (0.5, 0.3, 0.4)
    sc = _single_gauss_scene(mu, scales, (0.8, 0.3, -0.4, 0.2), cam=cam)
    p = oracle.project_instance(oracle.OracleScene(sc), 0)
    cov3 = p["cov3"][0]
    Sig = np.array([[cov3[0], cov3[1], cov3[2]], [cov3[1], cov3[3], cov3[4]], [cov3[2], cov3[4], cov3[5]]])
    # the Jacobian is taken where x/z and y/z are clamped to 1.3x the half field
    xcl = xc.copy()
    xcl[0] = np.clip(xc[0] / z, -limx, limx) * z
    xcl[1] = np.clip(xc[1] / z, -limy, limy) * z
    Jw = _fd_jacobian(cam, R.T @ (xcl - t))
    ref = Jw @ Sig @ Jw.T + 0.3 * np.eye(2)
    a, b, c = p["cov2"][0]
    got = np.array([[a, b], [b, c]])
    assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max()


def test_conic_and_radius():
    sc = S.single_avatar(n_gauss=2048)
    p = oracle.project_instance(oracle.OracleScene(sc), 0)
    ok = p["valid"] == 1
    assert ok.sum() > 1000
    for (a, b, c), (A, B, Cc), r in zip(p["cov2"][ok], p["conic"][ok], p["radius"][ok]):
        M = np.array([[a, b], [b, c]])
        assert np.abs(np.array([[A, B], [B, Cc]]) @ M - np.eye(2)).max() < 1e-12
        lam = np.linalg.eigvalsh(M)[-1]
        assert r >= math.ceil(3 * math.sqrt(lam) - 1e-9)
        if ((a - c) / 2) ** 2 + b * b >= 0.1:
            assert r == math.ceil(3 * math.sqrt(lam) - 1e-12)


def test_near_plane_cull():
    for z, ok in ((0.19, 0), (0.21, 1), (-1.0, 0)):
        sc = _single_gauss_scene([0.0, 0.0, z], (0.001, 0.001, 0.001), (1, 0, 0, 0))
        p = oracle.project_instance(oracle.OracleScene(sc), 0)
        assert p["valid"][0] == ok


# ---------------------------------------------------------------------------
# compositing
# ---------------------------------------------------------------------------

def _dc(c):
    """DC coefficient that yields base colour c."""
    return (np.asarray(c, np.float64) - 0.5) * 2 * math.sqrt(math.pi)


def test_isotropic_gaussian_renders_its_analytic_footprint():
    size, f, z, s, o = 64, 80.0, 3.0, 0.08, 0.7
    col = np.array([0.2, 0.5, 0.9])
    sc = _single_gauss_scene([0.0, 0.0, z], (s, s, s), (1, 0, 0, 0), opacity=o,
                             sh=_dc(col)[None, None, :], size=size, f=f)
    img = oracle.render(oracle.OracleScene(sc))["rgba"]
    fz = float(np.float32(f))
    s32, z32, o32 = float(np.float32(s)), float(np.float32(z)), float(np.float32(o))
    sig2 = (fz * s32 / z32) ** 2 + 0.3
    col32 = np.float32(_dc(col)).astype(np.float64) / (2 * math.sqrt(math.pi)) + 0.5
    ys, xs = np.mgrid[0:size, 0:size] + 0.5
    rho2 = (xs - size / 2) ** 2 + (ys - size / 2) ** 2
    alpha = np.minimum(0.99, o32 * np.exp(-rho2 / (2 * sig2)))
    inner = (np.abs(xs - size / 2) <= 3 * math.sqrt(sig2)) & (np.abs(ys - size / 2) <= 3 * math.sqrt(sig2))
    alpha = np.where(alpha >= 1 / 255, alpha, 0.0)
    m = inner
    assert np.abs(img[..., 3][m] - alpha[m]).max() < 1e-12
    for ch in range(3):
        assert np.abs(img[..., ch][m] - col32[ch] * alpha[m]).max() < 1e-12
    far = rho2 > (3 * math.sqrt(sig2 + 0.32) + 2) ** 2 * 2
    assert np.all(img[far] == 0)


def test_support_box_cuts_the_footprint():
    # an opaque wide isotropic splat still has alpha >= 1/255 just outside
    # its square support box: those pixels must stay empty
    size, f, z, s = 96, 100.0, 1.0, 0.1
    sc = _single_gauss_scene([0.0, 0.0, z], (s, s, s), (1, 0, 0, 0), opacity=1.0,
                             sh=_dc([1.0, 1.0, 1.0])[None, None, :], size=size, f=f)
    img = oracle.render(oracle.OracleScene(sc))["rgba"][..., 3]
    p = oracle.project_instance(oracle.OracleScene(sc), 0)
    r = int(p["radius"][0])
    sig2 = p["cov2"][0][0]
    ys, xs = np.mgrid[0:size, 0:size] + 0.5
    dx, dy = xs - size / 2, ys - size / 2
    alpha = np.minimum(0.99, np.exp(-(dx * dx + dy * dy) / (2 * sig2)))
    outside = (np.maximum(np.abs(dx), np.abs(dy)) > r) & (alpha >= 1 / 255)
    assert outside.sum() > 10
    assert np.all(img[outside] == 0)
    inside = (np.maximum(np.abs(dx), np.abs(dy)) <= r) & (alpha >= 1 / 255)
    assert np.abs(img[inside] - alpha[inside]).max() < 1e-12


def test_two_layers_closed_form_and_depth_order():
    cols = [np.array([0.9, 0.1, 0.1]), np.array([0.1, 0.2, 0.8])]
    for order in ((0, 1), (1, 0)):
        zs = [2.0, 3.0]
        means = [[0.0, 0.0, zs[k]] for k in order]
        sh = np.stack([_dc(cols[k])[None, :] for k in order])
        ops = [0.6, 0.8]
        tpl = U.template_from(means, [(0.05,) * 3, (0.05,) * 3], [(1, 0, 0, 0)] * 2,
                              [ops[k] for k in order], sh)
        eye = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32)
        sc = U.scene_of([tpl], U.instances(1, eye[None]), U.identity_camera(32, 32, 50.0))
        img = oracle.render(oracle.OracleScene(sc))["rgba"]
        p = oracle.project_instance(oracle.OracleScene(sc), 0)
        # pixel (16,16): centre (16.5,16.5), offset (0.5,0.5) from both means
        a = []
        for k in (0, 1):
            g = order.index(k)
            A, B, Cc = p["conic"][g]
            q = -0.5 * (A * 0.25 + Cc * 0.25) - B * 0.25
            a.append(min(0.99, p["opacity"][g] * math.exp(q)))
        c0, c1 = p["rgb"][order.index(0)], p["rgb"][order.index(1)]
        ref = c0 * a[0] + c1 * a[1] * (1 - a[0])
        assert np.abs(img[16, 16, :3] - ref).max() < 1e-14
        assert abs(img[16, 16, 3] - (1 - (1 - a[0]) * (1 - a[1]))) < 1e-14


def test_stop_rule_before_transmittance_below_1e4():
    # three nearly opaque layers: the third would leave T = 1e-6 < 1e-4
    cols = [np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])]
    means = [[0.0, 0.0, 2.0 + k] for k in range(3)]
    sh = np.stack([_dc(c)[None, :] for c in cols])
    tpl = U.template_from(means, [(1.0,) * 3] * 3, [(1, 0, 0, 0)] * 3, [1.0, 1.0, 1.0], sh)
    eye = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32)
    sc = U.scene_of([tpl], U.instances(1, eye[None]), U.identity_camera(16, 16, 20.0))
    r = oracle.render(oracle.OracleScene(sc))
    px = r["rgba"][8, 8]
    p = oracle.project_instance(oracle.OracleScene(sc), 0)
    a = [min(0.99, math.exp(-0.5 * (p["conic"][k][0] * 0.25 + p["conic"][k][2] * 0.25) - p["conic"][k][1] * 0.25))
         for k in range(3)]
    assert a[0] == 0.99 and a[1] == 0.99
    c = p["rgb"]
    ref = c[0] * a[0] + c[1] * a[1] * (1 - a[0])
    assert np.abs(px[:3] - ref).max() < 1e-14
    assert abs(px[3] - (1 - (1 - a[0]) * (1 - a[1]))) < 1e-14
    assert r["ncontrib"][8, 8] == 2


def test_transmittance_invariants():
    sc = U.random_small_scene(9, n_gauss=200, n_inst=4, size=48, sh_degree=2)
    r = oracle.render(oracle.OracleScene(sc))
    A = r["rgba"][..., 3]
    assert A.max() > 0.9
    assert np.abs(r["wsum"] - A).max() < 1e-12       # sum alpha_i T_i = 1 - T_final
    assert A.max() < 1 - 1e-4 * 0.999                 # T never drops below 1e-4
    # a layer placed behind everything never lowers coverage (T monotone)
    far = S.yaw_root(0.0, 0.0, 0.0, 6.0).astype(np.float32)
    inst2 = U.instances(5, np.concatenate([sc.instances.root, far[None]]),
                        np.concatenate([sc.instances.pose, np.zeros((1, 24, 3), np.float32)]),
                        np.zeros(5, np.int32))
    sc2 = U.scene_of(sc.templates, inst2, sc.camera)
    A2 = oracle.render(oracle.OracleScene(sc2))["rgba"][..., 3]
    assert np.all(A2 >= A - 1e-15)
    assert (A2 > A + 1e-6).any()


def _brute_force(sc):
    """Composite every splat at every pixel with no support box."""
    os_ = oracle.OracleScene(sc)
    splats = []
    for inst in range(sc.instances.n):
        p = oracle.project_instance(os_, inst)
        for g in np.nonzero(p["valid"])[0]:
            splats.append((p["depth"][g], inst, g, p["uv"][g], p["conic"][g], p["opacity"][g],
                           p["rgb"][g], p["radius"][g]))
    splats.sort(key=lambda s: (s[0], s[1], s[2]))
    W, H = sc.camera.width, sc.camera.height
    img = np.zeros((H, W, 4))
    box_matters = np.zeros((H, W), bool)
    for j in range(H):
        for i in range(W):
            T, Cc = 1.0, np.zeros(3)
            for d, inst, g, uv, con, o, rgb, r in splats:
                dx, dy = i + 0.5 - uv[0], j + 0.5 - uv[1]
                q = -0.5 * (con[0] * dx * dx + con[2] * dy * dy) - con[1] * dx * dy
                if q > 0:
                    continue
                a = min(0.99, o * math.exp(q))
                if a < 1 / 255:
                    continue
                if abs(dx) > r or abs(dy) > r:
                    box_matters[j, i] = True
                Tn = T * (1 - a)
                if Tn < 1e-4:
                    break
                Cc += rgb * a * T
                T = Tn
            img[j, i, :3] = Cc
            img[j, i, 3] = 1 - T
    return img, box_matters


def test_brute_force_agrees_where_the_support_box_is_irrelevant():
    sc = U.random_small_scene(10, n_gauss=40, n_inst=2, size=24, sh_degree=1)
    ref, box_matters = _brute_force(sc)
    got = oracle.render(oracle.OracleScene(sc))["rgba"]
    ok = ~box_matters
    assert ok.mean() > 0.5
    assert ref[..., 3].max() > 0.5
    assert np.abs(got[ok] - ref[ok]).max() < 1e-13


def test_rigid_world_motion_leaves_image_unchanged_in_root_frame():
    sc = U.random_small_scene(11, n_gauss=120, n_inst=3, size=40, sh_degree=3)
    base = oracle.render(oracle.OracleScene(sc))["rgba"]
    # move every root and the camera by the same rigid motion Q (world)
    Q = S.yaw_root(0.8, 0.5, 0.0, -1.0)
    Qr, Qt = Q[:, :3], Q[:, 3]
    roots = []
    for r in sc.instances.root.astype(np.float64):
        roots.append(np.concatenate([Qr @ r[:, :3], (Qr @ r[:, 3] + Qt)[:, None]], 1))
    R = np.asarray(sc.camera.R, np.float64)
    t = np.asarray(sc.camera.t, np.float64)
    cam = S.Camera(R=(R @ Qr.T).astype(np.float32), t=(t - R @ Qr.T @ Qt).astype(np.float32),
                   fx=sc.camera.fx, fy=sc.camera.fy, cx=sc.camera.cx, cy=sc.camera.cy,
                   width=sc.camera.width, height=sc.camera.height)
    sc2 = U.scene_of(sc.templates, U.instances(3, np.array(roots), sc.instances.pose), cam)
    moved = oracle.render(oracle.OracleScene(sc2))["rgba"]
    # inputs are rounded to float32 after the motion: compare loosely
    assert base[..., 3].max() > 0.5
    assert np.abs(moved - base).max() < 2e-4
    # the world-frame option does change the colours under the same motion
    w0 = oracle.render(oracle.OracleScene(sc, sh_frame=1))["rgba"]
    w1 = oracle.render(oracle.OracleScene(sc2, sh_frame=1))["rgba"]
    assert np.abs(w1 - w0).max() > 1e-2


def test_view_dependent_colour_and_clamp():
    # degree-1 colour of a Gaussian seen along a known direction: the basis
    # comes from scipy's complex SH; the view direction runs from the camera
    # centre to the mean, here expressed in the instance root frame
    cam = S.look_camera((0.4, 0.3, -1.0), 0.0, 32, 32)
    mu = np.array([0.1, -0.2, 2.0])
    yaw = 0.6
    root = S.yaw_root(yaw, 0.0, 0.0, 0.0).astype(np.float32)
    coef = np.zeros((1, 4, 3))
    coef[0, 1:4, 0] = [0.7, -0.4, 0.9]   # red uses degree 1
    coef[0, 1:4, 1] = [-3.0, -3.0, -3.0]  # green goes negative: clamped to 0
    tpl = U.template_from([mu], [(0.01,) * 3], [(1, 0, 0, 0)], [0.8], coef)
    sc = U.scene_of([tpl], U.instances(1, root[None]), cam)
    p = oracle.project_instance(oracle.OracleScene(sc), 0)
    assert p["valid"][0] == 1
    mu32 = np.float32(mu).astype(np.float64)
    world = root[:, :3].astype(np.float64) @ mu32 + root[:, 3]
    d = world - cam.center
    d = root[:, :3].astype(np.float64).T @ d
    d /= np.linalg.norm(d)
    Y = np.array([_sh_ref(1, m, d[None])[0] for m in (-1, 0, 1)])
    c32 = np.float32(coef[0, 1:4, 0]).astype(np.float64)
    assert abs(p["rgb"][0][0] - (0.5 + Y @ c32)) < 1e-12
    assert p["rgb"][0][1] == 0.0
    assert abs(p["rgb"][0][2] - 0.5) < 1e-15


def test_degree0_colour_is_view_independent():
    sc = S.single_avatar(n_gauss=256)
    roots = np.stack([S.yaw_root(a, 0, 0, 0) for a in (0.0, 1.0, 2.5)]).astype(np.float32)
    inst = U.instances(3, roots, np.repeat(sc.instances.pose, 3, 0))
    sc2 = U.scene_of(sc.templates, inst, sc.camera)
    os_ = oracle.OracleScene(sc2, sh_frame=1)
    cols = [oracle.project_instance(os_, i)["rgb"] for i in range(3)]
    ok = np.all([oracle.project_instance(os_, i)["valid"] for i in range(3)], 0).astype(bool)
    assert ok.sum() > 100
    assert np.abs(cols[0][ok] - cols[1][ok]).max() < 1e-15
    assert np.abs(cols[0][ok] - cols[2][ok]).max() < 1e-15


def test_pixel_centre_convention():
    # a tiny Gaussian placed on the ray through the centre of pixel (10, 5)
    f, z = 40.0, 2.0
    cam = U.identity_camera(32, 16, f)
    fz = float(np.float32(f))
    x = (10.5 - 16) * z / fz
    y = (5.5 - 8) * z / fz
    sc = _single_gauss_scene([x, y, z], (1e-4,) * 3, (1, 0, 0, 0), opacity=0.9,
                             sh=_dc([1.0, 1.0, 1.0])[None, None, :], cam=cam)
    img = oracle.render(oracle.OracleScene(sc))["rgba"][..., 3]
    j, i = np.unravel_index(np.argmax(img), img.shape)
    assert (i, j) == (10, 5)
    assert abs(img[5, 9] - img[5, 11]) < 1e-6 and abs(img[4, 10] - img[6, 10]) < 1e-6


def test_tile_lists_agree_with_per_pixel_membership():
    sc = U.random_small_scene(12, n_gauss=60, n_inst=2, size=40, sh_degree=0)
    os_ = oracle.OracleScene(sc)
    lists = oracle.tile_lists(os_, tile=16)
    W = H = 40
    members = {}
    depth = {}
    for inst in range(2):
        p = oracle.project_instance(os_, inst)
        for g in np.nonzero(p["valid"])[0]:
            key = (inst << 32) | int(g)
            depth[key] = p["depth"][g]
            u, v = p["uv"][g]
            r = p["radius"][g]
            for j in range(H):
                for i in range(W):
                    if abs(i + 0.5 - u) <= r and abs(j + 0.5 - v) <= r:
                        members.setdefault((j // 16) * 3 + i // 16, set()).add(key)
    assert set(lists) == set(members)
    for t, keys in lists.items():
        assert set(keys.tolist()) == members[t]
        d = [depth[k] for k in keys.tolist()]
        assert all(d[k] <= d[k + 1] for k in range(len(d) - 1))


# ---------------------------------------------------------------------------
# chosen LoD subsets and per-Gaussian contribution sums
# ---------------------------------------------------------------------------

def _paper_lod(mults=(1.0, 2.0, 4.0)):
    return S.LodConfig(thresholds=np.array([10.0, 30.0], np.float32),
                       fractions=np.array([1.0, 0.25, 0.06], np.float32),
                       scale_mult=np.array(mults, np.float32))


def test_lod_subset_equals_template_of_those_gaussians():
    """A level restricted to a chosen subset renders exactly like a template
    made of those Gaussians (in the subset's order) with the level's scale
    multiplier applied."""
    base = S.make_template(4321, 512, 1)
    cam = S.look_camera((0.0, 1.0, 0.0), 0.0, 96, 96, vfov_deg=8.0)
    root = S.yaw_root(0.7, 0.0, 0.0, 15.0).astype(np.float32)       # band 1 (10..30 m)
    pose = np.random.default_rng(8).normal(0, 0.3, (1, 24, 3)).astype(np.float32)
    idx = np.random.default_rng(9).permutation(512)[:90]
    sc = U.scene_of([base], U.instances(1, root[None], pose), cam, _paper_lod())
    os_ = oracle.OracleScene(sc, subsets={(0, 1): idx})
    assert oracle.level_size(os_, 0, 1) == 90
    assert oracle.level_size(os_, 0, 2) == round(0.06 * 512)
    img = oracle.render(os_)["rgba"]
    t2 = S.Template(means=base.means[idx], scales=base.scales[idx] * np.float32(2.0),
                    quats=base.quats[idx], opacity=base.opacity[idx], sh=base.sh[idx],
                    skin_idx=base.skin_idx[idx], skin_w=base.skin_w[idx],
                    rest_joints=base.rest_joints, parents=base.parents, sh_degree=1)
    img2 = oracle.render(oracle.OracleScene(U.scene_of([t2], U.instances(1, root[None], pose), cam)))["rgba"]
    assert img[..., 3].max() > 0.3
    assert np.abs(img - img2).max() < 1e-14
    p = oracle.project_instance(os_, 0)
    assert p["count"] == 90 and p["level"] == 1
    # a subset equal to the prefix changes nothing
    n1 = round(0.25 * 512)
    os3 = oracle.OracleScene(sc, subsets={(0, 1): np.arange(n1)})
    img3 = oracle.render(os3)["rgba"]
    img4 = oracle.render(oracle.OracleScene(sc))["rgba"]
    assert np.abs(img3 - img4).max() == 0.0


def test_contributions_sum_to_the_alpha_channel():
    """sum over Gaussians of sum over pixels of alpha T = sum over pixels of
    (1 - final T); every contribution is non-negative."""
    sc = U.random_small_scene(21, n_gauss=150, n_inst=4, size=40, sh_degree=1)
    r = oracle.render(oracle.OracleScene(sc), contrib=True)
    c = r["contrib"]
    assert c.shape == (150,)
    assert c.min() >= 0.0 and (c > 0).sum() > 50
    assert abs(c.sum() - r["rgba"][..., 3].sum()) < 1e-9 * max(1.0, c.sum())


def test_contribution_closed_form_for_two_layers():
    """Front splat f, back splat b: contrib_f = sum A_f, contrib_b =
    sum A_b (1 - A_f), with A_x the alpha channel of x rendered alone (no
    pixel reaches the stop rule or the 0.99 clamp here)."""
    means = [[0.0, 0.0, 2.0], [0.01, -0.01, 2.6]]
    scales = [[0.03, 0.02, 0.02], [0.04, 0.03, 0.03]]
    quats = [[1, 0, 0, 0], [0.9, 0.1, 0.2, 0.1]]
    op = [0.6, 0.7]
    sh = np.full((2, 1, 3), 0.2, np.float32)
    cam = U.identity_camera(48, 48, f=60.0)

    def scene(sel):
        t = U.template_from(np.asarray(means)[sel], np.asarray(scales)[sel], np.asarray(quats)[sel],
                            np.asarray(op)[sel], sh[sel])
        return U.scene_of([t], U.instances(1), cam)

    both = oracle.render(oracle.OracleScene(scene([0, 1])), contrib=True)
    Af = oracle.render(oracle.OracleScene(scene([0])))["rgba"][..., 3]
    Ab = oracle.render(oracle.OracleScene(scene([1])))["rgba"][..., 3]
    assert Af.max() < 0.99 and Ab.max() < 0.99
    assert abs(both["contrib"][0] - Af.sum()) < 1e-12 * Af.sum()
    assert abs(both["contrib"][1] - (Ab * (1 - Af)).sum()) < 1e-12 * Ab.sum()
    assert both["contrib"][1] < Ab.sum() * 0.9          # the front layer hides part of the back one


def test_contribution_lands_on_the_template_gaussian():
    """Two templates; level 0 of template 1 restricted to one Gaussian k:
    only entry n0 + k of the concatenated array receives weight."""
    ta = S.make_template(51, 40, 0)
    tb = S.make_template(52, 30, 0)
    cam = S.look_camera((0.0, 1.0, 0.0), 0.0, 64, 64, vfov_deg=40.0)
    roots = np.stack([S.yaw_root(0.0, 0.0, 0.0, 3.0), S.yaw_root(0.5, 0.0, 0.0, 3.0)]).astype(np.float32)
    inst = U.instances(2, roots, np.zeros((2, 24, 3), np.float32), template_id=[0, 1])
    sc = U.scene_of([ta, tb], inst, cam)
    k = 17
    os_ = oracle.OracleScene(sc, subsets={(0, 0): [], (1, 0): [k]})
    r = oracle.render(os_, contrib=True)
    c = r["contrib"]
    assert c.shape == (70,)
    nz = np.nonzero(c)[0]
    assert list(nz) == [40 + k]
    assert abs(c[40 + k] - r["rgba"][..., 3].sum()) < 1e-12


def test_direct_covariance_matches_scales_and_rotation():
    """A covariance given directly renders like the scales and quaternion
    it comes from: exactly for an axis-aligned Gaussian with dyadic scales,
    to float32 rounding of the covariance otherwise."""
    import dataclasses
    base = S.make_template(91, 300, 1)
    cam = S.look_camera((0.0, 1.0, -2.5), 0.0, 64, 64, vfov_deg=50.0)
    root = S.yaw_root(math.pi, 0.0, 0.0, 0.0).astype(np.float32)[None]
    pose = np.random.default_rng(3).normal(0, 0.3, (1, 24, 3)).astype(np.float32)
    lod = S.LodConfig(thresholds=np.zeros(0, np.float32), fractions=np.ones(1, np.float32),
                      scale_mult=np.array([1.5], np.float32))
    q = base.quats.astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    Rq = np.stack([oracle.quat_to_rot(x) for x in q])
    s2 = base.scales.astype(np.float64) ** 2
    C = np.einsum("nik,nk,njk->nij", Rq, s2, Rq)
    t2 = dataclasses.replace(base)
    t2.cov = np.stack([C[:, 0, 0], C[:, 0, 1], C[:, 0, 2], C[:, 1, 1], C[:, 1, 2], C[:, 2, 2]], 1).astype(np.float32)
    a = oracle.render(oracle.OracleScene(U.scene_of([base], U.instances(1, root, pose), cam, lod)))["rgba"]
    b = oracle.render(oracle.OracleScene(U.scene_of([t2], U.instances(1, root, pose), cam, lod)))["rgba"]
    assert a[..., 3].max() > 0.5
    assert np.abs(a - b).max() < 1e-4
    # axis-aligned, dyadic scales: the covariance is exact in float32
    t3 = U.template_from([[0.0, 1.0, 0.0]], [[0.03125, 0.0625, 0.015625]], [[1, 0, 0, 0]], [0.8],
                         np.full((1, 1, 3), 0.4, np.float32))
    t4 = dataclasses.replace(t3)
    t4.cov = np.array([[0.03125 ** 2, 0, 0, 0.0625 ** 2, 0, 0.015625 ** 2]], np.float32)
    c = oracle.render(oracle.OracleScene(U.scene_of([t3], U.instances(1, root, pose), cam, lod)))["rgba"]
    d = oracle.render(oracle.OracleScene(U.scene_of([t4], U.instances(1, root, pose), cam, lod)))["rgba"]
    assert c[..., 3].max() > 0.3
    assert np.abs(c - d).max() < 1e-14


def test_windowed_tile_lists_equal_the_full_lists_on_the_window():
    """The array-operation form restricted to a tile window returns exactly
    the lists of the plain per-splat loop for those tiles."""
    sc = U.random_small_scene(21, n_gauss=120, n_inst=3, size=72, sh_degree=0)
    os_ = oracle.OracleScene(sc)
    full = oracle.tile_lists(os_, tile=16)
    tw = (72 + 15) // 16
    lists, info = oracle.tile_lists_window(os_, 1, 1, 3, 2)
    want = {t: k for t, k in full.items() if 1 <= t % tw < 4 and 1 <= t // tw < 3}
    assert set(lists) == set(want) and len(want) > 2
    for t in want:
        assert np.array_equal(lists[t], want[t])
    assert all(k in info for ks in lists.values() for k in ks.tolist())
