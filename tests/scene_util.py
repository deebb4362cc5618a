"""Hand-built tiny scenes for the pins and parity tests (inputs only)."""
from __future__ import annotations

import math

import numpy as np

from paper_2501_17792_gb300 import scene as S


def template_from(means, scales, quats, opacity, sh, *, skin_idx=None, skin_w=None,
                  rest_joints=None, sh_degree=None) -> S.Template:
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    sh = np.asarray(sh, np.float32)
    if sh.ndim == 2:
        sh = sh[:, None, :]
    deg = int(round(math.sqrt(sh.shape[1]))) - 1 if sh_degree is None else sh_degree
    if skin_idx is None:
        skin_idx = np.tile(np.array([0, 1, 2, 3], np.uint8), (n, 1))
    if skin_w is None:
        skin_w = np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1))
    if rest_joints is None:
        rest_joints = S._REST.astype(np.float32)
    return S.Template(means=means, scales=np.asarray(scales, np.float32).reshape(n, 3),
                      quats=np.asarray(quats, np.float32).reshape(n, 4),
                      opacity=np.asarray(opacity, np.float32).reshape(n), sh=sh,
                      skin_idx=np.asarray(skin_idx, np.uint8).reshape(n, 4),
                      skin_w=np.asarray(skin_w, np.float32).reshape(n, 4),
                      rest_joints=np.asarray(rest_joints, np.float32).reshape(24, 3),
                      parents=S.PARENTS.copy(), sh_degree=deg)


def identity_camera(width, height, f, cx=None, cy=None, near=0.2) -> S.Camera:
    """Camera at the world origin, axes equal to the world axes (x right,
    y down, z forward)."""
    return S.Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=float(np.float32(f)),
                    fy=float(np.float32(f)), cx=width / 2.0 if cx is None else cx,
                    cy=height / 2.0 if cy is None else cy, width=width, height=height, near=near)


def instances(n, roots=None, poses=None, template_id=None) -> S.Instances:
    if roots is None:
        roots = np.tile(np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32), (n, 1, 1))
    if poses is None:
        poses = np.zeros((n, 24, 3), np.float32)
    if template_id is None:
        template_id = np.zeros(n, np.int32)
    return S.Instances(template_id=np.asarray(template_id, np.int32),
                       root=np.asarray(roots, np.float32).reshape(n, 3, 4),
                       pose=np.asarray(poses, np.float32).reshape(n, 24, 3))


def scene_of(templates, inst, cam, lod=None, name="tiny") -> S.Scene:
    return S.Scene(templates=list(templates), instances=inst, camera=cam,
                   lod=lod if lod is not None else S.single_lod(), name=name)


def random_small_scene(seed, n_gauss=64, n_inst=3, size=48, sh_degree=1, spread=0.25):
    """A few instances of one small random template in front of an identity
    camera; means within `spread` m of (0, 0, 2.5)."""
    rng = np.random.default_rng(seed)
    k = (sh_degree + 1) ** 2
    means = rng.uniform(-spread, spread, (n_gauss, 3)) + np.array([0.0, 0.0, 0.0])
    scales = np.exp(rng.normal(math.log(0.03), 0.4, (n_gauss, 3)))
    q = rng.standard_normal((n_gauss, 4))
    op = 1.0 / (1.0 + np.exp(-rng.standard_normal(n_gauss)))
    sh = 0.3 * rng.standard_normal((n_gauss, k, 3))
    idx = np.stack([rng.choice(24, 4, replace=False) for _ in range(n_gauss)])
    w = rng.random((n_gauss, 4))
    w /= w.sum(1, keepdims=True)
    rest = np.zeros((24, 3), np.float32) + rng.uniform(-0.2, 0.2, (24, 3)).astype(np.float32)
    tpl = template_from(means, scales, q, op, sh, skin_idx=idx, skin_w=w, rest_joints=rest)
    roots = []
    for i in range(n_inst):
        yaw = rng.uniform(0, 2 * math.pi)
        roots.append(S.yaw_root(yaw, rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3),
                                2.5 + rng.uniform(-0.3, 0.3)))
    poses = rng.normal(0, 0.3, (n_inst, 24, 3))
    cam = identity_camera(size, size, f=size * 1.2)
    return scene_of([tpl], instances(n_inst, roots, poses), cam)
