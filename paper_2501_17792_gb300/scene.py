"""Seeded synthetic crowd scenes shaped like CrowdSplat's workload.

This module only draws inputs. It holds none of the method's arithmetic
(no skinning, projection, colour evaluation or compositing); both the CUDA
path and the CPU oracle receive the arrays it returns.

What it draws (CrowdSplat Sec. 2 describes the real inputs: avatar
templates reconstructed from video, duplicated to 3,500 characters on a grid,
animated by 15 motion sequences, a static camera 3 m from the first row;
none of those assets exist here, so procedural stand-ins take their place):

* a 24-joint capsule body with the kinematic topology of a common
  parametric human body (pelvis, spine x3, neck, head; per side collar,
  shoulder, elbow, wrist, hand, hip, knee, ankle, foot);
* Gaussian means uniform on the capsule surfaces, top-4 bone-distance skin
  weights, log-normal scales, random unit quaternions, sigmoid-normal
  opacities and SH colour coefficients;
* instance layouts (a jittered ground grid with random yaw and template),
  axis-angle joint poses N(0, 0.3 rad) and pinhole cameras.

Coordinates: metres, right-handed, world y up.  Templates stand on y = 0,
face +z.  Cameras use the OpenCV convention (x right, y down, z forward).
Every array is float32 (the GPU's input precision); the oracle promotes the
same values to float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_JOINTS = 24

# Kinematic tree: parent of each joint (-1 for the root).
PARENTS = np.array(
    [-1, 0, 0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 9, 9, 12, 13, 14, 16, 17, 18, 19, 20, 21],
    dtype=np.int32,
)

JOINT_NAMES = (
    "pelvis", "l_hip", "r_hip", "spine1", "l_knee", "r_knee", "spine2",
    "l_ankle", "r_ankle", "spine3", "l_foot", "r_foot", "neck", "l_collar",
    "r_collar", "head", "l_shoulder", "r_shoulder", "l_elbow", "r_elbow",
    "l_wrist", "r_wrist", "l_hand", "r_hand",
)

# Rest (T-pose) joint positions of the unscaled body, metres.
_REST = np.array(
    [
        [0.000, 0.950, 0.000],   # pelvis
        [0.090, 0.880, 0.000],   # l_hip
        [-0.090, 0.880, 0.000],  # r_hip
        [0.000, 1.050, -0.010],  # spine1
        [0.100, 0.500, 0.010],   # l_knee
        [-0.100, 0.500, 0.010],  # r_knee
        [0.000, 1.180, -0.010],  # spine2
        [0.100, 0.080, -0.020],  # l_ankle
        [-0.100, 0.080, -0.020], # r_ankle
        [0.000, 1.320, -0.010],  # spine3
        [0.100, 0.030, 0.110],   # l_foot
        [-0.100, 0.030, 0.110],  # r_foot
        [0.000, 1.500, -0.010],  # neck
        [0.070, 1.420, -0.010],  # l_collar
        [-0.070, 1.420, -0.010], # r_collar
        [0.000, 1.600, 0.010],   # head
        [0.180, 1.430, -0.010],  # l_shoulder
        [-0.180, 1.430, -0.010], # r_shoulder
        [0.450, 1.430, -0.010],  # l_elbow
        [-0.450, 1.430, -0.010], # r_elbow
        [0.700, 1.430, -0.010],  # l_wrist
        [-0.700, 1.430, -0.010], # r_wrist
        [0.780, 1.430, -0.010],  # l_hand
        [-0.780, 1.430, -0.010], # r_hand
    ],
    dtype=np.float64,
)

# Terminal segment offsets for leaf joints (no children): feet, head, hands.
_TERMINAL = {
    10: np.array([0.0, 0.0, 0.08]),
    11: np.array([0.0, 0.0, 0.08]),
    15: np.array([0.0, 0.15, 0.0]),
    22: np.array([0.08, 0.0, 0.0]),
    23: np.array([-0.08, 0.0, 0.0]),
}

# Capsule radius of the segment owned by each joint (metres).
_RADIUS = np.array(
    [0.11, 0.085, 0.085, 0.13, 0.055, 0.055, 0.14, 0.045, 0.045, 0.15,
     0.04, 0.04, 0.05, 0.06, 0.06, 0.10, 0.05, 0.05, 0.04, 0.04,
     0.035, 0.035, 0.04, 0.04],
    dtype=np.float64,
)


@dataclasses.dataclass
class Template:
    """One avatar template in structure-of-arrays form (float32 unless noted).

    means [N,3] metres; scales [N,3] metres (activated); quats [N,4] (w,x,y,z);
    opacity [N] in (0,1); sh [N,K,3] with K = (sh_degree+1)^2;
    skin_idx [N,4] uint8 joint ids; skin_w [N,4] summing to 1;
    rest_joints [24,3]; parents [24] int32.
    Stored order is iid, so any prefix is a uniform random subset (the LoD
    levels are prefixes).
    """

    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    skin_idx: np.ndarray
    skin_w: np.ndarray
    rest_joints: np.ndarray
    parents: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


@dataclasses.dataclass
class Camera:
    """Pinhole camera: world->camera rotation R [3,3], translation t [3]
    (x_cam = R x_world + t), focal lengths and principal point in pixels,
    image size.  Pixel (i, j) has its centre at (i + 0.5, j + 0.5)."""

    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2
    # window of a larger image (0 = no window): this camera renders pixels
    # [win_x0, win_x0 + width) x [win_y0, win_y0 + height) of a full_width x
    # full_height image whose principal point is (cx, cy)
    win_x0: int = 0
    win_y0: int = 0
    full_width: int = 0
    full_height: int = 0

    @property
    def center(self) -> np.ndarray:
        return (-self.R.astype(np.float64).T @ self.t.astype(np.float64))


@dataclasses.dataclass
class Instances:
    """Per-frame instance state: template id [I] int32, root [I,3,4] rigid
    (row-major [R|t], template local -> world), joint poses [I,24,3]
    axis-angle radians."""

    template_id: np.ndarray
    root: np.ndarray
    pose: np.ndarray

    @property
    def n(self) -> int:
        return int(self.template_id.shape[0])


@dataclasses.dataclass
class LodConfig:
    """Distance LoD: thresholds [L-1] (metres, ascending), fractions [L],
    scale multipliers [L]."""

    thresholds: np.ndarray
    fractions: np.ndarray
    scale_mult: np.ndarray


def _segments(rest: np.ndarray):
    """Segments (a, b, owner joint, radius) of the capsule body."""
    segs = []
    children = {j: [] for j in range(N_JOINTS)}
    for j in range(1, N_JOINTS):
        children[int(PARENTS[j])].append(j)
    for j in range(N_JOINTS):
        if children[j]:
            for c in children[j]:
                segs.append((rest[j], rest[c], j, _RADIUS[j]))
        else:
            segs.append((rest[j], rest[j] + _TERMINAL[j] * (rest[15, 1] / 1.6),
                         j, _RADIUS[j]))
    return segs


def _sample_capsules(rng: np.random.Generator, segs, n: int) -> np.ndarray:
    """n points uniform (by area) on the union of capsule surfaces."""
    areas = np.array([2 * math.pi * r * np.linalg.norm(b - a) + 4 * math.pi * r * r
                      for a, b, _, r in segs])
    which = rng.choice(len(segs), size=n, p=areas / areas.sum())
    out = np.empty((n, 3))
    u = rng.random(n)
    phi = rng.random(n) * 2 * math.pi
    sph = rng.standard_normal((n, 3))
    sph /= np.linalg.norm(sph, axis=1, keepdims=True)
    for s, (a, b, _, r) in enumerate(segs):
        m = which == s
        if not m.any():
            continue
        axis = b - a
        length = np.linalg.norm(axis)
        z = axis / length
        helper = np.array([1.0, 0, 0]) if abs(z[0]) < 0.9 else np.array([0, 1.0, 0])
        x = np.cross(z, helper)
        x /= np.linalg.norm(x)
        y = np.cross(z, x)
        cyl_area = 2 * math.pi * r * length
        cap_area = 4 * math.pi * r * r
        on_cyl = u[m] < cyl_area / (cyl_area + cap_area)
        idx = np.nonzero(m)[0]
        # cylinder part
        ic = idx[on_cyl]
        t = rng.random(ic.size) * length
        ang = phi[ic]
        out[ic] = (a + np.outer(t, z) + r * (np.outer(np.cos(ang), x) + np.outer(np.sin(ang), y)))
        # caps: uniform on a sphere, hemisphere by the axial sign
        ik = idx[~on_cyl]
        d = sph[ik]
        along = d @ z
        base = np.where(along[:, None] >= 0, b, a)
        out[ik] = base + r * d
    return out


def _point_segment_dist(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    ab = b - a
    t = np.clip(((p - a) @ ab) / (ab @ ab), 0.0, 1.0)
    q = a + t[:, None] * ab
    return np.linalg.norm(p - q, axis=1)


def make_template(seed: int, n: int, sh_degree: int, *, sh_sigma: float = 0.3,
                  base_colour_uniform: bool = False) -> Template:
    """One procedural capsule-body template (seed-fixed).

    Scales: log-normal per axis with log-std 0.5 and mean 0.01 m.  Opacity:
    sigmoid of N(0,1).  SH coefficients N(0, sh_sigma) for every (k, channel),
    or, with base_colour_uniform and degree 0, a DC coefficient that makes
    the base colour uniform on (0,1) (DC = (c - 0.5) * 2 sqrt(pi), the
    inverse of the degree-0 basis constant).
    """
    rng = np.random.default_rng(seed)
    height_scale = rng.uniform(0.9, 1.1)
    rest = _REST * height_scale
    segs = _segments(rest)
    means = _sample_capsules(rng, segs, n)
    # top-4 skinning weights by distance to each joint's owned segments
    dist = np.full((n, N_JOINTS), np.inf)
    for a, b, owner, _ in segs:
        dist[:, owner] = np.minimum(dist[:, owner], _point_segment_dist(means, a, b))
    idx = np.argsort(dist, axis=1, kind="stable")[:, :4]
    d4 = np.take_along_axis(dist, idx, axis=1)
    w = (d4 + 1e-3) ** -2.0
    w /= w.sum(axis=1, keepdims=True)
    sigma_log = 0.5
    mu_log = math.log(0.01) - 0.5 * sigma_log ** 2
    scales = np.exp(mu_log + sigma_log * rng.standard_normal((n, 3)))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.standard_normal(n)))
    k = (sh_degree + 1) ** 2
    if base_colour_uniform:
        sh = np.zeros((n, k, 3))
        sh[:, 0, :] = (rng.random((n, 3)) - 0.5) * (2.0 * math.sqrt(math.pi))
        if k > 1:
            sh[:, 1:, :] = sh_sigma * rng.standard_normal((n, k - 1, 3))
    else:
        sh = sh_sigma * rng.standard_normal((n, k, 3))
    w32 = w.astype(np.float32)
    return Template(
        means=means.astype(np.float32),
        scales=scales.astype(np.float32),
        quats=q.astype(np.float32),
        opacity=opacity.astype(np.float32),
        sh=sh.astype(np.float32),
        skin_idx=idx.astype(np.uint8),
        skin_w=w32,
        rest_joints=rest.astype(np.float32),
        parents=PARENTS.copy(),
        sh_degree=sh_degree,
    )


def yaw_root(yaw: float, x: float, y: float, z: float) -> np.ndarray:
    """Rigid 3x4 root: rotation by `yaw` about world +y, then translation."""
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, 0.0, s, x], [0.0, 1.0, 0.0, y], [-s, 0.0, c, z]], dtype=np.float64)


def look_camera(position, pitch_down_deg: float, width: int, height: int,
                vfov_deg: float = 60.0, yaw_deg: float = 0.0, near: float = 0.2) -> Camera:
    """Camera at `position` looking along world +z (turned by yaw about +y),
    pitched down by `pitch_down_deg`; vertical field of view `vfov_deg`,
    square pixels, principal point at the image centre."""
    a = math.radians(pitch_down_deg)
    b = math.radians(yaw_deg)
    fwd = np.array([math.sin(b) * math.cos(a), -math.sin(a), math.cos(b) * math.cos(a)])
    up_world = np.array([0.0, 1.0, 0.0])
    right = np.cross(up_world, fwd)  # camera +x in world (points to screen right)
    right = -right / np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    # right-handed check: x_c cross y_c = z_c
    if np.dot(np.cross(R[0], R[1]), R[2]) < 0:
        R[0] = -R[0]
    pos = np.asarray(position, dtype=np.float64)
    t = -R @ pos
    fy = (height / 2.0) / math.tan(math.radians(vfov_deg) / 2.0)
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32), fx=float(fy), fy=float(fy),
                  cx=width / 2.0, cy=height / 2.0, width=int(width), height=int(height),
                  near=near)


def random_poses(seed: int, n: int, sigma: float = 0.3) -> np.ndarray:
    """Axis-angle joint poses [n,24,3], every component N(0, sigma) radians."""
    rng = np.random.default_rng(seed)
    return (sigma * rng.standard_normal((n, N_JOINTS, 3))).astype(np.float32)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    templates: list
    instances: Instances
    camera: Camera
    lod: LodConfig
    name: str


def single_lod() -> LodConfig:
    return LodConfig(thresholds=np.zeros(0, np.float32), fractions=np.ones(1, np.float32),
                     scale_mult=np.ones(1, np.float32))


def paper_lod() -> LodConfig:
    """Three distance bands: 100% / 25% / 6% of each template, thresholds
    10 m and 30 m, scale multiplier fraction^(-1/2) (1, 2, 4.08)."""
    f = np.array([1.0, 0.25, 0.06])
    return LodConfig(thresholds=np.array([10.0, 30.0], np.float32),
                     fractions=f.astype(np.float32),
                     scale_mult=(f ** -0.5).astype(np.float32))


def single_avatar(n_gauss: int = 16384, size: int = 256, sh_degree: int = 0,
                  pose_seed: int = 11, template_seed: int = 1000) -> Scene:
    """One template of `n_gauss` Gaussians, one instance at the origin facing
    the camera, camera 2.5 m away at pelvis height, `size` x `size`, vertical
    field of view 60 degrees, poses N(0, 0.3 rad) from `pose_seed`."""
    tpl = make_template(template_seed, n_gauss, sh_degree,
                        base_colour_uniform=(sh_degree == 0))
    pelvis_y = float(tpl.rest_joints[0, 1])
    root = yaw_root(math.pi, 0.0, 0.0, 0.0)[None].astype(np.float32)
    inst = Instances(template_id=np.zeros(1, np.int32), root=root,
                     pose=random_poses(pose_seed, 1))
    cam = look_camera((0.0, pelvis_y, -2.5), 0.0, size, size)
    return Scene([tpl], inst, cam, single_lod(), f"single_avatar_{n_gauss}g_{size}px")


def crowd_instances(n_templates: int, cols: int, rows: int, *, spacing: float = 1.2,
                    jitter: float = 0.3, first_row_z: float = 3.0, layout_seed: int = 7,
                    pose_seed: int = 100) -> Instances:
    """Jittered grid of cols x rows instances (row-major, nearest row first),
    yaw U(0, 2 pi), template id uniform, poses N(0, 0.3 rad)."""
    rng = np.random.default_rng(layout_seed)
    n = cols * rows
    tid = rng.integers(0, n_templates, size=n).astype(np.int32)
    yaw = rng.uniform(0.0, 2.0 * math.pi, size=n)
    jit = rng.uniform(-jitter, jitter, size=(n, 2))
    roots = np.empty((n, 3, 4))
    for k in range(n):
        r, c = divmod(k, cols)
        x = (c - (cols - 1) / 2.0) * spacing + jit[k, 0]
        z = first_row_z + r * spacing + jit[k, 1]
        roots[k] = yaw_root(yaw[k], x, 0.0, z)
    return Instances(template_id=tid, root=roots.astype(np.float32),
                     pose=random_poses(pose_seed, n))


def band_instances(n_templates: int, n: int, d_lo: float, d_hi: float, seed: int, *,
                   camera_position=(0.0, 1.6, 0.0), half_angle_deg: float = 40.0) -> Instances:
    """n instances on the ground whose root lies at a distance U(d_lo, d_hi)
    from the camera centre, at an azimuth U(-half_angle, half_angle) about
    the camera's +z heading, with yaw U(0, 2 pi), template uniform and poses
    N(0, 0.3 rad).  Views of one LoD distance band."""
    rng = np.random.default_rng(seed)
    cx, cy, cz = camera_position
    d = rng.uniform(d_lo, d_hi, n)
    dh = np.sqrt(np.maximum(d * d - cy * cy, 0.0))
    az = np.radians(rng.uniform(-half_angle_deg, half_angle_deg, n))
    yaw = rng.uniform(0.0, 2.0 * math.pi, n)
    tid = rng.integers(0, n_templates, n).astype(np.int32)
    roots = np.stack([yaw_root(yaw[k], cx + dh[k] * math.sin(az[k]), 0.0, cz + dh[k] * math.cos(az[k]))
                      for k in range(n)]).astype(np.float32)
    return Instances(template_id=tid, root=roots, pose=random_poses(seed + 1, n))


def crowd(n_templates: int = 14, n_gauss: int = 65536, sh_degree: int = 3,
          cols: int = 50, rows: int = 70, width: int = 1920, height: int = 1080,
          frame: int = 0, lod: LodConfig | None = None) -> Scene:
    """The paper-scale crowd: `n_templates` templates (seeds 1000 + t) of
    `n_gauss` Gaussians with SH degree `sh_degree` (coefficients N(0, 0.3)),
    a cols x rows grid at 1.2 m spacing starting 3 m from the camera, camera
    at (0, 1.6, 0) pitched down 10 degrees looking +z, vertical field of view
    60 degrees, poses drawn from seed 100 + frame, three distance LoD bands."""
    tpls = [make_template(1000 + t, n_gauss, sh_degree) for t in range(n_templates)]
    inst = crowd_instances(n_templates, cols, rows, pose_seed=100 + frame)
    cam = look_camera((0.0, 1.6, 0.0), 10.0, width, height)
    return Scene(tpls, inst, cam, lod if lod is not None else paper_lod(),
                 f"crowd_{n_templates}x{n_gauss}g_{cols * rows}inst_{width}x{height}")
