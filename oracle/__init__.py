"""FP64 CPU oracle for the CrowdSplat crowd-synthesis path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may
import this package.  The CUDA library and its Python binding never do.  The
oracle shares no code with the CUDA path: it is plain C (``crowdsplat_oracle.c``,
compiled with gcc) plus this ctypes marshalling layer.

Inputs are duck-typed scene objects (``templates``, ``instances``, ``camera``,
``lod``) holding float32 arrays; the oracle promotes every value to float64.
What each function computes, with its citation, is stated in the C source.
Every function is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crowdsplat_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libcrowdsplat_oracle.so")
_lib = None

EV_EDGE, EV_ALPHA, EV_RADIUS, EV_TIE, EV_NEAR, EV_QZERO, EV_LOD = 1, 2, 4, 8, 16, 32, 64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Template(C.Structure):
    _fields_ = [("n", C.c_int32), ("sh_degree", C.c_int32),
                ("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p), ("skin_idx", C.c_void_p),
                ("skin_w", C.c_void_p), ("rest_joints", C.c_void_p), ("parents", C.c_void_p),
                ("cov", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("near_z", C.c_double)]


class _Scene(C.Structure):
    _fields_ = [("n_templates", C.c_int32), ("templates", C.POINTER(_Template)),
                ("n_instances", C.c_int32), ("template_id", C.c_void_p), ("root", C.c_void_p),
                ("pose", C.c_void_p), ("n_levels", C.c_int32), ("thresholds", C.c_void_p),
                ("fractions", C.c_void_p), ("scale_mult", C.c_void_p),
                ("skin_mode", C.c_int32), ("sh_frame", C.c_int32), ("cam", _Camera),
                ("sub_n", C.c_void_p), ("sub_off", C.c_void_p), ("sub_idx", C.c_void_p)]

MAX_LEVELS = 4  # LoD levels of the subset table


class _Eps(C.Structure):
    _fields_ = [("px", C.c_double), ("q", C.c_double), ("radius", C.c_double),
                ("depth_rel", C.c_double), ("near_z", C.c_double), ("impact", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        L.orc_rodrigues.argtypes = [P, P]
        L.orc_quat_to_rot.argtypes = [P, P]
        L.orc_sh_basis.argtypes = [C.c_int, P, P]
        L.orc_fk.argtypes = [C.POINTER(_Template), P, P, P, P]
        L.orc_instance_level.argtypes = [C.POINTER(_Scene), C.c_int, P, P]
        L.orc_instance_level.restype = C.c_int
        L.orc_level_count.argtypes = [C.POINTER(_Scene), C.c_int, C.c_int]
        L.orc_level_count.restype = C.c_int
        L.orc_level_size.argtypes = [C.POINTER(_Scene), C.c_int, C.c_int]
        L.orc_level_size.restype = C.c_int
        L.orc_project_instance.argtypes = [C.POINTER(_Scene), C.c_int] + [P] * 13
        L.orc_project_instance.restype = C.c_int
        L.orc_render_lattice.argtypes = [C.POINTER(_Scene), C.POINTER(_Eps)] + [C.c_int] * 6 + [P] * 6
        L.orc_render_lattice.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class OracleScene:
    """Marshals a scene (templates, instances, camera, lod) into the C
    structures.  Keeps references to every array it hands to C.

    ``subsets`` (optional): {(template, level): template-local Gaussian
    indices} -- the level renders exactly those Gaussians, in that order,
    instead of its prefix."""

    def __init__(self, scene, *, skin_mode: int = 0, sh_frame: int = 0, subsets=None):
        keep = []
        tpls = (_Template * len(scene.templates))()
        for k, t in enumerate(scene.templates):
            arrs = dict(means=_c(t.means, np.float32), scales=_c(t.scales, np.float32),
                        quats=_c(t.quats, np.float32), opacity=_c(t.opacity, np.float32),
                        sh=_c(t.sh, np.float32), skin_idx=_c(t.skin_idx, np.uint8),
                        skin_w=_c(t.skin_w, np.float32), rest_joints=_c(t.rest_joints, np.float32),
                        parents=_c(t.parents, np.int32))
            keep.append(arrs)
            tpls[k].n = int(arrs["means"].shape[0])
            tpls[k].sh_degree = int(t.sh_degree)
            cov = getattr(t, "cov", None)
            if cov is not None:  # canonical covariance given directly [n, 6]
                arrs["cov"] = _c(np.asarray(cov).reshape(-1, 6), np.float32)
            for name, a in arrs.items():
                setattr(tpls[k], name, a.ctypes.data)
        inst = scene.instances
        self.template_id = _c(inst.template_id, np.int32)
        self.root = _c(inst.root, np.float32).reshape(-1, 12)
        self.pose = _c(inst.pose, np.float32).reshape(-1, 72)
        lod = scene.lod
        self.thr = _c(np.asarray(lod.thresholds, np.float32), np.float64)
        self.frac = _c(np.asarray(lod.fractions, np.float32), np.float64)
        self.mult = _c(np.asarray(lod.scale_mult, np.float32), np.float64)
        cam = scene.camera
        c = _Camera()
        R = np.asarray(cam.R, np.float32).astype(np.float64).reshape(9)
        t = np.asarray(cam.t, np.float32).astype(np.float64).reshape(3)
        for i in range(9):
            c.R[i] = R[i]
        for i in range(3):
            c.t[i] = t[i]
        c.fx, c.fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
        c.cx, c.cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
        c.width, c.height = int(cam.width), int(cam.height)
        c.near_z = float(np.float32(cam.near))
        s = _Scene()
        s.n_templates = len(scene.templates)
        s.templates = C.cast(tpls, C.POINTER(_Template))
        s.n_instances = int(self.template_id.shape[0])
        s.template_id = self.template_id.ctypes.data
        s.root = self.root.ctypes.data
        s.pose = self.pose.ctypes.data
        s.n_levels = int(self.frac.shape[0])
        s.thresholds = self.thr.ctypes.data if self.thr.size else None
        s.fractions = self.frac.ctypes.data
        s.scale_mult = self.mult.ctypes.data
        s.skin_mode = int(skin_mode)
        s.sh_frame = int(sh_frame)
        s.cam = c
        nt = len(scene.templates)
        self.sub_n = np.full(nt * MAX_LEVELS, -1, np.int32)
        self.sub_off = np.zeros(nt * MAX_LEVELS, np.int64)
        idx_parts, off = [], 0
        for (t, l), idx in sorted((subsets or {}).items()):
            a = np.asarray(idx, np.int64)
            if not (0 <= t < nt and 0 <= l < MAX_LEVELS):
                raise ValueError(f"subset key {(t, l)} out of range")
            if a.size and (a.min() < 0 or a.max() >= _template_size(scene, t) or np.unique(a).size != a.size):
                raise ValueError(f"subset {(t, l)}: indices must be distinct and in range")
            self.sub_n[t * MAX_LEVELS + l] = a.size
            self.sub_off[t * MAX_LEVELS + l] = off
            idx_parts.append(a.astype(np.int32))
            off += a.size
        self.sub_idx = np.ascontiguousarray(np.concatenate(idx_parts) if idx_parts else np.zeros(1, np.int32))
        s.sub_n = self.sub_n.ctypes.data
        s.sub_off = self.sub_off.ctypes.data
        s.sub_idx = self.sub_idx.ctypes.data
        self._keep = (keep, tpls)
        self.s = s
        self.n_gauss = [int(t.means.shape[0]) for t in scene.templates]
        self.width, self.height = int(cam.width), int(cam.height)

    @property
    def ref(self):
        return C.byref(self.s)


def _template_size(scene, t: int) -> int:
    return int(np.asarray(scene.templates[t].means).shape[0])


def default_eps(**kw) -> _Eps:
    """Event windows: 2e-4 px box edge, 1e-3 (relative) alpha threshold,
    1e-4 radius, 1e-6 relative depth tie, 1e-6 m near plane; an event counts
    when it can move the pixel by more than 5e-4."""
    e = _Eps(px=2e-4, q=1e-3, radius=1e-4, depth_rel=1e-6, near_z=1e-6, impact=5e-4)
    for k, v in kw.items():
        setattr(e, k, v)
    return e


# ---------------------------------------------------------------------------
# building blocks (exposed for the pins)
# ---------------------------------------------------------------------------

def rodrigues(v) -> np.ndarray:
    v = _c(v, np.float64)
    R = np.zeros(9)
    lib().orc_rodrigues(_p(v), _p(R))
    return R.reshape(3, 3)


def quat_to_rot(q) -> np.ndarray:
    q = _c(q, np.float64)
    R = np.zeros(9)
    lib().orc_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def sh_basis(deg: int, dirs) -> np.ndarray:
    """Real SH basis values [n, (deg+1)^2] at unit directions [n, 3]."""
    dirs = _c(np.atleast_2d(dirs), np.float64)
    K = (deg + 1) ** 2
    out = np.zeros((dirs.shape[0], 16))
    for i in range(dirs.shape[0]):
        lib().orc_sh_basis(deg, _p(dirs[i]), _p(out[i]))
    return out[:, :K]


def fk(os_: OracleScene, inst: int, with_global: bool = False):
    """Skinning transforms B [24,3,4] (and global joint transforms G) of one
    instance."""
    tp_index = int(os_.template_id[inst])
    B = np.zeros(24 * 12)
    G = np.zeros(24 * 12)
    tp = os_.s.templates[tp_index]
    lib().orc_fk(C.byref(tp), _p(os_.pose[inst]), _p(os_.root[inst]), _p(B), _p(G))
    if with_global:
        return B.reshape(24, 3, 4), G.reshape(24, 3, 4)
    return B.reshape(24, 3, 4)


def instance_level(os_: OracleScene, inst: int):
    d = np.zeros(1)
    nt = np.zeros(1)
    lvl = lib().orc_instance_level(os_.ref, inst, _p(d), _p(nt))
    return lvl, float(d[0]), float(nt[0])


def level_count(os_: OracleScene, lvl: int, n: int) -> int:
    return int(lib().orc_level_count(os_.ref, lvl, n))


def level_size(os_: OracleScene, template: int, lvl: int) -> int:
    """Gaussians that level `lvl` of the template renders (subset or prefix)."""
    return int(lib().orc_level_size(os_.ref, template, lvl))


def project_instance(os_: OracleScene, inst: int) -> dict:
    """Per-Gaussian results of one instance over its LoD level (prefix in
    template order, or the chosen subset in its order): valid, radius, uv, conic, depth, rgb, opacity, mu, cov3, cov2,
    r_exact, plus level and the skinning transforms B."""
    tp_index = int(os_.template_id[inst])
    n_max = os_.n_gauss[tp_index]
    out = dict(valid=np.zeros(n_max, np.int32), radius=np.zeros(n_max, np.int32),
               uv=np.zeros((n_max, 2)), conic=np.zeros((n_max, 3)), depth=np.zeros(n_max),
               rgb=np.zeros((n_max, 3)), opacity=np.zeros(n_max), mu=np.zeros((n_max, 3)),
               cov3=np.zeros((n_max, 6)), cov2=np.zeros((n_max, 3)), r_exact=np.zeros(n_max))
    lvl = np.zeros(1, np.int32)
    B = np.zeros(24 * 12)
    n = lib().orc_project_instance(os_.ref, inst, _p(lvl), *(_p(out[k]) for k in
                                   ("valid", "radius", "uv", "conic", "depth", "rgb", "opacity",
                                    "mu", "cov3", "cov2", "r_exact")), _p(B))
    res = {k: v[:n] for k, v in out.items()}
    res["level"] = int(lvl[0])
    res["B"] = B.reshape(24, 3, 4)
    res["count"] = n
    return res


def render(os_: OracleScene, eps: _Eps | None = None, lattice=None, contrib: bool = False) -> dict:
    """Composite the lattice of pixels (ox, oy, sx, sy, nx, ny); default is
    the full image.  Returns rgba [ny,nx,4], wsum, flags, impact, ncontrib,
    and with ``contrib`` the per-Gaussian sum of compositing weights
    alpha * T over the lattice (templates concatenated)."""
    if lattice is None:
        lattice = (0, 0, 1, 1, os_.width, os_.height)
    ox, oy, sx, sy, nx, ny = (int(x) for x in lattice)
    rgba = np.zeros((ny, nx, 4))
    wsum = np.zeros((ny, nx))
    flags = np.zeros((ny, nx), np.uint32)
    impact = np.zeros((ny, nx))
    nc = np.zeros((ny, nx), np.int32)
    e = eps if eps is not None else default_eps()
    cb = np.zeros(sum(os_.n_gauss)) if contrib else None
    rc = lib().orc_render_lattice(os_.ref, C.byref(e), ox, oy, sx, sy, nx, ny, _p(rgba),
                                  _p(wsum), _p(flags), _p(impact), _p(nc),
                                  _p(cb) if cb is not None else None)
    if rc != 0:
        raise MemoryError("oracle render failed to allocate")
    out = dict(rgba=rgba, wsum=wsum, flags=flags, impact=impact, ncontrib=nc)
    if cb is not None:
        out["contrib"] = cb
    return out


def tile_lists(os_: OracleScene, tile: int = 16) -> dict:
    """Per-tile splat lists of the 3DGS binning: a splat belongs to every
    tile that holds a pixel centre of its support box (clipped to the image),
    each list ordered by (view depth, instance, Gaussian).  Returns
    {tile_index: int64 array of keys instance * 2^32 + gaussian} for tiles
    with at least one splat."""
    W, H = os_.width, os_.height
    tw = (W + tile - 1) // tile
    keys, depth, tiles = [], [], []
    for inst in range(int(os_.template_id.shape[0])):
        p = project_instance(os_, inst)
        ok = np.nonzero(p["valid"])[0]
        for g in ok:
            u, v = p["uv"][g]
            r = p["radius"][g]
            i0 = max(0, int(np.ceil(u - r - 0.5)))
            i1 = min(W - 1, int(np.floor(u + r - 0.5)))
            j0 = max(0, int(np.ceil(v - r - 0.5)))
            j1 = min(H - 1, int(np.floor(v + r - 0.5)))
            for ty in range(j0 // tile, j1 // tile + 1):
                for tx in range(i0 // tile, i1 // tile + 1):
                    tiles.append(ty * tw + tx)
                    keys.append((inst << 32) | int(g))
                    depth.append(p["depth"][g])
    tiles = np.asarray(tiles, np.int64)
    keys = np.asarray(keys, np.int64)
    depth = np.asarray(depth)
    order = np.lexsort((keys, depth, tiles))
    tiles, keys = tiles[order], keys[order]
    out = {}
    if tiles.size:
        bounds = np.nonzero(np.diff(tiles))[0] + 1
        for seg_t, seg_k in zip(np.split(tiles, bounds), np.split(keys, bounds)):
            out[int(seg_t[0])] = seg_k
    return out


def tile_lists_window(os_: OracleScene, tx0: int, ty0: int, ntx: int, nty: int, tile: int = 16,
                      instances=None) -> tuple[dict, dict]:
    """``tile_lists`` restricted to the tiles [tx0, tx0 + ntx) x [ty0, ty0 + nty)
    (same membership rule and order: a splat belongs to every tile holding a
    pixel centre of its support box clipped to the image; each list ordered
    by view depth, then instance, then Gaussian), computed with array
    operations over the given instances (default: all).  Returns (lists,
    info): lists as in ``tile_lists``; info maps every listed key to its
    projection (u, v, radius, r_exact, A, B, C, opacity, depth)."""
    W, H = os_.width, os_.height
    tw = (W + tile - 1) // tile
    insts = range(int(os_.template_id.shape[0])) if instances is None else instances
    T_, K_, D_, info = [], [], [], {}
    for inst in insts:
        p = project_instance(os_, int(inst))
        g = np.nonzero(p["valid"])[0]
        if g.size == 0:
            continue
        u, v, r = p["uv"][g, 0], p["uv"][g, 1], p["radius"][g].astype(np.float64)
        i0 = np.maximum(0, np.ceil(u - r - 0.5)).astype(np.int64)
        i1 = np.minimum(W - 1, np.floor(u + r - 0.5)).astype(np.int64)
        j0 = np.maximum(0, np.ceil(v - r - 0.5)).astype(np.int64)
        j1 = np.minimum(H - 1, np.floor(v + r - 0.5)).astype(np.int64)
        a0 = np.maximum(i0 // tile, tx0); a1 = np.minimum(i1 // tile, tx0 + ntx - 1)
        b0 = np.maximum(j0 // tile, ty0); b1 = np.minimum(j1 // tile, ty0 + nty - 1)
        keep = (i0 <= i1) & (j0 <= j1) & (a0 <= a1) & (b0 <= b1)
        if not keep.any():
            continue
        g, a0, a1, b0, b1 = g[keep], a0[keep], a1[keep], b0[keep], b1[keep]
        nx, ny = a1 - a0 + 1, b1 - b0 + 1
        cnt = nx * ny
        rep = np.repeat(np.arange(g.size), cnt)
        k = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        tiles = (b0[rep] + k // nx[rep]) * tw + a0[rep] + k % nx[rep]
        keys = (np.int64(inst) << 32) | g[rep].astype(np.int64)
        T_.append(tiles)
        K_.append(keys)
        D_.append(p["depth"][g][rep])
        for m, gg in enumerate(g.tolist()):
            info[(int(inst) << 32) | gg] = (p["uv"][gg, 0], p["uv"][gg, 1], int(p["radius"][gg]), p["r_exact"][gg],
                                            p["conic"][gg, 0], p["conic"][gg, 1], p["conic"][gg, 2],
                                            p["opacity"][gg], p["depth"][gg])
    out = {}
    if T_:
        tiles, keys, depth = np.concatenate(T_), np.concatenate(K_), np.concatenate(D_)
        order = np.lexsort((keys, depth, tiles))
        tiles, keys = tiles[order], keys[order]
        bounds = np.nonzero(np.diff(tiles))[0] + 1
        for seg_t, seg_k in zip(np.split(tiles, bounds), np.split(keys, bounds)):
            out[int(seg_t[0])] = seg_k
    return out, info


def num_threads() -> int:
    return int(lib().orc_num_threads())
