"""Thin Python binding of libcrowdsplat.so (argument marshalling only).

Every function of ``include/crowdsplat.h``, ``include/crowdsplat_lod.h`` and
``include/crowdsplat_grad.h`` is reachable under the same name through
:func:`lib`; :class:`Renderer`
wraps a render context and :class:`Mlp` the LoD ranking network, with
PyTorch device memory and streams.  All computation runs in the library's CUDA kernels:
there is no CPU path, and :func:`load` raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

CS_OK, CS_ERR_ARG, CS_ERR_CUDA, CS_ERR_OOM, CS_ERR_CAPACITY, CS_ERR_TIMEOUT, CS_ERR_STATE = range(7)
CS_SKIN_FULL, CS_SKIN_MEANS_ONLY = 0, 1
CS_SH_ROOT_FRAME, CS_SH_WORLD_FRAME = 0, 1
CS_STORE_FP32, CS_STORE_BF16 = 0, 1
CS_BLEND_ITEMS_AUTO, CS_BLEND_ITEMS_TILES, CS_BLEND_ITEMS_BLOCKS = 0, 1, 2
DBG = dict(skin_b=1, visible=2, groups=3, records=4, depth_keys=5, rects=6, depth_order=7,
           pair_tiles=8, pair_splats=9, tile_ranges=10)
STAGES = ("fk", "cull_lod", "skin_project", "depth_sort", "pair_emit", "tile_sort", "tile_ranges",
          "blend")


class CreateParams(C.Structure):
    _fields_ = [("device", C.c_int32), ("stream", C.c_void_p), ("skin_mode", C.c_int32),
                ("sh_frame", C.c_int32), ("instance_cull", C.c_int32), ("stage_timing", C.c_int32),
                ("template_storage", C.c_int32)]


class TemplateDesc(C.Structure):
    _fields_ = [("n_gauss", C.c_int32), ("sh_degree", C.c_int32), ("means", C.c_void_p),
                ("scales", C.c_void_p), ("quats", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p), ("skin_idx", C.c_void_p), ("skin_w", C.c_void_p),
                ("rest_joints", C.c_void_p), ("parents", C.c_void_p)]


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float), ("win_x0", C.c_int32), ("win_y0", C.c_int32),
                ("full_width", C.c_int32), ("full_height", C.c_int32)]


class FrameStats(C.Structure):
    _fields_ = [("instances", C.c_int32), ("instances_visible", C.c_int32),
                ("instances_per_level", C.c_int32 * 4), ("splats", C.c_int64),
                ("splats_live", C.c_int64), ("pairs", C.c_int64), ("tiles_x", C.c_int32),
                ("tiles_y", C.c_int32), ("kernel_launches", C.c_int32), ("depth_key_bits", C.c_int32)]

    def as_dict(self) -> dict:
        return dict(instances=self.instances, instances_visible=self.instances_visible,
                    instances_per_level=list(self.instances_per_level), splats=self.splats,
                    splats_live=self.splats_live, pairs=self.pairs, tiles_x=self.tiles_x,
                    tiles_y=self.tiles_y, kernel_launches=self.kernel_launches,
                    depth_key_bits=self.depth_key_bits)


class Grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p), ("pose", C.c_void_p)]


class MemoryStats(C.Structure):
    _fields_ = [("template_bytes", C.c_int64), ("instance_bytes", C.c_int64),
                ("frame_bytes", C.c_int64), ("total_bytes", C.c_int64)]


_lib = None

# name -> (restype, argtypes) for every function of include/crowdsplat.h
_P = C.c_void_p
SIGNATURES = {
    "cs_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(CreateParams)]),
    "cs_destroy": (None, [_P]),
    "cs_upload_templates": (C.c_int, [_P, C.c_int32, C.POINTER(TemplateDesc)]),
    "cs_set_lod": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "cs_set_lod_subset": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P]),
    "cs_set_instances": (C.c_int, [_P, C.c_int32, _P, _P, _P, C.c_int32]),
    "cs_render": (C.c_int, [_P, C.POINTER(Camera), _P, C.POINTER(FrameStats)]),
    "cs_render_contrib": (C.c_int, [_P, C.POINTER(Camera), _P, _P, C.POINTER(FrameStats)]),
    "cs_render_to_host": (C.c_int, [_P, C.POINTER(Camera), _P, C.POINTER(FrameStats)]),
    "cs_render_static": (C.c_int, [_P, C.POINTER(Camera), _P, C.POINTER(FrameStats)]),
    "cs_get_stage_times": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]),
    "cs_memory_stats": (C.c_int, [_P, C.POINTER(MemoryStats)]),
    "cs_last_error": (C.c_char_p, [_P]),
    "cs_debug_read": (C.c_int, [_P, C.c_int32, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "cs_debug_fail_allocs": (C.c_int, [_P, C.c_int32]),
    "cs_debug_blend_items": (C.c_int, [_P, C.c_int32]),
    "cs_debug_checks": (C.c_int, [_P, C.POINTER(C.c_uint32), C.POINTER(C.c_int32)]),
    "cs_version": (C.c_char_p, []),
    # ranked LoD (include/crowdsplat_lod.h)
    "cs_lod_features": (C.c_int, [_P, _P]),
    "cs_lod_rank": (C.c_int, [_P, _P, _P]),
    "cs_lod_targets": (C.c_int, [_P, C.c_int32, _P, C.c_float, _P]),
    "cs_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, _P, C.c_uint64]),
    "cs_mlp_destroy": (None, [_P]),
    "cs_mlp_last_error": (C.c_char_p, [_P]),
    "cs_mlp_get_params": (C.c_int, [_P, _P]),
    "cs_mlp_set_params": (C.c_int, [_P, _P]),
    "cs_mlp_forward": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "cs_mlp_train_step": (C.c_int, [_P, C.c_int64, _P, _P, _P, C.c_float, C.POINTER(C.c_float)]),
    "cs_mlp_get_grad": (C.c_int, [_P, _P]),
    # gradients (include/crowdsplat_grad.h)
    "cs_render_train": (C.c_int, [_P, C.POINTER(Camera), _P, C.POINTER(FrameStats)]),
    "cs_backward": (C.c_int, [_P, _P, C.POINTER(Grads)]),
}

LOD_FEATURES, MLP_PARAMS = 32, 48 * 64 + 64 + 64 * 64 + 64 + 64 + 1


_libs = {}


def load(path: str | None = None):
    """Load libcrowdsplat.so (or the library at `path`, e.g. the bounds-checked
    debug build); raises RuntimeError if it has not been built."""
    global _lib
    p = os.path.abspath(path or LIB_PATH)
    if p not in _libs:
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it first (python -m paper_2501_17792_gb300.build "
                               "or __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _libs[p] = L
    if path is None:
        _lib = _libs[p]
    return _libs[p]


lib = load


class CrowdSplatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"crowdsplat error {code}: {msg}")
        self.code = code


def camera_struct(cam) -> Camera:
    """Camera from an object with R, t, fx, fy, cx, cy, width, height, near."""
    c = Camera()
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(getattr(cam, "near", 0.2))
    c.win_x0, c.win_y0 = int(getattr(cam, "win_x0", 0)), int(getattr(cam, "win_y0", 0))
    c.full_width, c.full_height = int(getattr(cam, "full_width", 0)), int(getattr(cam, "full_height", 0))
    return c


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Renderer:
    """One library context on one CUDA device.

    Device memory and streams come from PyTorch: ``render`` writes into a
    torch CUDA tensor on the context's stream (the current torch stream at
    creation unless ``stream`` is given).
    """

    def __init__(self, device: int = 0, stream=None, skin_mode: int = CS_SKIN_FULL,
                 sh_frame: int = CS_SH_ROOT_FRAME, instance_cull: bool = True,
                 stage_timing: bool = False, template_storage: int = CS_STORE_FP32, library: str | None = None):
        import torch
        self.torch = torch
        self.L = load(library)
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        p = CreateParams(device=self.device, stream=C.c_void_p(int(stream.cuda_stream)),
                         skin_mode=int(skin_mode), sh_frame=int(sh_frame),
                         instance_cull=1 if instance_cull else 0,
                         stage_timing=1 if stage_timing else 0, template_storage=int(template_storage))
        h = C.c_void_p()
        rc = self.L.cs_create(C.byref(h), C.byref(p))
        if rc != CS_OK:
            raise CrowdSplatError(rc, "cs_create failed")
        self.h = h
        self._keep = []

    # -- helpers ----------------------------------------------------------
    def _check(self, rc: int):
        if rc != CS_OK:
            raise CrowdSplatError(rc, self.L.cs_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.cs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ---------------------------------------------------------------
    def upload_templates(self, templates):
        descs = (TemplateDesc * len(templates))()
        keep = []
        for k, t in enumerate(templates):
            arrs = [_host(t.means, np.float32), _host(t.scales, np.float32), _host(t.quats, np.float32),
                    _host(t.opacity, np.float32), _host(t.sh, np.float32), _host(t.skin_idx, np.uint8),
                    _host(t.skin_w, np.float32), _host(t.rest_joints, np.float32),
                    _host(t.parents, np.int32)]
            keep.append(arrs)
            d = descs[k]
            d.n_gauss = int(arrs[0].shape[0])
            d.sh_degree = int(t.sh_degree)
            (d.means, d.scales, d.quats, d.opacity, d.sh, d.skin_idx, d.skin_w, d.rest_joints,
             d.parents) = (a.ctypes.data for a in arrs)
        self._check(self.L.cs_upload_templates(self.h, len(templates), descs))
        self.template_sizes = [int(np.asarray(t.means).shape[0]) for t in templates]
        self.n_gauss_total = sum(self.template_sizes)

    def set_lod(self, lod):
        thr = _host(lod.thresholds, np.float32)
        frac = _host(lod.fractions, np.float32)
        mult = _host(lod.scale_mult, np.float32)
        n = int(frac.shape[0])
        self._check(self.L.cs_set_lod(self.h, n, thr.ctypes.data if thr.size else None,
                                      frac.ctypes.data, mult.ctypes.data))

    def set_lod_subset(self, template_id: int, level: int, idx):
        """Gaussians (template-local indices) that `level` of the template
        renders; an empty array restores the level's prefix."""
        a = _host(np.asarray(idx), np.uint32)
        self._check(self.L.cs_set_lod_subset(self.h, int(template_id), int(level), int(a.shape[0]),
                                             a.ctypes.data if a.size else None))

    def set_instances(self, template_id, root, pose):
        """Host arrays (numpy, or CPU tensors) or CUDA tensors on this device."""
        torch = self.torch
        if isinstance(root, torch.Tensor) and root.is_cuda:
            tid = template_id.to(torch.int32).contiguous()
            r = root.to(torch.float32).contiguous()
            p = pose.to(torch.float32).contiguous()
            self._check(self.L.cs_set_instances(self.h, int(tid.shape[0]), tid.data_ptr(), r.data_ptr(),
                                                p.data_ptr(), 1))
            self._keep = [tid, r, p]  # keep alive until the stream has copied them
            return
        tid = _host(np.asarray(template_id), np.int32)
        r = _host(np.asarray(root), np.float32)
        p = _host(np.asarray(pose), np.float32)
        self._check(self.L.cs_set_instances(self.h, int(tid.shape[0]), tid.ctypes.data, r.ctypes.data,
                                            p.ctypes.data, 0))
        self._keep = [tid, r, p]

    def render(self, camera, out=None, stats: bool = False):
        """Render into a CUDA tensor [H, W, 4] float32 (allocated if None)."""
        torch = self.torch
        cam = camera_struct(camera)
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32,
                                  device=f"cuda:{self.device}")
        st = FrameStats()
        self._check(self.L.cs_render(self.h, C.byref(cam), out.data_ptr(), C.byref(st) if stats else None))
        return (out, st.as_dict()) if stats else out

    def render_contrib(self, camera, contrib, out=None, stats: bool = False):
        """Render and ADD each template Gaussian's summed compositing weight
        to `contrib` (CUDA float32 tensor, one entry per uploaded Gaussian,
        templates concatenated in upload order)."""
        torch = self.torch
        cam = camera_struct(camera)
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32,
                                  device=f"cuda:{self.device}")
        if not (contrib.is_cuda and contrib.dtype == torch.float32 and contrib.is_contiguous()):
            raise ValueError("contrib must be a contiguous float32 CUDA tensor")
        st = FrameStats()
        self._check(self.L.cs_render_contrib(self.h, C.byref(cam), out.data_ptr(), contrib.data_ptr(),
                                             C.byref(st) if stats else None))
        return (out, st.as_dict()) if stats else out

    def render_train(self, camera, out=None, stats: bool = False):
        """Render and keep the state :meth:`backward` needs."""
        torch = self.torch
        cam = camera_struct(camera)
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32,
                                  device=f"cuda:{self.device}")
        st = FrameStats()
        self._check(self.L.cs_render_train(self.h, C.byref(cam), out.data_ptr(), C.byref(st) if stats else None))
        self._train_shape = (cam.height, cam.width)
        return (out, st.as_dict()) if stats else out

    def backward(self, dl_drgba, n_instances: int, grads: dict | None = None) -> dict:
        """Gradients of the last :meth:`render_train` frame for dL/d(RGBA)
        [H, W, 4] (CUDA float32).  Returns (and adds into, when given) CUDA
        tensors means [N,3], scales [N,3], quats [N,4], opacity [N],
        sh [N,16,3] and pose [I,24,3]."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        g = dl_drgba.to(device=dev, dtype=torch.float32).contiguous()
        n = self.n_gauss_total
        if grads is None:
            with torch.cuda.stream(self.stream):
                grads = dict(means=torch.zeros((n, 3), device=dev), scales=torch.zeros((n, 3), device=dev),
                             quats=torch.zeros((n, 4), device=dev), opacity=torch.zeros(n, device=dev),
                             sh=torch.zeros((n, 16, 3), device=dev),
                             pose=torch.zeros((int(n_instances), 24, 3), device=dev))
        cg = Grads(*(grads[k].data_ptr() if grads.get(k) is not None else None
                     for k in ("means", "scales", "quats", "opacity", "sh", "pose")))
        self._check(self.L.cs_backward(self.h, g.data_ptr(), C.byref(cg)))
        self._keep_grad = g
        return grads

    def render_to_host(self, camera, out: np.ndarray | None = None, stats: bool = False):
        cam = camera_struct(camera)
        if out is None:
            out = np.empty((cam.height, cam.width, 4), np.float32)
        st = FrameStats()
        self._check(self.L.cs_render_to_host(self.h, C.byref(cam), out.ctypes.data,
                                             C.byref(st) if stats else None))
        return (out, st.as_dict()) if stats else out

    def stage_times(self, average: bool = False):
        """Per-stage ms of the last frame, or (average=True) the mean over the
        frames since the previous average call; returns (dict, frames)."""
        ms = (C.c_float * len(STAGES))()
        frames = C.c_int64()
        n = self.L.cs_get_stage_times(self.h, ms, len(STAGES), 1 if average else 0, C.byref(frames))
        if n < 0:
            self._check(-n)
        return {STAGES[i]: float(ms[i]) for i in range(n)}, int(frames.value)

    def memory_stats(self) -> dict:
        m = MemoryStats()
        self._check(self.L.cs_memory_stats(self.h, C.byref(m)))
        return dict(template_bytes=m.template_bytes, instance_bytes=m.instance_bytes,
                    frame_bytes=m.frame_bytes, total_bytes=m.total_bytes)

    def lod_features(self):
        """[n_total, 32] float32 CUDA tensor of per-Gaussian ranking features."""
        torch = self.torch
        n = self.n_gauss_total
        with torch.cuda.stream(self.stream):
            f = torch.empty((n, LOD_FEATURES), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.L.cs_lod_features(self.h, f.data_ptr()))
        return f

    def lod_targets(self, contrib, floor: float = 1e-3):
        """ln(c / template mean + floor) per (band, Gaussian); contrib is a
        CUDA float32 tensor [n_bands, n_total]."""
        torch = self.torch
        c = contrib.to(torch.float32).contiguous()
        if c.dim() != 2 or c.shape[1] != self.n_gauss_total:
            raise ValueError("contrib must be [n_bands, n_total]")
        with torch.cuda.stream(self.stream):
            t = torch.empty_like(c)
        self._check(self.L.cs_lod_targets(self.h, int(c.shape[0]), c.data_ptr(), float(floor), t.data_ptr()))
        return t

    def lod_rank(self, score):
        """Per-template orders (uint32 as int32 CUDA tensor [n_total]) of the
        Gaussians by descending score (float32 CUDA tensor [n_total])."""
        torch = self.torch
        s = score.to(torch.float32).contiguous()
        with torch.cuda.stream(self.stream):
            o = torch.empty(s.shape[0], dtype=torch.int32, device=f"cuda:{self.device}")
        if s.shape[0] != self.n_gauss_total:
            raise ValueError(f"score has {s.shape[0]} entries, templates hold {self.n_gauss_total}")
        self._check(self.L.cs_lod_rank(self.h, s.data_ptr(), o.data_ptr()))
        return o

    def debug_checks(self) -> tuple[int, bool]:
        """Bounds-check word of the checked debug build since the last call
        (read and cleared; 0 = every check passed) and whether the loaded
        library was built with the checks (cs_debug_checks)."""
        failed, enabled = C.c_uint32(), C.c_int32()
        self._check(self.L.cs_debug_checks(self.h, C.byref(failed), C.byref(enabled)))
        return int(failed.value), bool(enabled.value)

    def debug_blend_items(self, mode: int) -> None:
        """Testing hook: the compositing schedule of plain frames
        (CS_BLEND_ITEMS_AUTO, _TILES or _BLOCKS; cs_debug_blend_items)."""
        self._check(self.L.cs_debug_blend_items(self.h, int(mode)))

    def debug(self, which: str) -> np.ndarray:
        code = DBG[which]
        size = C.c_size_t()
        self._check(self.L.cs_debug_read(self.h, code, None, 0, C.byref(size)))
        buf = np.empty(size.value, np.uint8)
        if size.value:
            self._check(self.L.cs_debug_read(self.h, code, buf.ctypes.data, size.value, None))
        dt = {"skin_b": np.float32, "visible": np.int32, "groups": np.int32, "records": np.float32,
              "depth_keys": np.uint32, "rects": np.uint16, "depth_order": np.uint32,
              "pair_tiles": np.uint16, "pair_splats": np.uint32, "tile_ranges": np.uint32}[which]
        a = buf.view(dt)
        shape = {"skin_b": (-1, 24, 3, 4), "groups": (-1, 7), "records": (-1, 16), "rects": (-1, 4),
                 "tile_ranges": (-1, 2)}.get(which)
        return a.reshape(shape) if shape else a


class Mlp:
    """The LoD ranking MLP (48 -> 64 -> 64 -> 1, BF16 tensor-core kernels)
    on one CUDA device; inputs and outputs are CUDA tensors."""

    def __init__(self, device: int = 0, stream=None, seed: int = 0):
        import torch
        self.torch = torch
        self.L = load()
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        rc = self.L.cs_mlp_create(C.byref(h), self.device, C.c_void_p(int(self.stream.cuda_stream)),
                                  C.c_uint64(int(seed)))
        if rc != CS_OK:
            raise CrowdSplatError(rc, "cs_mlp_create failed")
        self.h = h

    def _check(self, rc: int):
        if rc != CS_OK:
            raise CrowdSplatError(rc, self.L.cs_mlp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.cs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        self._check(self.L.cs_mlp_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, p):
        a = _host(np.asarray(p), np.float32)
        if a.shape != (MLP_PARAMS,):
            raise ValueError(f"need {MLP_PARAMS} parameters")
        self._check(self.L.cs_mlp_set_params(self.h, a.ctypes.data))

    def grad(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        self._check(self.L.cs_mlp_get_grad(self.h, out.ctypes.data))
        return out

    def _dev(self, t, dtype):
        torch = self.torch
        return t.to(device=f"cuda:{self.device}", dtype=dtype).contiguous()

    def forward(self, feat, band, out=None):
        torch = self.torch
        f = self._dev(feat, torch.float32)
        b = self._dev(band, torch.int32)
        n = int(f.shape[0])
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty(n, dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.L.cs_mlp_forward(self.h, n, f.data_ptr(), b.data_ptr(), out.data_ptr()))
        return out

    def train_step(self, feat, band, target, lr: float, want_loss: bool = True):
        torch = self.torch
        f = self._dev(feat, torch.float32)
        b = self._dev(band, torch.int32)
        t = self._dev(target, torch.float32)
        loss = C.c_float()
        self._check(self.L.cs_mlp_train_step(self.h, int(f.shape[0]), f.data_ptr(), b.data_ptr(), t.data_ptr(),
                                             float(lr), C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None


def render_scene(scene, *, device: int = 0, **kw):
    """Convenience: upload a scene object (templates, instances, camera, lod)
    and render one frame; returns (renderer, image tensor)."""
    r = Renderer(device=device, **kw)
    r.upload_templates(scene.templates)
    r.set_lod(scene.lod)
    r.set_instances(scene.instances.template_id, scene.instances.root, scene.instances.pose)
    img = r.render(scene.camera)
    return r, img
