"""cs_render_static: the render call that allocates no device memory.

Some callers cannot let the library call cudaMalloc while a frame is being
produced: a real-time render thread may not take the allocator's implicit
device synchronisation and latency spikes, and an engine that hands the
library a fixed GPU memory budget up front may not see it grow.  This call
renders exactly what cs_render renders, with the per-frame scratch in one
static device array.  The test drives it through the C ABI on two frames in
a row (the array keeps the previous frame's contents) and compares each with
cs_render within the parity tolerance, then checks the size limit.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_17792_gb300 import build
    build.build()


TOL = 2e-3  # per-pixel bound used by the parity tests


def test_render_static_matches_render_on_two_calls_in_a_row():
    from paper_2501_17792_gb300 import binding
    from paper_2501_17792_gb300 import scene as S
    sc = S.single_avatar()  # 16,384 splats, 256 x 256
    r = binding.Renderer(device=0)
    r.upload_templates(sc.templates)
    r.set_lod(sc.lod)
    L = binding.load()
    cam = binding.camera_struct(sc.camera)
    out = torch.empty((sc.camera.height, sc.camera.width, 4), dtype=torch.float32, device="cuda")
    frames = []
    for pose in (sc.instances.pose, S.random_poses(12, 1)):
        r.set_instances(sc.instances.template_id, sc.instances.root, pose)
        ref = r.render(sc.camera).cpu().numpy()
        out.fill_(float("nan"))  # every pixel must be written by the call
        torch.cuda.synchronize()
        st = binding.FrameStats()
        rc = L.cs_render_static(r.h, C.byref(cam), C.c_void_p(out.data_ptr()), C.byref(st))
        assert rc == binding.CS_OK, L.cs_last_error(r.h).decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= TOL
        assert st.splats == 16384 and st.pairs > 0
        frames.append(got)
    assert np.abs(frames[0] - frames[1]).max() > 0.1  # the second frame is a new pose
    r.close()


def test_render_static_rejects_frames_over_its_limit():
    from paper_2501_17792_gb300 import binding
    from paper_2501_17792_gb300 import scene as S
    sc = S.crowd(n_templates=2, n_gauss=4096, sh_degree=0, cols=8, rows=6, width=320, height=180)
    r = binding.Renderer(device=0)
    r.upload_templates(sc.templates)
    r.set_instances(sc.instances.template_id, sc.instances.root, sc.instances.pose)
    L = binding.load()
    cam = binding.camera_struct(sc.camera)
    out = torch.empty((sc.camera.height, sc.camera.width, 4), dtype=torch.float32, device="cuda")
    rc = L.cs_render_static(r.h, C.byref(cam), C.c_void_p(out.data_ptr()), None)
    assert rc == binding.CS_ERR_CAPACITY
    assert b"static limit" in L.cs_last_error(r.h)
    r.close()
