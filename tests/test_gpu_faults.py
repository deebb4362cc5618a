"""Out-of-memory paths, driven by host-side failure injection.

cs_debug_fail_allocs makes the context's buffer allocations fail after a
given number of successful ones, exactly as a failed cudaMalloc would (the
buffer being grown is released first); no GPU call fails.  Every allocation
point of a first frame is made to fail in turn: the call must return
CS_ERR_OOM with a message naming the buffer, and once the injection is off
the same context must render the same image as a context that never
failed.
"""
import numpy as np
import pytest

from paper_2501_17792_gb300 import scene as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_17792_gb300 import build
    build.build()


def _scene():
    return S.crowd(n_templates=2, n_gauss=2048, sh_degree=1, cols=6, rows=4, width=160, height=96)


def test_every_allocation_point_fails_cleanly_and_the_context_recovers():
    from paper_2501_17792_gb300 import binding
    sc = _scene()
    ref = binding.Renderer(device=0)
    ref.upload_templates(sc.templates)
    ref.set_lod(sc.lod)
    ref.set_instances(sc.instances.template_id, sc.instances.root, sc.instances.pose)
    want = ref.render(sc.camera).cpu().numpy()
    ref.close()
    failures = 0
    for after in range(64):
        r = binding.Renderer(device=0)
        r.upload_templates(sc.templates)
        r.set_lod(sc.lod)
        assert r.L.cs_debug_fail_allocs(r.h, after) == binding.CS_OK
        try:
            r.set_instances(sc.instances.template_id, sc.instances.root, sc.instances.pose)
            r.render(sc.camera)
            torch.cuda.synchronize()
            ok = True
        except binding.CrowdSplatError as e:
            assert e.code == binding.CS_ERR_OOM, e
            assert "injected failure" in str(e), e
            failures += 1
            ok = False
        r.L.cs_debug_fail_allocs(r.h, -1)
        r.set_instances(sc.instances.template_id, sc.instances.root, sc.instances.pose)
        got = r.render(sc.camera).cpu().numpy()
        assert np.array_equal(got, want), after
        r.close()
        if ok:
            break
    # a frame makes many allocations; each one failed once before the sweep ended
    assert failures >= 8 and ok
