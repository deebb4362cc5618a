"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every function the headers under include/ declare; host-only calls behave."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("crowdsplat.h", "crowdsplat_lod.h", "crowdsplat_grad.h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(cs_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2501_17792_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cs_create", "cs_destroy", "cs_upload_templates", "cs_set_lod", "cs_set_instances",
                 "cs_render", "cs_render_to_host", "cs_get_stage_times", "cs_memory_stats",
                 "cs_last_error", "cs_debug_read", "cs_version", "cs_set_lod_subset", "cs_render_contrib",
                 "cs_lod_features", "cs_lod_rank", "cs_mlp_create", "cs_mlp_forward", "cs_mlp_train_step",
                 "cs_render_train", "cs_backward"):
        assert must in names
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == sorted(os.path.basename(h) for h in HEADERS)


def test_library_exports_every_declared_symbol(lib):
    from paper_2501_17792_gb300 import binding
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, name


def test_checked_debug_build_compiles_and_exports_every_declared_symbol():
    """The debug build with bounds checks in the kernels (CS_CHECKS=1) builds
    for sm_103a and exports the same ABI; the release build reports its
    checks as absent without touching a GPU (NULL arguments)."""
    from paper_2501_17792_gb300 import build
    path = build.build(checks=True)
    assert os.path.basename(path) == "libcrowdsplat_checks.so" and path != build.LIB
    L = C.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), name
    from paper_2501_17792_gb300 import binding
    L.cs_debug_checks.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    assert L.cs_debug_checks(None, None, None) == binding.CS_ERR_ARG


def test_library_is_built_for_sm103a():
    from paper_2501_17792_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_host_only_calls(lib):
    lib.cs_version.restype = C.c_char_p
    assert b"sm_103a" in lib.cs_version()
    lib.cs_last_error.restype = C.c_char_p
    lib.cs_last_error.argtypes = [C.c_void_p]
    assert lib.cs_last_error(None) == b"null context"
    lib.cs_destroy.argtypes = [C.c_void_p]
    lib.cs_destroy(None)  # accepted


def test_create_rejects_bad_arguments_without_touching_a_gpu(lib):
    from paper_2501_17792_gb300 import binding
    L = binding.load()
    h = C.c_void_p()
    assert L.cs_create(C.byref(h), None) == binding.CS_ERR_ARG
    p = binding.CreateParams(device=0, stream=None, skin_mode=7, sh_frame=0, instance_cull=1, stage_timing=0)
    assert L.cs_create(C.byref(h), C.byref(p)) == binding.CS_ERR_ARG
    p = binding.CreateParams(device=0, stream=None, skin_mode=0, sh_frame=5, instance_cull=1, stage_timing=0)
    assert L.cs_create(C.byref(h), C.byref(p)) == binding.CS_ERR_ARG
    assert not h.value


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2501_17792_gb300 import binding
    saved = binding._lib
    try:
        binding._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            binding.load(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved
