"""The C ABI without a GPU: libhrc.so builds for sm_103a, loads, exports every
function include/hrc.h declares, the Python binding declares each of them
with the C name, and the argument checks that run before any CUDA call
answer HRC_EINVAL."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hrc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:hrc_status|int|long long|const char \*)\s*(hrc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_02041_gb300 import _lib
    from paper_2505_02041_gb300.build import build
    build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hrc_create", "hrc_destroy", "hrc_fluence", "hrc_fluence_backward", "hrc_create_batched",
                     "hrc_fluence_batched", "hrc_fluence_backward_batched", "hrc_scene_offsets", "hrc_last_error",
                     "hrc_set_stream", "hrc_set_precision", "hrc_fluence_noalloc"):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_mirrors_the_header():
    from paper_2505_02041_gb300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert bound == set(declared_functions())


def test_argument_errors_before_any_cuda_call(lib):
    from paper_2505_02041_gb300 import _lib
    out = ctypes.c_void_p()
    assert lib.hrc_create(0, 8, 1, 0, ctypes.byref(out)) == _lib.HRC_EINVAL
    assert "W and H" in _lib.hrc_last_error()
    assert lib.hrc_create(8, 8, 5, 0, ctypes.byref(out)) == _lib.HRC_EINVAL
    assert lib.hrc_create(20000, 8, 1, 0, ctypes.byref(out)) == _lib.HRC_EINVAL
    assert lib.hrc_create(8, 8, 1, 0, None) == _lib.HRC_EINVAL
    W = (ctypes.c_int * 2)(8, 0)
    H = (ctypes.c_int * 2)(8, 8)
    assert lib.hrc_create_batched(2, W, H, 1, 0, ctypes.byref(out)) == _lib.HRC_EINVAL
    assert lib.hrc_create_batched(0, W, H, 1, 0, ctypes.byref(out)) == _lib.HRC_EINVAL
    assert lib.hrc_create_batched_prec(1, W, H, 1, 0, 3, ctypes.byref(out)) == _lib.HRC_EINVAL
    for fn in (lib.hrc_destroy,):
        assert fn(None) == _lib.HRC_EINVAL
    assert lib.hrc_set_stream(None, None) == _lib.HRC_EINVAL
    assert lib.hrc_set_precision(None, 0) == _lib.HRC_EINVAL
    assert lib.hrc_set_schedule(None, 0) == _lib.HRC_EINVAL
    assert lib.hrc_fluence(None, None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_fluence_backward(None, None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_fluence_batched(None, None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_scene_offsets(None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_batched_sync(None) == _lib.HRC_EINVAL
    assert lib.hrc_batched_schedule(None, 1) == _lib.HRC_EINVAL
    assert lib.hrc_set_backward_recompute(None, 1) == _lib.HRC_EINVAL
    assert lib.hrc_set_cross_blur(None, 1, 0.5) == _lib.HRC_EINVAL
    assert lib.hrc_get_cross_blur(None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_reserve_bounces(None, 2) == _lib.HRC_EINVAL
    assert lib.hrc_set_environment(None, None, 4) == _lib.HRC_EINVAL
    assert lib.hrc_set_channel_extinction(None, 1) == _lib.HRC_EINVAL
    assert lib.hrc_fluence_bounces(None, None, None, None, 1, None) == _lib.HRC_EINVAL
    assert lib.hrc_fluence_bounces_backward(None, None, None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_bounce_source(None, None, None, None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_sync(None) == _lib.HRC_EINVAL
    assert lib.hrc_debug_bulk_wait(None, 0, 0) == _lib.HRC_EINVAL
    assert lib.hrc_get_launch_config(None, None) == _lib.HRC_EINVAL
    assert lib.hrc_set_launch_config(None, None) == _lib.HRC_EINVAL
    # the allocation-free entry point rejects sizes beyond its fixed scratch
    assert lib.hrc_fluence_noalloc(129, 8, 1, None, None, None, None) == _lib.HRC_EINVAL
    assert "128" in _lib.hrc_last_error()
    assert lib.hrc_fluence_noalloc(8, 8, 5, None, None, None, None) == _lib.HRC_EINVAL
    assert lib.hrc_fluence_noalloc(8, 8, 1, None, None, None, None) == _lib.HRC_EINVAL
    assert _lib.hrc_version().startswith("hrc-gb300")


def test_product_path_does_not_reach_the_oracle():
    """The product package never imports the oracle (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2505_02041_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "hrc_oracle" not in text, f
