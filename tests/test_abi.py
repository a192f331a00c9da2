"""The C ABI without a GPU: libvr.so builds for sm_103a, loads, and exports every
entry point include/vr.h declares; the Python binding covers exactly those."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(vr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_19737_gb300 import build
    return build.build()


def test_header_declares_core_calls():
    d = _declared()
    for name in ("vr_create", "vr_load_volume", "vr_precompute_morphology", "vr_set_tissue_params", "vr_render"):
        assert name in d


def test_library_exports_every_declared_symbol(libpath):
    from paper_2605_19737_gb300 import build
    for path in (libpath, build.OUT_DEBUG):
        lib = ctypes.CDLL(path)
        missing = [n for n in _declared() if not hasattr(lib, n)]
        assert not missing, (path, missing)


def test_debug_library_is_the_checked_build(libpath):
    from paper_2605_19737_gb300 import vr
    assert vr.load().vr_debug_build() == 0
    assert vr.load(debug=True).vr_debug_build() == 1


def test_binding_matches_header(libpath):
    from paper_2605_19737_gb300 import vr
    assert vr.exported_symbols() == _declared()
    lib = vr.load()
    assert lib.vr_version().decode().startswith("vr ")


def test_struct_layouts():
    from paper_2605_19737_gb300 import vr
    assert ctypes.sizeof(vr.vr_camera) == 48
    assert ctypes.sizeof(vr.vr_counters) == 48
    assert ctypes.sizeof(vr.vr_render_opts) == 24
    # 3 ints, pointer (8-aligned), 3 ints, 10 floats -> 12 + 4 pad + 8 + 12 + 40 = 76 -> 80 (8-aligned)
    assert ctypes.sizeof(vr.vr_tissue_params) == 80


def test_null_context_is_rejected_without_gpu(libpath):
    from paper_2605_19737_gb300 import vr
    lib = vr.load()
    assert lib.vr_destroy(None) == 0
    assert lib.vr_synchronize(None) == vr.VR_ERR_INVALID_ARG
    assert lib.vr_render(None, 1, None, 1, 1, 1, None, 0, None, None, None) == vr.VR_ERR_INVALID_ARG
    assert lib.vr_create(None, 0, None) == vr.VR_ERR_INVALID_ARG
