"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/sd.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(sd_[a-z_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libsd():
    from paper_2609_32308_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sd_load_energy", "sd_design", "sd_design_batch", "sd_result_free",
                 "sd_energy_free", "sd_strerror", "sd_plan_create", "sd_plan_run",
                 "sd_plan_results", "sd_plan_dump", "sd_plan_free"):
        assert must in names


def test_library_exports_every_declared_symbol(libsd):
    missing = [n for n in declared_functions() if not hasattr(libsd, n)]
    assert not missing, missing


def test_library_is_built_for_sm103a():
    from paper_2609_32308_b300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_host_only_calls_without_gpu(libsd):
    libsd.sd_strerror.restype = ctypes.c_char_p
    assert libsd.sd_strerror(0) == b"ok"
    assert b"range" in libsd.sd_strerror(-2)
    h = ctypes.c_void_p()
    libsd.sd_load_energy.argtypes = [ctypes.c_char_p, ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_void_p)]
    assert libsd.sd_load_energy(b"/nonexistent/params.par", 0, ctypes.byref(h)) == -1
    assert not h.value


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    import paper_2609_32308_b300 as sd
    monkeypatch.setattr(sd, "_lib", None)
    monkeypatch.setattr(sd, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        sd.lib()


def test_host_only_argument_checks(libsd):
    """Argument checks that return before any CUDA call: a NULL plan for the
    scheduling setters, and the message of a bounded-wait timeout."""
    libsd.sd_plan_set_group.argtypes = [ctypes.c_void_p, ctypes.c_int]
    libsd.sd_plan_set_streams.argtypes = [ctypes.c_void_p, ctypes.c_int]
    for group in (0, 8, 16, 32, 7):
        assert libsd.sd_plan_set_group(None, group) == -1
    assert libsd.sd_plan_set_streams(None, 2) == -1
    libsd.sd_strerror.restype = ctypes.c_char_p
    assert b"wait" in libsd.sd_strerror(-6)
