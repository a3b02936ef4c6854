"""C-ABI checks that need no GPU: the library builds, loads, exports every symbol that
include/holo.h declares, and rejects invalid arguments before touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_20304_gb300 import build as b
    b.build()
    from paper_2407_20304_gb300 import _lib
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "holo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(holo_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2407_20304_gb300 import _lib
    decl = _declared()
    assert len(decl) >= 16
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTS) == decl


def test_status_strings(lib):
    from paper_2407_20304_gb300 import _lib
    for s in range(9):
        assert lib.holo_status_string(s)
    assert lib.holo_status_string(8) == b"device bounds check failed"
    assert lib.holo_last_error(None) == b""
    # every status of the header's enum has a name in the binding
    src = open(os.path.join(ROOT, "include", "holo.h")).read()
    enum = {int(v): k for k, v in re.findall(r"\b(HOLO_(?:OK|ERR_[A-Z]+))\s*=\s*(\d+)", src)}
    assert enum == {k: v for k, v in _lib.STATUS.items()} | {0: "HOLO_OK"}


def test_bounds_check_build_variant():
    """The HOLO_BOUNDS_CHECK variant: its own flag and output directory, selected by the
    environment (nothing is compiled here; the -m gpu tests build and run it)."""
    import subprocess
    import sys
    from paper_2407_20304_gb300 import build as b
    assert "-DHOLO_BOUNDS_CHECK" in b.compile_flags(bounds_check=True)
    assert "-DHOLO_BOUNDS_CHECK" not in b.compile_flags()
    code = "from paper_2407_20304_gb300 import _lib; print(_lib.LIB_PATH)"
    env = dict(os.environ, HOLO_BOUNDS_CHECK="1")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, check=True).stdout.strip()
    assert out.endswith(os.path.join("_build_bc", "libholo.so"))
    env["HOLO_BOUNDS_CHECK"] = "0"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, check=True).stdout.strip()
    assert out.endswith(os.path.join("_build", "libholo.so"))


def _geo(**kw):
    from paper_2407_20304_gb300 import _lib
    g = _lib.HoloGeometry()
    base = dict(n=64, pad=128, n_angles=4, n_dist=4, chunk=0, wavelength=3.72e-11, pixel=1e-8,
                Z=1.208, w_ref=1.0, ext=1.0)
    base.update({k: v for k, v in kw.items() if k != "z"})
    for k, v in base.items():
        setattr(g, k, v)
    for j, z in enumerate(kw.get("z", (4.6e-4, 5.1e-4, 6.2e-4, 8.3e-4))):
        g.z[j] = z
    return g


@pytest.mark.parametrize("kw,expect", [
    (dict(n=63), 1), (dict(n=8), 1), (dict(pad=32), 1), (dict(n_dist=0), 1), (dict(n_dist=9), 1),
    (dict(z=(5e-4, 4e-4, 6e-4, 7e-4)), 1), (dict(z=(4e-4, 5e-4, 6e-4, 2.0)), 1),
    (dict(wavelength=-1.0), 1), (dict(chunk=9), 1), (dict(n_angles=0), 1),
    (dict(pad=80), 7), (dict(pad=112), 7), (dict(pad=6144, n=64), 7), (dict(pad=8192, n=64), 7),
])
def test_create_rejects_bad_geometry(lib, kw, expect):
    g = _geo(**kw)
    out = ctypes.c_void_p(123)
    st = lib.holo_create(ctypes.byref(g), None, ctypes.byref(out))
    assert st == expect
    assert out.value is None


def test_null_arguments(lib):
    assert lib.holo_create(None, None, None) == 1
    assert lib.holo_destroy(None) == 0
    d = ctypes.c_double()
    assert lib.holo_forward(None, 0, 1, None, None, ctypes.byref(d)) == 1
    assert lib.holo_gradient(None, 0, 1, None, None, None, None, 0) == 1
    assert lib.holo_dot(None, None, None, 0, ctypes.byref(d)) == 1
    assert lib.holo_step(None, None, None, 1.0, 0) == 1


def test_injected_allocation_failure_needs_no_gpu(lib, monkeypatch):
    """HOLO_FAULT=alloc fails the first workspace allocation of holo_create before cudaMalloc
    (HOLO_ERR_OOM) and returns no context; the check runs on the host only."""
    monkeypatch.setenv("HOLO_FAULT", "alloc")
    g = _geo()
    out = ctypes.c_void_p(123)
    assert lib.holo_create(ctypes.byref(g), None, ctypes.byref(out)) == 3
    assert out.value is None
    # an invalid geometry is still reported as such (validation comes first)
    g = _geo(n=63)
    assert lib.holo_create(ctypes.byref(g), None, ctypes.byref(out)) == 1


def test_device_error_hook_rejects_a_null_context(lib):
    assert lib.holo_set_device_error(None, 1) == 1


def _prototypes():
    """{name: [parameter type strings]} of the function declarations in include/holo.h."""
    src = open(os.path.join(ROOT, "include", "holo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w ]*?[\s\*]+)(holo_[a-z_0-9]+)\s*\(([^)]*)\)\s*;",
                                        src):
        ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        out[name] = ps
    return out


def test_binding_prototypes_match_the_header():
    """Every ctypes prototype of the binding has the header's parameter count, and pointer
    parameters are bound as pointers, integers as integers and doubles as doubles."""
    from paper_2407_20304_gb300 import _lib
    protos = _prototypes()
    assert sorted(protos) == sorted(_lib.EXPORTS)
    sigs = _lib._signatures()
    assert sorted(sigs) == sorted(set(protos) - {"holo_status_string", "holo_last_error"})
    for name, params in protos.items():
        if name not in sigs:
            continue
        args = sigs[name]
        assert len(args) == len(params), (name, params, args)
        for p, a in zip(params, args):
            if "*" in p:
                assert a is ctypes.c_void_p or issubclass(a, ctypes._Pointer), (name, p, a)
            elif p.startswith("double"):
                assert a is ctypes.c_double, (name, p, a)
            elif p.startswith(("int", "long long", "unsigned", "holo_status")):
                assert a in (ctypes.c_int, ctypes.c_longlong, ctypes.c_uint,
                             ctypes.c_ulonglong), (name, p, a)
