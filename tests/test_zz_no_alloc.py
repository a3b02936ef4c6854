"""holo_dot_noalloc, the inner product for callers that cannot allocate device memory.

It keeps its partial sums in a fixed array inside the library instead of a context's
workspace.  Checked through the C ABI against the allocating holo_dot on two calls in a
row (the second call reuses the array left by the first).  Collected last, so a failure
here stops a -x run only after every other test has run.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_20304_gb300 import _lib
    return _lib.load()


def _noalloc(lib, a, b):
    out = ctypes.c_double(0.0)
    st = lib.holo_dot_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                              a.numel(), ctypes.byref(out),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return out.value


def test_noalloc_dot_matches_holo_dot_twice(lib):
    from paper_2407_20304_gb300 import Holo
    h = Holo(16, 1, 1, 3.72e-11, 1e-8, 1.208, (4.6e-4,), pad=32)
    gen = torch.Generator(device="cuda").manual_seed(7)
    for n in (1, 4097, 1_000_003):
        a = torch.randn(n, dtype=torch.complex64, device="cuda", generator=gen)
        b = torch.randn(n, dtype=torch.complex64, device="cuda", generator=gen)
        ref = h.dot(a, b)
        first = _noalloc(lib, a, b)
        second = _noalloc(lib, a, b)
        assert abs(first - ref) <= TOL * (abs(ref) + 1.0)
        assert abs(second - ref) <= TOL * (abs(ref) + 1.0)
        assert first == second
    h.close()


def test_noalloc_dot_rejects_oversize_without_device_work(lib):
    from paper_2407_20304_gb300 import _lib
    a = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = ctypes.c_double(123.0)
    st = lib.holo_dot_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                              _lib.NOALLOC_MAX_ELEMENTS + 1, ctypes.byref(out), None)
    assert st == 7 and out.value == 123.0
    st = lib.holo_dot_noalloc(None, None, 4, ctypes.byref(out), None)
    assert st == 1


def test_noalloc_dot_of_zero_elements_is_zero(lib):
    """n = 0 launches only the final reduction, over no partials: the result is 0.0 even
    though the array still holds the previous call's partial sums."""
    a = torch.ones(8, dtype=torch.complex64, device="cuda")
    assert _noalloc(lib, a, a) == 8.0
    out = ctypes.c_double(123.0)
    st = lib.holo_dot_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), 0,
                              ctypes.byref(out),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0 and out.value == 0.0


def test_noalloc_dot_rejects_host_memory_before_device_work(lib):
    """Inputs that are not device memory of the current device are refused on the host
    (HOLO_ERR_ARG), before any launch; the output is left untouched."""
    host = np.ones(16, np.complex64)
    a = torch.ones(16, dtype=torch.complex64, device="cuda")
    out = ctypes.c_double(123.0)
    for pa, pb in ((host.ctypes.data, a.data_ptr()), (a.data_ptr(), host.ctypes.data)):
        st = lib.holo_dot_noalloc(ctypes.c_void_p(pa), ctypes.c_void_p(pb), 16,
                                  ctypes.byref(out), None)
        assert st == 1 and out.value == 123.0


def test_noalloc_python_wrapper_matches_holo_dot(lib):
    from paper_2407_20304_gb300 import Holo
    from paper_2407_20304_gb300.holo import dot_noalloc
    h = Holo(16, 1, 1, 3.72e-11, 1e-8, 1.208, (4.6e-4,), pad=32)
    gen = torch.Generator(device="cuda").manual_seed(11)
    a = torch.randn(70001, dtype=torch.complex64, device="cuda", generator=gen)
    b = torch.randn(70001, dtype=torch.complex64, device="cuda", generator=gen)
    ref = h.dot(a, b)
    for _ in range(2):
        assert abs(dot_noalloc(a, b) - ref) <= TOL * (abs(ref) + 1.0)
    with pytest.raises(ValueError):
        dot_noalloc(a.cpu(), b.cpu())
    h.close()
