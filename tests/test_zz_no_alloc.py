"""fehom_mean_flux_noalloc: the volume average computed without allocating device memory.

Some callers cannot allocate device memory while they run (a fixed memory budget or pool that may
not grow, or code paths where cudaMalloc is not allowed).  This entry point keeps its scratch in a
fixed array inside the library.  The test calls it through the C ABI twice in a row and checks both
results against fehom_mean_flux (which allocates its scratch) to the FP64 operator tolerance used by
the other tests, and checks that a grid too large for the fixed array is rejected with a message.
It lives in a file of its own, collected last, so a failure here never hides the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, s, e, u):
    out = np.zeros(s.m)
    st = lib.fehom_mean_flux_noalloc(s.ctx, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.c_void_p(u.data_ptr()),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return st, out


@pytest.mark.parametrize("elem,physics,shape", [("hex8_3d", "elastic", (32, 24, 48)),
                                                 ("p1tri2_2d", "scalar", (64, 96))])
def test_noalloc_mean_flux_matches_allocating_call(elem, physics, shape):
    import torch
    from paper_2203_02962_gb300 import fehom, inputs
    lib = fehom.load_library()
    rng = np.random.default_rng(7)
    ids = rng.integers(0, 2, size=shape).astype(np.uint8)
    dim = len(shape)
    if physics == "elastic":
        mod = np.stack([inputs.isotropic_elastic_mandel(1.0, 0.3), inputs.isotropic_elastic_mandel(50.0, 0.2)])
    else:
        mod = np.stack([inputs.isotropic_conductivity(1.0, dim), inputs.isotropic_conductivity(20.0, dim)])
    s = fehom.Solver(elem, physics, tuple(shape[::-1]), ids, mod)
    u = torch.tensor(rng.standard_normal(s.c * s.N), device="cuda")
    e = np.ascontiguousarray(rng.standard_normal(s.m))
    ref = s.mean_flux(e, u)
    for _ in range(2):
        st, out = _call_noalloc(lib, s, e, u)
        assert st == 0, lib.fehom_last_error(s.ctx)
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2203_02962_gb300 import fehom, inputs
    lib = fehom.load_library()
    n = (1024, 1024, 1)
    ids = np.zeros((1024, 1024), np.uint8)
    s = fehom.Solver("p1tri2_2d", "scalar", n, ids, inputs.isotropic_conductivity(1.0, 2)[None])
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, _ = _call_noalloc(lib, s, np.ones(2), u)
    assert st == 2  # FEHOM_E_UNSUPPORTED_SIZE
    assert b"scratch" in lib.fehom_last_error(s.ctx)
    s.close()


def test_noalloc_refuses_a_stream_under_capture():
    """The call copies from host memory and waits for its stream, which a stream being captured into a
    CUDA graph does not allow: it returns FEHOM_E_STATE there, and the capture still ends cleanly."""
    import torch
    from paper_2203_02962_gb300 import fehom, inputs
    lib = fehom.load_library()
    shape = (16, 24, 32)
    ids = np.zeros(shape, np.uint8)
    stream = torch.cuda.Stream()
    s = fehom.Solver("hex8_3d", "scalar", shape[::-1], ids, inputs.isotropic_conductivity(1.0, 3)[None],
                     stream=stream)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    e = np.ones(3)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        st, _ = _call_noalloc(lib, s, e, u)
    assert st == 7  # FEHOM_E_STATE
    assert b"captured" in lib.fehom_last_error(s.ctx)
    st, out = _call_noalloc(lib, s, e, u)  # outside the capture it works again
    assert st == 0 and np.abs(out - s.mean_flux(e, u)).max() <= 1e-12 * np.abs(out).max()
    s.close()
