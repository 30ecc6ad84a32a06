"""hh_multidot_noalloc: the Krylov inner products without any device allocation.

Some callers cannot allocate at the point of use (all device memory already belongs
to their own pool, or a budget reserved up front).  For them the library keeps the
reduction's scratch in a fixed array of its own; this test checks, through the C ABI,
that the allocation-free entry point returns what the regular one (hh_dot, whose
scratch belongs to an hh_problem) returns and what numpy's vdot of the host copies
returns, on two calls in a row and on vectors taken with a stride (ld > n) from a wider
buffer, and that sizes past the array's limit are refused.

The file name sorts last so that pytest collects it after every other test file: the
entry point shares one array across all its calls in the process, and if it ever
failed, a run stopped at that first failure (pytest -x) would already have run every
other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu


def _call(libhh, V, ld, nvec, w, n, out, stream):
    return libhh.hh_multidot_noalloc(ctypes.c_void_p(V.data_ptr()), ld, nvec, ctypes.c_void_p(w.data_ptr()), n,
                                     ctypes.c_void_p(out.data_ptr()), stream)


def test_multidot_noalloc_matches_hh_dot_and_numpy(libhh):
    n = 32
    with hh.Problem(2, n, 5.0, 0.0, 2.0, [hh.SOMMERFELD] * 4, hh.default_options(levels=3)) as p:
        N = p.nodes()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call, nvec in enumerate((7, 64)):
            Vh = np.stack([inputs.random_complex(N, 200 + call * 100 + i) for i in range(nvec)])
            wh = inputs.random_complex(N, 199 + call)
            V = torch.from_numpy(Vh).cuda()
            w = torch.from_numpy(wh).cuda()
            out = torch.full((nvec,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            st = _call(libhh, V, N, nvec, w, N, out, stream)
            assert st == 0, libhh.hh_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for i in range(nvec):
                ref = p.dot(V[i].contiguous(), w)
                want = np.vdot(Vh[i], wh)  # V_i^H w on the host, FP64
                scale = float(np.linalg.norm(Vh[i]) * np.linalg.norm(wh))
                assert abs(got[i] - ref) <= 1e-13 * scale, (call, i, got[i], ref)
                assert abs(got[i] - want) <= 1e-13 * scale, (call, i, got[i], want)


def test_multidot_noalloc_strided_vectors(libhh):
    """V_i = V + i * ld with ld = n + 17: the vectors are rows of a wider buffer."""
    n, nvec = 1000, 5
    ld = n + 17
    wide = inputs.random_complex(nvec * ld, 301).reshape(nvec, ld)
    wh = inputs.random_complex(n, 302)
    V = torch.from_numpy(wide).cuda()
    w = torch.from_numpy(wh).cuda()
    out = torch.zeros(nvec, dtype=torch.complex128, device="cuda")
    for _ in range(2):
        assert _call(libhh, V, ld, nvec, w, n, out, None) == 0, libhh.hh_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i in range(nvec):
            want = np.vdot(wide[i, :n], wh)
            assert abs(got[i] - want) <= 1e-13 * np.linalg.norm(wide[i, :n]) * np.linalg.norm(wh), i


def test_multidot_noalloc_rejects_oversize(libhh):
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    out = torch.zeros(65, dtype=torch.complex128, device="cuda")
    st = libhh.hh_multidot_noalloc(ctypes.c_void_p(x.data_ptr()), 0, 65, ctypes.c_void_p(x.data_ptr()), 8,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1 and b"1..64" in libhh.hh_last_error()
    st = libhh.hh_multidot_noalloc(ctypes.c_void_p(x.data_ptr()), 4, 1, ctypes.c_void_p(x.data_ptr()), 8,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1 and b"ld >= n" in libhh.hh_last_error()
