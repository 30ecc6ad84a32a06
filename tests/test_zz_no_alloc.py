"""hh_multidot_noalloc: the Krylov inner products without any device allocation.

Some callers cannot allocate at the point of use (all device memory already belongs
to their own pool, or a budget reserved up front).  For them the library keeps the
reduction's scratch in a fixed array of its own; this test checks, through the C ABI,
that the allocation-free entry point returns what the regular one (hh_dot, whose
scratch belongs to an hh_problem) returns, on two calls in a row, and that sizes past
the array's limit are refused.  The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu


def test_multidot_noalloc_matches_hh_dot(libhh):
    n = 32
    with hh.Problem(2, n, 5.0, 0.0, 2.0, [hh.SOMMERFELD] * 4, hh.default_options(levels=3)) as p:
        N = p.nodes()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call, nvec in enumerate((7, 64)):
            V = torch.from_numpy(np.stack([inputs.random_complex(N, 200 + call * 100 + i)
                                           for i in range(nvec)])).cuda()
            w = torch.from_numpy(inputs.random_complex(N, 199 + call)).cuda()
            out = torch.full((nvec,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            st = libhh.hh_multidot_noalloc(ctypes.c_void_p(V.data_ptr()), N, nvec, ctypes.c_void_p(w.data_ptr()),
                                           N, ctypes.c_void_p(out.data_ptr()), stream)
            assert st == 0, libhh.hh_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for i in range(nvec):
                ref = p.dot(V[i].contiguous(), w)
                scale = float(torch.linalg.vector_norm(V[i]) * torch.linalg.vector_norm(w))
                assert abs(got[i] - ref) <= 1e-13 * scale, (call, i, got[i], ref)


def test_multidot_noalloc_rejects_oversize(libhh):
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    out = torch.zeros(65, dtype=torch.complex128, device="cuda")
    st = libhh.hh_multidot_noalloc(ctypes.c_void_p(x.data_ptr()), 0, 65, ctypes.c_void_p(x.data_ptr()), 8,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1 and b"1..64" in libhh.hh_last_error()
