"""The allocation-free entry point, d8_flowdir_accumulate_noalloc.

Some callers cannot allocate device memory when they call: a process running
under a fixed memory budget reserved at start-up, a caller whose own pool or
arena allocator owns every byte of the device, or a caller that cannot create
a library context (creating one allocates).  This entry point serves them from
a fixed scratch array inside the library.  These tests call it through the C
ABI and check that it returns exactly what d8_flowdir_accumulate returns, on
two calls in a row (the second reuses the scratch the first left behind), and
that a grid larger than the scratch is refused before any GPU work."""
import ctypes

import numpy as np
import pytest
import torch

import demgen
from paper_1605_05773_gb300 import build

pytestmark = pytest.mark.gpu
D8_ERR_CAPACITY = 8


@pytest.fixture(scope="module")
def noalloc(d8):
    L = ctypes.CDLL(build.LIB)
    f = L.d8_flowdir_accumulate_noalloc
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    f.argtypes = [vp, i64, i64, i64, i32, vp, i64, vp, i64, vp, vp]
    f.restype = i32
    return f


def _call(f, z, d, A, status, rule=0):
    H, W = z.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(z.data_ptr(), H, W, z.stride(0), rule, d.data_ptr(), d.stride(0), A.data_ptr(), A.stride(0),
             status.data_ptr(), stream)


def test_noalloc_matches_the_context_entry_point_twice(d8, noalloc):
    status = torch.full((1,), 0xFF, dtype=torch.int32, device="cuda")
    for k, (H, W, rule) in enumerate([(1500, 1300, "steepest"), (2900, 3100, "lowest")]):
        z = torch.from_numpy(demgen.fractal(H, W, seed=70 + k, cache=False)).cuda()
        d_ref, A_ref = d8.flowdir_accumulate(z, rule)
        assert d8.get_status() == "OK"
        d = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        A = torch.zeros((H, W), dtype=torch.int32, device="cuda")
        assert _call(noalloc, z, d, A, status, d8.RULES[rule]) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(d, d_ref)
        assert torch.equal(A, A_ref.view(torch.int32))


def test_noalloc_refuses_grids_beyond_its_scratch(noalloc):
    small = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    d = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    A = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    st = torch.zeros((1,), dtype=torch.int32, device="cuda")
    H = W = 10000  # 157^2 tiles of 64 x 64: more than the scratch holds; refused before any launch
    rc = noalloc(small.data_ptr(), H, W, W, 0, d.data_ptr(), W, A.data_ptr(), W, st.data_ptr(),
                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == D8_ERR_CAPACITY
