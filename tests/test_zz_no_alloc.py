"""Decompression without a caller workspace (pc_decompress_noalloc).

Callers that cannot allocate device memory when they decompress (under a
device-memory budget fixed up front, or as a plugin that only gets an input
and an output buffer) use pc_decompress_noalloc, which takes its scratch
space from a fixed array built into the library.  This test calls it
through the C ABI and checks that it returns exactly what pc_decompress (with
a caller workspace) returns, on two calls in a row, and that a container
needing more scratch than the built-in array is refused before any work.
The file sorts last so that a run stopping at the first failure has already
run every other test; it passes alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_09778_gb300.pc as pcm
    return pcm


def call_noalloc(pc, blob, out):
    fn = pc.lib().pc_decompress_noalloc
    dims = (C.c_size_t * 3)()
    dt = C.c_int()
    st = fn(C.c_void_p(blob.data_ptr()), blob.numel(), C.c_void_p(out.data_ptr()),
            out.numel() * out.element_size(), dims, C.byref(dt),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, tuple(dims), dt.value


def test_noalloc_matches_workspace_decompress_twice(pc):
    from paper_2309_09778_gb300 import gen
    cases = [((40, 90, 100), 1e-3, np.float32), ((33, 64, 70), 1e-2, np.float32), ((17, 30, 41), 1e-5, np.float64)]
    for i, (shape, eb, dt) in enumerate(cases):
        x = gen.signed_lognormal(shape, 11.0 / 3.0, i, 2.0, 0.02, dtype=dt)
        d = torch.from_numpy(x).cuda()
        blob = pc.compress(d, pc.make_params(eb, (8, 8, 8)))
        ref = pc.decompress(blob)
        view = torch.int32 if dt == np.float32 else torch.int64
        for _ in range(2):
            out = torch.full_like(ref, float("nan"))
            st, dims, dtype = call_noalloc(pc, blob, out)
            assert st == 0, pc.pc_strerror(st)
            torch.cuda.synchronize()
            assert dims == shape and dtype == (0 if dt == np.float32 else 1)
            assert torch.equal(out.view(view), ref.view(view))


def test_noalloc_refuses_fields_beyond_the_scratch(pc):
    shape = (300, 256, 256)  # needs about 40 MB of scratch, more than the built-in 32 MiB
    d = torch.ones(shape, dtype=torch.float32, device="cuda")
    blob = pc.compress(d, pc.make_params(1e-2, (8, 8, 8)))
    out = torch.zeros_like(d)
    st, _, _ = call_noalloc(pc, blob, out)
    assert st == -4
    assert torch.count_nonzero(out).item() == 0
