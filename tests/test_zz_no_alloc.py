"""rplu_dense_noalloc: the dense factorization for callers that cannot let a
library allocate device memory (for example code running under a framework
that owns the device through its own pooled allocator, or a service that
reserves all memory at start-up).  Its working memory is a fixed array inside
the library, shared by all calls.

Checked through the C-ABI: two calls in a row (the second finds the first
call's leftovers in the shared array) give the same pivots and factors as
rplu_dense, and a problem too large for the array is refused.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process (the first call sets
the array up).
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding  # noqa: E402  (raises if librplu.so is missing)

P, i64 = ctypes.c_void_p, ctypes.c_int64
lib = binding.lib
lib.rplu_dense_noalloc.restype = ctypes.c_int
lib.rplu_dense_noalloc.argtypes = [P, i64, i64, i64, ctypes.c_uint64, ctypes.POINTER(binding.Opts), P, P, P, P,
                                   ctypes.POINTER(i64)]

TDT = {"f32": torch.float32, "f64": torch.float64, "c64": torch.complex64, "c128": torch.complex128}
CODE = {"f32": 0, "f64": 1, "c64": 2, "c128": 3}


def _noalloc(A, k, seed, dt, pivot="random", given=None):
    n, m = A.shape
    I = torch.empty(k, dtype=torch.int64, device="cuda")
    J = torch.empty(k, dtype=torch.int64, device="cuda")
    L = torch.empty((k, n), dtype=TDT[dt], device="cuda")
    U = torch.empty((k, m), dtype=TDT[dt], device="cuda")
    o = binding.Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.dtype = CODE[dt]
    o.pivot = binding.PIVOTS[pivot]
    if given is not None:
        o.given_I, o.given_J = given[0].data_ptr(), given[1].data_ptr()
    o.stream = torch.cuda.current_stream().cuda_stream
    kd = i64(0)
    st = lib.rplu_dense_noalloc(A.data_ptr(), n, m, k, seed, ctypes.byref(o), I.data_ptr(), J.data_ptr(),
                                L.data_ptr(), U.data_ptr(), ctypes.byref(kd))
    return st, kd.value, I, J, L.T, U


def _input(dt, shape, seed=4):
    A = W.dense_haar_decay(*shape, 0.9, seed=seed)
    if dt.startswith("c"):
        A = A + 1j * W.dense_haar_decay(*shape, 0.9, seed=seed + 1)
    return torch.from_numpy(A).to(TDT[dt]).cuda()


# Both entry points launch the same kernels on the same data, so the results
# must be identical bit for bit, not merely close.
@pytest.mark.parametrize("dt,shape,k,pivot", [("f32", (700, 610), 90, "random"), ("f64", (300, 257), 40, "random"),
                                              ("c64", (260, 301), 30, "random"), ("c128", (150, 130), 25, "random"),
                                              ("f64", (120, 97), 30, "complete"), ("c128", (90, 70), 20, "c2"),
                                              ("f32", (200, 180), 24, "given")])
def test_noalloc_matches_dense_on_two_calls(dt, shape, k, pivot):
    A = _input(dt, shape)
    given = None
    if pivot == "given":
        rng = np.random.default_rng(3)
        given = (torch.from_numpy(rng.permutation(shape[0])[:k]).cuda(),
                 torch.from_numpy(rng.permutation(shape[1])[:k]).cuda())
    ref = rp.rplu_dense(A, k, seed=21, pivot=pivot,
                        given=None if given is None else (given[0].cpu().numpy(), given[1].cpu().numpy()))
    for call in range(2):
        st, kd, I, J, L, U = _noalloc(A, k, 21, dt, pivot, given)
        torch.cuda.synchronize()
        assert st == rp.RPLU_OK, f"call {call}: status {st}"
        assert kd == ref.k_done == k
        assert torch.equal(I, ref.I) and torch.equal(J, ref.J), f"call {call}: pivots differ"
        assert torch.equal(L, ref.L) and torch.equal(U, ref.U), f"call {call}: factors differ"


def test_noalloc_refuses_problems_beyond_its_array():
    A = torch.ones((4096, 4096), dtype=torch.float32, device="cuda")  # 64 MiB residual > 32 MiB array
    st, kd, I, J, L, U = _noalloc(A, 4, 1, "f32")
    assert st == rp.RPLU_ERR_NOMEM and kd == 0


def test_noalloc_needs_device_buffers():
    A = np.ones((8, 8))
    kd = i64(0)
    I = np.zeros(2, np.int64)
    L = np.zeros(16)
    st = lib.rplu_dense_noalloc(A.ctypes.data, 8, 8, 2, 0, None, I.ctypes.data, I.ctypes.data, L.ctypes.data,
                                L.ctypes.data, ctypes.byref(kd))
    assert st == rp.RPLU_ERR_INVALID
