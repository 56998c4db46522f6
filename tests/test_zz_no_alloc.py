"""The allocation-free entry point (morlet_forward_noalloc) against the regular plan-based forward.

Some callers cannot allocate device memory (their framework or allocator owns all of it); this entry
point keeps every working buffer in a fixed array inside the library. Its output must equal that of
morlet_plan + morlet_forward with the same parameters, on two calls in a row (the second call reuses
the array the first one left behind). The file is named to run last, so that a failure here does
not stop the other tests of a `-x` run.
"""
import ctypes

import numpy as np
import pytest

import paper_2110_11866_gb300 as m

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("N,sigma,K", [(50000, 8.0, 4), (200000, 3000.0, 6)])
def test_noalloc_matches_plan_forward_twice(N, sigma, K):
    import torch
    rng = np.random.default_rng(N)
    x = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    plan = m.morlet_plan([N], [sigma], xi=6.0, K=K, precision=m.MORLET_FP32_COMP)
    ref = torch.empty(N, dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, x, ref)
    torch.cuda.synchronize()
    lib = m.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        W = torch.full((N,), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda")
        rc = lib.morlet_forward_noalloc(ctypes.c_void_p(x.data_ptr()), N, sigma, 6.0, K,
                                        ctypes.c_void_p(W.data_ptr()), stream)
        assert rc == m.MORLET_OK, m.morlet_strerror(rc)
        torch.cuda.synchronize()
        err = float((W - ref).abs().max() / ref.abs().max())
        assert err <= 1e-5, (call, err)


def test_noalloc_rejects_sizes_beyond_its_array():
    lib = m.lib()
    # 2^27 outputs need more than the 16384 sub-tiles the fixed array can describe
    rc = lib.morlet_forward_noalloc(ctypes.c_void_p(16), 1 << 27, 8.0, 6.0, 4, ctypes.c_void_p(16), None)
    assert rc == m.MORLET_ERR_ARG
