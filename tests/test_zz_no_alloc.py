"""The allocation-free entry point (morlet_forward_noalloc) against the oracle and the plan path.

Some callers cannot allocate device memory: code running under an allocator or framework that owns
all of the GPU's memory, where a cudaMalloc inside a library would fail or break its accounting. For
them the library keeps every working buffer of one transform in a fixed device array of its own.
This file checks that entry point through the C ABI: its output agrees with the oracle's O-SFT (the
double-double kernel integral) and with morlet_plan + morlet_forward within the compensated-FP32
gate, on two calls in a row (the second call reuses the array the first one left behind). The file
is named to run last, so that a failure here does not stop the other tests of a `-x` run.
"""
import ctypes

import numpy as np
import pytest

import paper_2110_11866_gb300 as m
from oracle import morlet as om
from oracle import sft_dd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("N,sigma,K", [(50000, 8.0, 4), (200000, 3000.0, 6), (100003, 300.0, 3)])
def test_noalloc_matches_oracle_and_plan_forward_twice(N, sigma, K):
    import torch
    rng = np.random.default_rng(N)
    xh = rng.standard_normal(N).astype(np.float32)
    x = torch.from_numpy(xh).cuda()
    ref = sft_dd.sft_direct_method(xh.astype(np.float64), om.fit_direct(sigma, 6.0, K))
    scale = np.abs(ref).max()
    plan = m.morlet_plan([N], [sigma], xi=6.0, K=K, precision=m.MORLET_FP32_COMP)
    Wp = torch.empty(N, dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, x, Wp)
    torch.cuda.synchronize()
    Wp = Wp.cpu().numpy()
    lib = m.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        W = torch.full((N,), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda")
        rc = lib.morlet_forward_noalloc(ctypes.c_void_p(x.data_ptr()), N, sigma, 6.0, K,
                                        ctypes.c_void_p(W.data_ptr()), stream)
        assert rc == m.MORLET_OK, m.morlet_strerror(rc)
        torch.cuda.synchronize()
        Wh = W.cpu().numpy()
        e_oracle = float(np.abs(Wh - ref).max() / scale)
        e_plan = float(np.abs(Wh - Wp).max() / scale)
        print(f"noalloc N={N} sigma={sigma} K={K} call {call}: vs oracle {e_oracle:.2e}, vs plan {e_plan:.2e}")
        assert e_oracle <= 1e-5 and e_plan <= 2e-5, (call, e_oracle, e_plan)


def test_noalloc_rejects_sizes_beyond_its_array():
    lib = m.lib()
    # 2^27 samples at sigma = 8 need more than the 16384 work items the fixed array can describe
    rc = lib.morlet_forward_noalloc(ctypes.c_void_p(16), 1 << 27, 8.0, 6.0, 4, ctypes.c_void_p(16), None)
    assert rc == m.MORLET_ERR_ARG
