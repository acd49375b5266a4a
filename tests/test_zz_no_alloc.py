"""The no-allocation risk-measure entry point against ara_risk_measures.

ara_risk_measures_noalloc() is for callers that cannot allocate device memory when they need
PML/TVaR (inside a pre-sized pool or a foreign allocator, in a real-time loop that must not meet
cudaMalloc's synchronisation, or without an ara_ctx).  It must return what ara_risk_measures
returns on the same YLT, call after call, although every call reuses the same fixed scratch.

The test calls the C ABI directly through ctypes.  It lives in a file of its own that pytest
collects last, and passes alone in a fresh process as well as after the other tests.
"""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_TRIALS = 1 << 20


def entry(ara):
    fn = ara.lib().ara_risk_measures_noalloc
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                   C.c_void_p]
    fn.restype = C.c_int
    return fn


def call(fn, ylt_dev, rps):
    import torch

    r = np.ascontiguousarray(rps, dtype=np.float64)
    pml = torch.full((len(rps),), -1.0, dtype=torch.float64, device="cuda")
    tvar = torch.full((len(rps),), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = fn(ylt_dev.data_ptr(), ylt_dev.numel(), r.ctypes.data, len(rps), pml.data_ptr(),
            tvar.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return st, pml.cpu().numpy(), tvar.cpu().numpy()


def test_noalloc_matches_risk_measures_twice_in_a_row(ara):
    import torch

    fn = entry(ara)
    rng = np.random.default_rng(2024)
    cases = [
        (np.maximum(rng.lognormal(19.0, 0.6, 800_000) - 1.5e8, 0.0), [100.0, 250.0, 500.0, 1000.0]),
        (rng.choice([0.0, 3.0, 5e7, 1.25e6], size=1000), [1.5, 10.0, 100.0, 250.0]),
    ]
    with ara.Context(seed=42) as ctx:
        for y, rps in cases:
            ref_p, ref_t = ctx.risk_measures(y, rps)
            yd = torch.from_numpy(y).cuda()
            for _ in range(2):  # two calls in a row on the shared scratch
                st, p, t = call(fn, yd, rps)
                assert st == 0
                np.testing.assert_array_equal(p, ref_p)
                np.testing.assert_allclose(t, ref_t, rtol=1e-13)


def test_noalloc_rejects_what_it_cannot_hold(ara):
    import torch

    fn = entry(ara)
    too_long = torch.zeros(MAX_TRIALS + 1, dtype=torch.float64, device="cuda")
    st, _, _ = call(fn, too_long, [100.0])
    assert st == 1  # ARA_ERR_INVALID_ARG
    host = np.zeros(10)
    pml = torch.zeros(1, dtype=torch.float64, device="cuda")
    tvar = torch.zeros(1, dtype=torch.float64, device="cuda")
    rps = np.array([10.0])
    assert fn(host.ctypes.data, 10, rps.ctypes.data, 1, pml.data_ptr(), tvar.data_ptr(),
              None) == 1  # a host YLT is refused
    ok = torch.ones(10, dtype=torch.float64, device="cuda")
    bad_rp = np.array([1.0])
    assert fn(ok.data_ptr(), 10, bad_rp.ctypes.data, 1, pml.data_ptr(), tvar.data_ptr(),
              None) == 1
