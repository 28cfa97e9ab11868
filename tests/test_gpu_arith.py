"""The Newton-refined FP64 reciprocal / quotient of the Godunov kernels against
IEEE division (CUDA's `/` through torch) -- within 2 ulp over a wide range."""
import ctypes

import numpy as np
import pytest

from paper_1710_08774_gb300 import hfav as H

pytestmark = pytest.mark.gpu


def test_rcp_and_quotient_within_two_ulp():
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-12, 12, 200000), rng.uniform(0.5, 2.0, 50000),
                        -10.0 ** rng.uniform(-6, 6, 50000)])
    xt = torch.from_numpy(x).cuda()
    r = torch.empty_like(xt); q = torch.empty_like(xt)
    H.check(H.load().hfav_selftest_arith(ctypes.c_void_p(xt.data_ptr()), xt.numel(), ctypes.c_void_p(r.data_ptr()),
                                         ctypes.c_void_p(q.data_ptr()), None))
    torch.cuda.synchronize()
    ref_r = (1.0 / xt).cpu().numpy(); ref_q = (1.5 / xt).cpu().numpy()
    for got, ref in ((r.cpu().numpy(), ref_r), (q.cpu().numpy(), ref_q)):
        ulp = np.spacing(np.abs(ref))
        assert np.max(np.abs(got - ref) / ulp) <= 2.0


def test_refined_rsqrt_within_2_pow_minus_38():
    """The FP32-bulk Newton iteration's FP64 reciprocal square root (hardware
    estimate + one Newton-Raphson step) against CUDA's rsqrt: one step takes
    the estimate's relative error e to about 1.5 e^2, 2^-38 here -- some 100x
    below the iteration's 1e-10 stopping tolerance."""
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([10.0 ** rng.uniform(-12, 12, 200000), rng.uniform(0.1, 10.0, 100000)])
    xt = torch.from_numpy(x).cuda()
    r = torch.empty_like(xt)
    H.check(H.load().hfav_selftest_rsqrt(ctypes.c_void_p(xt.data_ptr()), xt.numel(), ctypes.c_void_p(r.data_ptr()),
                                         None))
    torch.cuda.synchronize()
    ref = torch.rsqrt(xt).cpu().numpy()
    assert np.max(np.abs(r.cpu().numpy() - ref) / ref) <= 2.0 ** -38
