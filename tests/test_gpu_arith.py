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
