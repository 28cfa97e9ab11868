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


def test_integer_halving_is_the_ieee_product_bit_for_bit():
    """The Godunov kernels halve FP64 values on the integer pipe: bit for bit
    x * 0.5 (round to nearest even) over zeros, subnormals, the smallest
    normals (whose halves are subnormal, with ties), the largest finite
    values, infinities and random values of every exponent; NaN stays NaN."""
    import torch
    rng = np.random.default_rng(2)
    tiny = np.finfo(np.float64).tiny          # smallest normal, exponent field 1
    sub = np.nextafter(0.0, 1.0)              # smallest subnormal
    special = np.array([0.0, -0.0, sub, -sub, 3 * sub, 2 * sub, tiny, -tiny, tiny * (2 - 2 ** -52),
                        np.nextafter(tiny, 0.0), np.nextafter(tiny, 1.0), 2 * tiny, np.nextafter(2 * tiny, 0.0),
                        np.finfo(np.float64).max, -np.finfo(np.float64).max, 1.0, -1.5, np.inf, -np.inf])
    bits = rng.integers(0, 2 ** 63 - 1, 400000, dtype=np.int64, endpoint=False)
    rand = bits.view(np.float64)
    rand = rand[np.isfinite(rand)]
    subs = rng.integers(1, 2 ** 52, 50000, dtype=np.int64).view(np.float64)   # subnormals and the e = 1 band
    x = np.concatenate([special, rand, -rand[:1000], subs, subs + tiny, 10.0 ** rng.uniform(-300, 300, 50000)])
    xt = torch.from_numpy(x).cuda()
    r = torch.empty_like(xt)
    H.check(H.load().hfav_selftest_half(ctypes.c_void_p(xt.data_ptr()), xt.numel(), ctypes.c_void_p(r.data_ptr()),
                                        None))
    torch.cuda.synchronize()
    got = r.cpu().numpy()
    ref = x * 0.5
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    nan = np.array([np.nan, -np.nan])
    nt = torch.from_numpy(nan).cuda()
    nr = torch.empty_like(nt)
    H.check(H.load().hfav_selftest_half(ctypes.c_void_p(nt.data_ptr()), nt.numel(), ctypes.c_void_p(nr.data_ptr()),
                                        None))
    torch.cuda.synchronize()
    assert np.all(np.isnan(nr.cpu().numpy()))


def test_integer_conversions_are_the_ieee_conversions_bit_for_bit():
    """The FP32-bulk Riemann solver widens its face states to FP64 and narrows
    the star state back on the integer pipe: bit for bit the IEEE conversions
    (narrowing rounds to nearest even, ties included) over random bit
    patterns of every exponent, values at and beyond FP32's range and its
    subnormals, zeros and infinities; NaN stays NaN."""
    import torch
    rng = np.random.default_rng(3)
    f32 = np.finfo(np.float32)
    bits = rng.integers(0, 2 ** 63 - 1, 300000, dtype=np.int64)
    xd = bits.view(np.float64)
    # doubles near FP32's grid: a float plus a dropped part of 0, exactly half an ulp, or just either side
    base = rng.standard_normal(100000).astype(np.float32).astype(np.float64) * 10.0 ** rng.integers(-30, 30, 100000)
    ulp = np.spacing(base.astype(np.float32)).astype(np.float64)
    ties = np.concatenate([base + 0.5 * ulp, base - 0.5 * ulp, base + 0.5 * ulp * (1 + 2 ** -40), base])
    edge = np.array([0.0, -0.0, float(f32.max), -float(f32.max), float(f32.max) * (1 + 2 ** -25),
                     float(f32.max) * (1 + 2 ** -23), float(f32.tiny), float(f32.tiny) * 0.75, float(f32.tiny) / 3,
                     1e-50, -1e-50, 1e50, np.inf, -np.inf, 1.0, -3.0])
    x = np.concatenate([xd[np.isfinite(xd)], ties, edge, 10.0 ** rng.uniform(-45, 39, 100000)])
    fb = rng.integers(0, 2 ** 32, x.size, dtype=np.int64).astype(np.uint32).view(np.float32).copy()
    fb[:16] = np.array([0.0, -0.0, f32.tiny, -f32.tiny, f32.tiny / 2, f32.max, -f32.max, np.inf, -np.inf, 1.0, -2.5,
                        1e-40, 3e-45, 1.5, 7.0, 1e30], dtype=np.float32)
    nan_f = np.isnan(fb)
    fb[nan_f] = 1.0
    xt = torch.from_numpy(x).cuda()
    ft = torch.from_numpy(fb).cuda()
    nr = torch.empty(x.size, dtype=torch.float32, device="cuda")
    wd = torch.empty(x.size, dtype=torch.float64, device="cuda")
    H.check(H.load().hfav_selftest_convert(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(ft.data_ptr()), x.size,
                                           ctypes.c_void_p(nr.data_ptr()), ctypes.c_void_p(wd.data_ptr()), None))
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        ref_n = x.astype(np.float32)
    assert np.array_equal(nr.cpu().numpy().view(np.uint32), ref_n.view(np.uint32))
    assert np.array_equal(wd.cpu().numpy().view(np.int64), fb.astype(np.float64).view(np.int64))
