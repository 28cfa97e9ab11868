"""The allocation-free entry point hfav_chain2d_static against the planned path.

hfav_chain2d_static serves callers that cannot allocate device memory while
running; its only scratch is a static device array inside the library.  This
test calls it through the C ABI twice in a row (the second call reuses the
array the first one left behind) and checks both results against the planned
"sweep" schedule of hfav_run, within the FP64 tolerance of the chain tests
(1e-12 normwise).  It also checks that a grid too large for the array is
refused on the host.  Collected last so that a failure here does not hide the
other GPU tests in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _planned(ut, bc):
    import torch
    out = torch.full_like(ut, float("nan"))
    P = H.Plan(H.chain2d_dag(), [H.Grid.of(ut, 2)], H.HFAV_F64, bc, "sweep:reg:32x4")
    P.run([ut], [out])
    torch.cuda.synchronize()
    return out[2:-2, 2:-2].cpu().numpy()


def _static(ut, bc):
    import torch
    ny, nx = ut.shape[0] - 4, ut.shape[1] - 4
    out = torch.full_like(ut, float("nan"))
    rc = H.load().hfav_chain2d_static(ctypes.c_void_p(ut.data_ptr()), nx, ny, ut.stride(0), 2, bc, None,
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    H.check(rc)
    torch.cuda.synchronize()
    return out[2:-2, 2:-2].cpu().numpy()


def _err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("shape", [(256, 256), (130, 67)])
def test_static_matches_planned_twice(shape):
    import torch
    nx, ny = shape
    u1 = torch.from_numpy(I.chain2d_input(nx, seed=0, ny=ny)).cuda()
    u2 = torch.from_numpy(I.chain2d_input(nx, seed=1, ny=ny)).cuda()
    ref1 = _planned(u1, H.HFAV_BC_PERIODIC)
    ref2 = _planned(u2, H.HFAV_BC_PERIODIC)
    got1 = _static(u1, H.HFAV_BC_PERIODIC)
    got2 = _static(u2, H.HFAV_BC_PERIODIC)
    assert _err(got1, ref1) <= 1e-12
    assert _err(got2, ref2) <= 1e-12


def test_static_halo_given_matches_planned():
    import torch
    j, i = np.meshgrid(np.arange(-2, 70), np.arange(-2, 52), indexing="ij")
    u = torch.from_numpy(np.sin(0.3 * i) * np.cos(0.2 * j) + 0.01 * i * j).cuda()
    ref = _planned(u, H.HFAV_BC_HALO_GIVEN)
    for _ in range(2):
        assert _err(_static(u, H.HFAV_BC_HALO_GIVEN), ref) <= 1e-12


def test_static_rejects_grid_beyond_capacity():
    # (nx+2)*(ny+2)*8 > 16 MiB is refused before any device work
    rc = H.load().hfav_chain2d_static(ctypes.c_void_p(16), 2048, 2048, 2052, 2, H.HFAV_BC_PERIODIC, None,
                                      ctypes.c_void_p(32), None)
    assert rc == -1
    assert b"16777216" in H.load().hfav_last_error()
