"""The allocation-free entry point hfav_chain2d_static against the oracle and the planned path.

hfav_chain2d_static serves callers that cannot allocate device memory while
running; its only scratch is a static device array inside the library.  These
tests call it through the C ABI twice in a row (the second call reuses the
array the first one left behind) and check both results against the CPU
oracle (oracle.chain2d) and the planned "sweep" schedule of hfav_run, within
the FP64 tolerance of the chain tests (1e-12 normwise); non-default weights
are checked against a planned run with the same weights and a numpy
evaluation; the device's free memory is unchanged across a call after the
first; a grid too large for the array is refused on the host.  Collected
last so that a failure here does not hide the other GPU tests in a run that
stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _weighted_dag(w):
    D = H.DagSpec(2, stream_axis=1)
    D.rule("STENCIL_LINEAR", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))], ["L"],
           params=list(w))
    D.rule("GRADMAG_HALF", [("L", (1, 0)), ("L", (-1, 0)), ("L", (0, 1)), ("L", (0, -1))], ["G"])
    D.rule("SQUASH", ["G"], ["out"])
    D.axiom("u")
    D.goal("out")
    return D


def _planned(ut, bc, w=None):
    import torch
    out = torch.full_like(ut, float("nan"))
    dag = H.chain2d_dag() if w is None else _weighted_dag(w)
    P = H.Plan(dag, [H.Grid.of(ut, 2)], H.HFAV_F64, bc, "sweep:reg:32x4")
    P.run([ut], [out])
    torch.cuda.synchronize()
    return out[2:-2, 2:-2].cpu().numpy()


def _static(ut, bc, w=None, out=None):
    import torch
    ny, nx = ut.shape[0] - 4, ut.shape[1] - 4
    out = torch.full_like(ut, float("nan")) if out is None else out
    wts = None if w is None else (ctypes.c_double * 5)(*w)
    rc = H.load().hfav_chain2d_static(ctypes.c_void_p(ut.data_ptr()), nx, ny, ut.stride(0), 2, bc, wts,
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    H.check(rc)
    torch.cuda.synchronize()
    return out[2:-2, 2:-2].cpu().numpy()


def _err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("shape", [(256, 256), (130, 67), (8, 8)])
def test_static_matches_oracle_and_planned_twice(shape):
    import torch
    nx, ny = shape
    h1 = I.chain2d_input(nx, seed=0, ny=ny)
    h2 = I.chain2d_input(nx, seed=1, ny=ny)
    u1 = torch.from_numpy(h1).cuda()
    u2 = torch.from_numpy(h2).cuda()
    ref1 = _planned(u1, H.HFAV_BC_PERIODIC)
    ref2 = _planned(u2, H.HFAV_BC_PERIODIC)
    got1 = _static(u1, H.HFAV_BC_PERIODIC)
    got2 = _static(u2, H.HFAV_BC_PERIODIC)
    assert _err(got1, oracle.chain2d(h1)[2]) <= 1e-12
    assert _err(got2, oracle.chain2d(h2)[2]) <= 1e-12
    assert _err(got1, ref1) <= 1e-12
    assert _err(got2, ref2) <= 1e-12


def _numpy_chain(core, w):
    """The chain on a periodic interior with stencil weights w, by np.roll."""
    L = (w[0] * np.roll(core, -1, 1) + w[1] * np.roll(core, 1, 1) + w[2] * np.roll(core, -1, 0)
         + w[3] * np.roll(core, 1, 0) + w[4] * core)
    gx = np.roll(L, -1, 1) - np.roll(L, 1, 1)
    gy = np.roll(L, -1, 0) - np.roll(L, 1, 0)
    G = np.sqrt(gx * gx + gy * gy) / 2
    return G / (1 + G)


def test_static_weights_match_planned_and_numpy():
    import torch
    w = (0.5, 1.5, -1.0, 2.0, -3.0)
    h = I.chain2d_input(100, seed=3, ny=61)
    u = torch.from_numpy(h).cuda()
    ref = _planned(u, H.HFAV_BC_PERIODIC, w)
    for _ in range(2):
        got = _static(u, H.HFAV_BC_PERIODIC, w)
        assert _err(got, ref) <= 1e-12
        assert _err(got, _numpy_chain(h[2:-2, 2:-2], w)) <= 1e-12


def test_static_allocates_nothing_after_the_first_call():
    import torch
    u = torch.from_numpy(I.chain2d_input(512, seed=2, ny=300)).cuda()
    out = torch.full_like(u, float("nan"))
    _static(u, H.HFAV_BC_PERIODIC, out=out)       # loads the module (and its array) on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        _static(u, H.HFAV_BC_PERIODIC, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_halo_given_matches_planned():
    import torch
    j, i = np.meshgrid(np.arange(-2, 70), np.arange(-2, 52), indexing="ij")
    u = torch.from_numpy(np.sin(0.3 * i) * np.cos(0.2 * j) + 0.01 * i * j).cuda()
    ref = _planned(u, H.HFAV_BC_HALO_GIVEN)
    for _ in range(2):
        assert _err(_static(u, H.HFAV_BC_HALO_GIVEN), ref) <= 1e-12


def test_static_rejects_grid_beyond_capacity():
    # (nx+2)*(ny+2)*8 > 16 MiB is refused before any device work
    rc = H.load().hfav_chain2d_static(ctypes.c_void_p(1 << 32), 2048, 2048, 2052, 2, H.HFAV_BC_PERIODIC, None,
                                      ctypes.c_void_p(1 << 40), None)
    assert rc == -1
    assert b"16777216" in H.load().hfav_last_error()
