"""GPU parity of the COSMO horizontal diffusion (Sec. 5.3) against the oracle, through the C ABI.

FP64 bar: <= 1e-12 normwise; FP32 bar: <= 2e-5 normwise (a few FP32 roundings
on O(1) values).  Every schedule the pipeline runs is checked; ragged sizes;
the closed forms of the oracle's pins (limited fluxes, quadratics, a Fourier
eigenmode); sampled cells of the benchmark's full-size grid.
"""
import numpy as np
import pytest

import oracle
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I
from tests.gpu_util import normwise, to_dev
from tests.test_gpu_chain import _block_wrap, _sample_points

pytestmark = pytest.mark.gpu

C = 0.05


def run_cosmo(u, schedule, dtype=np.float64, bc=H.HFAV_BC_PERIODIC, c=C, ndim=3):
    import torch
    td = torch.float64 if dtype == np.float64 else torch.float32
    ut = to_dev(u, td)
    op = torch.full(ut.shape, float("nan"), dtype=td, device=ut.device)
    P = H.Plan(H.cosmo_dag(c, ndim=ndim), [H.Grid.of(ut, 2)], H.HFAV_F64 if dtype == np.float64 else H.HFAV_F32,
               bc, schedule)
    P.run([ut], [op])
    torch.cuda.synchronize()
    return op[2:-2, 2:-2, 2:-2].double().cpu().numpy() if ndim == 3 else op[2:-2, 2:-2].double().cpu().numpy()


VARIANTS = [f"{f}:{t}" for f in ("full:reg", "unfused:hbm") for t in ("32x4", "64x4", "128x2", "32x8")]


@pytest.mark.parametrize("schedule", VARIANTS)
def test_cosmo_all_schedules_f64(schedule):
    u = I.cosmo_input(64, 48, 5, seed=7)
    ref = oracle.cosmo(u, C)[3]
    assert normwise(run_cosmo(u, schedule), ref) <= 1e-12


@pytest.mark.parametrize("shape", [(13, 7, 2), (37, 29, 3), (130, 67, 2), (300, 5, 1)])
@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:128x2", "unfused:hbm:32x4"])
def test_cosmo_ragged(shape, schedule):
    nx, ny, nz = shape
    u = I.cosmo_input(nx, ny, nz, seed=8)
    ref = oracle.cosmo(u, C)[3]
    assert normwise(run_cosmo(u, schedule), ref) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:32x8", "unfused:hbm:64x4"])
def test_cosmo_f32(schedule):
    u = I.cosmo_input(200, 90, 3, seed=9)
    ref = oracle.cosmo(u.astype(np.float32).astype(np.float64), C)[3]
    assert normwise(run_cosmo(u, schedule, np.float32), ref) <= 2e-5


def test_cosmo_2d_dag():
    """The same DAG in 2D (no k axis) runs the same kernels."""
    u3 = I.cosmo_input(96, 40, 1, seed=10)
    ref = oracle.cosmo(u3, C)[3][0]
    got = run_cosmo(u3[2], "full:reg:32x4", ndim=2)
    assert normwise(got, ref) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:128x2", "unfused:hbm:32x4"])
def test_cosmo_halo_given_closed_forms(schedule):
    """u = i^4: every flux is limited, out = u exactly; quadratics: out = u exactly."""
    nx, ny, nz = 40, 12, 2
    k, j, i = np.meshgrid(np.arange(-2, nz + 2), np.arange(-2, ny + 2), np.arange(-2, nx + 2), indexing="ij")
    for u in ((i.astype(np.float64)) ** 4, 3.0 * i * i - 2.0 * j * j + 5.0 * i * j + i - 7.0 * j + 11.0 + k):
        got = run_cosmo(u, schedule, bc=H.HFAV_BC_HALO_GIVEN)
        assert np.array_equal(got, u[2:-2, 2:-2, 2:-2])


def test_cosmo_fourier_eigenmode():
    nx, ny, nz = 128, 64, 2
    w, v = 2 * np.pi * 5 / nx, 2 * np.pi * 3 / ny
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    core = np.broadcast_to(np.sin(w * i) * np.sin(v * j), (nz, ny, nx))
    u = np.full((nz + 4, ny + 4, nx + 4), np.nan)
    u[2:-2, 2:-2, 2:-2] = core
    lam = 4 * np.sin(w / 2) ** 2 + 4 * np.sin(v / 2) ** 2
    got = run_cosmo(u, "full:reg:32x4")
    assert np.max(np.abs(got - (1 - C * lam * lam) * core)) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:128x2"])
def test_cosmo_1024_f32_full_size_sampled(schedule):
    """The benchmark's 1024 x 1024 x 64 FP32 grid at full size: sampled cells
    (strip and chunk borders among them) against the oracle run on each cell's
    periodic 5 x 5 neighbourhood in its plane; 2e-5 of max |out|."""
    import torch
    nx = ny = 1024
    nz = 64
    u = I.cosmo_input(nx, ny, nz, seed=7, dtype=np.float32)
    ut = to_dev(u)
    op = torch.full_like(ut, float("nan"))
    P = H.Plan(H.cosmo_dag(C), [H.Grid.of(ut, 2)], H.HFAV_F32, H.HFAV_BC_PERIODIC, schedule)
    P.run([ut], [op])
    torch.cuda.synchronize()
    pts = _sample_points(ny, 2, 300, seed=13)
    ks = np.random.default_rng(14).integers(0, nz, size=len(pts))
    kk = torch.from_numpy(ks + 2).cuda()
    jj, ii = (torch.from_numpy(pts[:, x] + 2).cuda() for x in range(2))
    got = op[kk, jj, ii].double().cpu().numpy()
    ref = []
    for kq, p in zip(ks, pts):
        blk = _block_wrap(u[kq + 2, 2:-2, 2:-2], p, 2).astype(np.float64)[None]
        ref.append(oracle.cosmo(np.pad(blk, 2), C)[3][0, 2, 2])
    assert np.all(np.isfinite(got))
    assert normwise(got, np.array(ref)) <= 2e-5
