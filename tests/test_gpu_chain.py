"""GPU parity of the stencil chains against the oracle, through the C ABI.

FP64 bar: <= 1e-12 normwise; FP32 bar: <= 2e-5 normwise (single rounding of
a handful of ops on O(1) values, derived from the arithmetic: ~20 FP32 ops
of relative error 6e-8 each).  Every schedule (fusion x placement x tile) is
checked at 256^2, at sizes that leave a ragged tail, and in the halo-given
mode against the exact closed form of quadratics.
"""
import numpy as np
import pytest

import oracle
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I
from tests.gpu_util import normwise, to_dev

pytestmark = pytest.mark.gpu


def run_chain2d(u, schedule, dtype=np.float64, bc=H.HFAV_BC_PERIODIC):
    import torch
    td = torch.float64 if dtype == np.float64 else torch.float32
    ny, nx = u.shape[0] - 4, u.shape[1] - 4
    ut = to_dev(u, td)
    P = H.Plan(H.chain2d_dag(), [H.Grid.of(ut, 2)], H.HFAV_F64 if dtype == np.float64 else H.HFAV_F32, bc,
               schedule)
    # the goal array shares the axiom's layout (one grid per plan)
    op = torch.full((ny + 4, nx + 4), float("nan"), dtype=td, device=ut.device)
    P.run([ut], [op])
    torch.cuda.synchronize()
    return op[2:-2, 2:-2].double().cpu().numpy(), P


VARIANTS = H.Plan(H.chain2d_dag(), [H.Grid.make((256, 256), (1, 260), 2)], 0, 0).variants()


@pytest.mark.parametrize("schedule", VARIANTS)
def test_chain2d_256_all_schedules_f64(schedule):
    u = I.chain2d_input(256, seed=0)
    _, _, ref = oracle.chain2d(u)
    got, _ = run_chain2d(u, schedule)
    assert normwise(got, ref) <= 1e-12


@pytest.mark.parametrize("shape", [(13, 7), (100, 37), (130, 67)])
@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:smem:64x4", "full:hbm:128x2", "sweep:reg:32x8",
                                      "unfused"])
def test_chain2d_ragged(shape, schedule):
    nx, ny = shape
    u = I.chain2d_input(nx, seed=3, ny=ny)
    _, _, ref = oracle.chain2d(u)
    got, _ = run_chain2d(u, schedule)
    assert normwise(got, ref) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:smem:32x8", "sweep:hbm:64x4", "unfused"])
def test_chain2d_halo_given_quadratic_exact(schedule):
    j, i = np.meshgrid(np.arange(-2, 70), np.arange(-2, 52), indexing="ij")
    u = 3.0 * i * i - 2.0 * j * j + 5.0 * i * j + i - 7.0 * j + 11.0
    got, _ = run_chain2d(u, schedule, bc=H.HFAV_BC_HALO_GIVEN)
    assert np.all(got == 0.0)


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:smem:128x2", "sweep:reg:64x4", "unfused"])
def test_chain2d_f32(schedule):
    u = I.chain2d_input(256, seed=1)
    _, _, ref = oracle.chain2d(u)
    got, _ = run_chain2d(u, schedule, dtype=np.float32)
    assert normwise(got, ref) <= 2e-5


def run_chain3d(u, schedule, dtype=np.float64):
    import torch
    td = torch.float64 if dtype == np.float64 else torch.float32
    ut = to_dev(u, td)
    op = torch.full(ut.shape, float("nan"), dtype=td, device=ut.device)
    P = H.Plan(H.chain3d_dag(), [H.Grid.of(ut, 3)], H.HFAV_F64 if dtype == np.float64 else H.HFAV_F32,
               H.HFAV_BC_PERIODIC, schedule)
    P.run([ut], [op])
    torch.cuda.synchronize()
    return op[3:-3, 3:-3, 3:-3].double().cpu().numpy()


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:64x4", "full:reg:128x2", "full:reg:32x8",
                                      "full:smem:64x4", "full:hbm:32x8", "full:smem:128x2", "sweep:reg:32x4",
                                      "unfused"])
def test_chain3d_f64(schedule):
    u = I.chain3d_input(40, seed=4)
    ref = oracle.chain3d(u)
    assert normwise(run_chain3d(u, schedule), ref) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:128x2", "full:reg:32x8", "full:smem:64x4",
                                      "sweep:reg:32x4", "unfused"])
def test_chain3d_f32_ragged(schedule):
    u = I.chain3d_input(37, seed=9)
    ref = oracle.chain3d(u)
    assert normwise(run_chain3d(u, schedule, np.float32), ref) <= 2e-5


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:32x8", "full:smem:64x4", "unfused"])
def test_chain3d_halo_given_quintic_exact(schedule):
    import torch
    n = 20
    k, j, i = np.meshgrid(*(np.arange(-3, n + 3),) * 3, indexing="ij")
    u = torch.from_numpy((i.astype(np.float64)) ** 5).cuda()
    op = torch.full_like(u, float("nan"))
    P = H.Plan(H.chain3d_dag(), [H.Grid.of(u, 3)], H.HFAV_F64, H.HFAV_BC_HALO_GIVEN, schedule)
    P.run([u], [op])
    torch.cuda.synchronize()
    assert np.all(op[3:-3, 3:-3, 3:-3].cpu().numpy() == 120.0 / 121.0)


TMA_TILES = [("full:reg:32x4", 32, 16), ("full:reg:64x4", 64, 16), ("full:reg:128x2", 128, 8),
             ("full:reg:32x8", 32, 16)]


def _tma_eligible(tx, tyo, es, nx, ny, h, periodic=True):
    """The fused 3D kernel's TMA copy needs a 16-byte aligned tile start
    i0 - 4 after the halo offset; on a periodic grid whole tiles, at least
    two per axis (each edge tile patches one band per axis)."""
    A = 16 // es
    if (h - 4) % A:
        return False
    return (nx % tx == 0 and nx >= 2 * tx and ny % tyo == 0 and ny >= 2 * tyo) if periodic else h >= 4


def _chain3d_halo(core, h, schedule, dtype, bc=H.HFAV_BC_PERIODIC, pad=None):
    """Run the 3D chain on `core` placed in an array with halo h (NaN, or
    `pad` when halo-given); returns (interior result, kernel names)."""
    import torch
    td = torch.float64 if dtype == np.float64 else torch.float32
    if pad is None:
        nz, ny, nx = core.shape
        arr = np.full((nz + 2 * h, ny + 2 * h, nx + 2 * h), np.nan)
        arr[h:h + nz, h:h + ny, h:h + nx] = core
    else:
        arr = pad
    ut = to_dev(arr, td)
    op = torch.full_like(ut, float("nan"))
    P = H.Plan(H.chain3d_dag(), [H.Grid.of(ut, h)], H.HFAV_F64 if dtype == np.float64 else H.HFAV_F32, bc, schedule)
    P.timing(True)
    P.run([ut], [op])
    names = set(P.kernel_times())
    torch.cuda.synchronize()
    crop = tuple(slice(h, op.shape[d] - h) for d in range(3))
    return op[crop].double().cpu().numpy(), names


@pytest.mark.parametrize("schedule,tx,tyo", TMA_TILES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,h", [((19, 64, 128), 0), ((9, 48, 256), 4), ((7, 32, 96), 8), ((5, 32, 64), 0),
                                     ((5, 21, 44), 0), ((6, 40, 72), 3)])
def test_chain3d_tma_periodic(schedule, tx, tyo, dtype, shape, h):
    """The fused 3D kernel with its u planes staged by the tensor memory
    accelerator (one tensor box per plane tile; on the periodic edges the
    wrapped cells patched from registers) against the oracle: interior, edge
    and corner tiles, halo offsets 0, 4, 8, short k extents; layouts it
    cannot use (halo 3, partial tiles, one tile per axis) fall back to
    per-element copies, which must give the same results."""
    rng = np.random.default_rng(sum(shape) + h)
    core = rng.normal(size=shape)
    ref = oracle.chain3d(np.pad(core, 3))
    got, names = _chain3d_halo(core, h, schedule, dtype)
    es = 8 if dtype == np.float64 else 4
    want = "chain3d_fused_tma" if _tma_eligible(tx, tyo, es, shape[2], shape[1], h) else "chain3d_fused"
    assert want in names, names
    assert normwise(got, ref) <= (1e-12 if dtype == np.float64 else 2e-5)


@pytest.mark.parametrize("schedule,tx,tyo", TMA_TILES)
def test_chain3d_tma_halo_given_quintic_exact(schedule, tx, tyo):
    """Halo-given grids with a halo of 4 read their halo through the tensor
    box: u = i^5 gives out = 120/121 exactly on every cell."""
    n, h = 20, 4
    k, j, i = np.meshgrid(*(np.arange(-h, n + h),) * 3, indexing="ij")
    u = (i.astype(np.float64)) ** 5
    got, names = _chain3d_halo(None, h, schedule, np.float64, H.HFAV_BC_HALO_GIVEN, pad=u)
    assert "chain3d_fused_tma" in names, names
    assert np.all(got == 120.0 / 121.0)


def _block_wrap(interior, centre, r):
    """The (2r+1)^d block of a periodic interior array around `centre`."""
    idx = [np.arange(c - r, c + r + 1) % n for c, n in zip(centre, interior.shape)]
    return interior[np.ix_(*idx)]


def _sample_points(n, dims, count, seed):
    """Random cells plus the domain's corners and cells on tile / chunk borders."""
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, n, size=(count, dims))
    fixed = [[0] * dims, [n - 1] * dims, [n // 2] * dims]
    for b in (31, 32, 55, 56, 63, 64, 127, 128, 255, 256):
        if b < n:
            fixed.append([b] * dims)
            fixed.append([(b + 7 * d) % n for d in range(dims)])
    return np.vstack([pts, np.array(fixed)])


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:32x8"])
def test_chain3d_512_f32_full_size_sampled(schedule):
    """The 512^3 FP32 3D chain at full size, in the fused schedules the bench's
    autotuner picks: sampled cells (tile and chunk borders among them) against
    the oracle run on each cell's periodic 7^3 neighbourhood, which fixes the
    cell's value exactly; the FP32 bar of 2e-5 of max |out|."""
    import torch
    n = 512
    u = I.chain3d_input(n, seed=4, dtype=np.float32)
    ut = to_dev(u)
    op = torch.full_like(ut, float("nan"))
    P = H.Plan(H.chain3d_dag(), [H.Grid.of(ut, 3)], H.HFAV_F32, H.HFAV_BC_PERIODIC, schedule)
    P.run([ut], [op])
    torch.cuda.synchronize()
    pts = _sample_points(n, 3, 300, seed=11)
    kk, jj, ii = (torch.from_numpy(pts[:, x] + 3).cuda() for x in range(3))
    got = op[kk, jj, ii].double().cpu().numpy()
    interior = u[3:-3, 3:-3, 3:-3]
    ref = np.array([oracle.chain3d(np.pad(_block_wrap(interior, p, 3).astype(np.float64), 3))[3, 3, 3]
                    for p in pts])
    assert np.all(np.isfinite(got))
    assert normwise(got, ref) <= 2e-5


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:32x8"])
def test_chain3d_512_f32_halo0_tma_sampled(schedule):
    """The bench's layout of the 512^3 FP32 workload: a periodic grid stored
    without halo, which the fused kernel stages through TMA; sampled cells
    against the oracle on their 7^3 neighbourhoods (2e-5 of max |out|)."""
    import torch
    n = 512
    u = I.chain3d_input(n, seed=4, dtype=np.float32, halo=0)
    ut = to_dev(u)
    op = torch.full_like(ut, float("nan"))
    P = H.Plan(H.chain3d_dag(), [H.Grid.of(ut, 0)], H.HFAV_F32, H.HFAV_BC_PERIODIC, schedule)
    P.timing(True)
    P.run([ut], [op])
    assert "chain3d_fused_tma" in P.kernel_times()
    torch.cuda.synchronize()
    pts = _sample_points(n, 3, 300, seed=13)
    kk, jj, ii = (torch.from_numpy(pts[:, x]).cuda() for x in range(3))
    got = op[kk, jj, ii].double().cpu().numpy()
    ref = np.array([oracle.chain3d(np.pad(_block_wrap(u, p, 3).astype(np.float64), 3))[3, 3, 3] for p in pts])
    assert np.all(np.isfinite(got))
    assert normwise(got, ref) <= 2e-5


@pytest.mark.parametrize("schedule", ["full:reg:32x4", "full:reg:128x2"])
def test_chain2d_16384_f32_full_size_sampled(schedule):
    """The 16384^2 FP32 2D chain (the large-grid point of the bench) at full
    size: sampled cells (strip and chunk borders among them) against the oracle
    run on each cell's periodic 5 x 5 neighbourhood; 2e-5 of max |out|."""
    import torch
    n = 16384
    u = I.chain2d_input(n, seed=0).astype(np.float32)
    ut = to_dev(u)
    op = torch.full_like(ut, float("nan"))
    P = H.Plan(H.chain2d_dag(), [H.Grid.of(ut, 2)], H.HFAV_F32, H.HFAV_BC_PERIODIC, schedule)
    P.run([ut], [op])
    torch.cuda.synchronize()
    pts = _sample_points(n, 2, 500, seed=12)
    jj, ii = (torch.from_numpy(pts[:, x] + 2).cuda() for x in range(2))
    got = op[jj, ii].double().cpu().numpy()
    interior = u[2:-2, 2:-2]
    ref = np.array([oracle.chain2d(np.pad(_block_wrap(interior, p, 2).astype(np.float64), 2))[2][2, 2] for p in pts])
    assert np.all(np.isfinite(got))
    assert normwise(got, ref) <= 2e-5
