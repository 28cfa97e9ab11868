"""GPU parity of the Godunov pipelines against the oracle, through the C ABI.

FP64 bar: <= 1e-12 normwise per field after 10 steps (every schedule, grids
that span several tiles with ragged tails, and the 1024^2 workload).  FP32
bulk (Newton + CFL in FP64): <= 1e-4 normwise per field after 10 steps.
Also: conservation to 1e-12 on the GPU, the uniform state as a fixed point,
dt history equal to the oracle's, a CUDA-graph replay bitwise equal to a
plain run, and batches of uneven grids equal to per-grid oracle runs.
Ordering: a plain run on other arrays between two replays of a captured graph
leaves the graph's tables intact, and two runs queued back to back on a
non-blocking stream (the second reading the first one's goals) equal the
oracle's 20 steps.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I
from tests.gpu_util import empty_like_state, normwise, state_tensors

pytestmark = pytest.mark.gpu


def gpu_godunov(Us, nsteps, schedule, dtype=H.HFAV_F64, graph=False, plan=None):
    """Us: list of (4, ny, nx) states (one per grid).  Returns (results, plan)."""
    import torch
    td = torch.float64 if dtype == H.HFAV_F64 else torch.float32
    ins = [state_tensors(U, td) for U in Us]
    outs = [empty_like_state(t) for t in ins]
    grids = [H.Grid.of(t[0], 0) for t in ins]
    P = plan or H.Plan(H.godunov_dag(), grids, dtype, H.HFAV_BC_PERIODIC, schedule)
    P.run(ins, outs, nsteps, graph=graph)
    st = P.status()
    res = [np.stack([o.double().cpu().numpy() for o in out]) for out in outs]
    return res, P, st


def check_fields(got, ref, tol):
    errs = [normwise(got[f], ref[f]) for f in range(4)]
    assert max(errs) <= tol, errs
    return errs


SCHEDULES = ["sweep:reg:32x4", "sweep:reg:128x2", "sweep:smem:64x4", "sweep:hbm:32x8", "full:reg:32x4",
             "full:reg:64x4", "full:smem:128x2", "full:hbm:32x8", "unfused"]


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("shape", [(96, 64), (100, 37)])
def test_f64_schedules_match_oracle(schedule, shape):
    nx, ny = shape
    U = I.sod_state(nx, ny, seed=1)
    ref, dts, st = oracle.godunov(U, 10)
    assert st.floor_hits == 0
    (got,), P, s = gpu_godunov([U], 10, schedule)
    check_fields(got, ref, 1e-12)
    assert s["newton_nonconverged"] == 0 and s["nonphysical"] == 0
    assert np.allclose(s["dt"][:10], dts, rtol=1e-13)


def test_f64_small_odd_grid():
    U = I.sod_state(13, 7, seed=2)
    ref, _, _ = oracle.godunov(U, 10)
    for sch in ("sweep:reg:32x4", "sweep:smem:32x4", "full:reg:32x4", "unfused"):
        (got,), _, _ = gpu_godunov([U], 10, sch)
        check_fields(got, ref, 1e-12)


def test_f64_1024_workload():
    U = I.sod_state(1024, 1024, seed=1)
    ref, dts, st = oracle.godunov(U, 10)
    (got,), P, s = gpu_godunov([U], 10, "sweep:reg:32x4")
    check_fields(got, ref, 1e-12)
    assert np.allclose(s["dt"][:10], dts, rtol=1e-13)


@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "sweep:reg:64x4", "sweep:smem:32x8", "unfused"])
def test_f64_2048_two_steps(schedule):
    U = I.sod_state(2048, 2048, seed=1)
    ref, dts, _ = oracle.godunov(U, 2)
    (got,), _, s = gpu_godunov([U], 2, schedule)
    check_fields(got, ref, 1e-12)
    assert np.allclose(s["dt"][:2], dts, rtol=1e-13)


@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "sweep:smem:64x4", "full:reg:32x4", "unfused"])
def test_f32_bulk_matches_f64_oracle(schedule):
    U = I.sod_state(128, 96, seed=5)
    ref, _, _ = oracle.godunov(U, 10)
    (got,), _, s = gpu_godunov([U], 10, schedule, dtype=H.HFAV_F32)
    errs = check_fields(got, ref, 1e-4)
    assert s["newton_nonconverged"] == 0


def test_conservation_f64_gpu():
    U = I.sod_state(128, 64, seed=7)
    (got,), _, _ = gpu_godunov([U], 10, "sweep:reg:32x4")
    for f in (0, 3):
        t0 = math.fsum(U[f].ravel().tolist()); t1 = math.fsum(got[f].ravel().tolist())
        assert abs(t1 - t0) <= 1e-12 * abs(t0)
    for f in (1, 2):
        sc = math.fsum(np.abs(U[f]).ravel().tolist())
        assert abs(math.fsum(got[f].ravel().tolist()) - math.fsum(U[f].ravel().tolist())) <= 1e-12 * sc


def test_uniform_fixed_point_gpu():
    U = np.empty((4, 40, 64))
    rho, u, v, p = 0.9, 0.3, -0.2, 0.7
    U[0] = rho; U[1] = rho * u; U[2] = rho * v; U[3] = p / 0.4 + 0.5 * rho * (u * u + v * v)
    for sch in ("sweep:reg:32x4", "full:reg:32x4", "unfused"):
        (got,), _, _ = gpu_godunov([U], 5, sch)
        assert np.array_equal(got, U)


def test_graph_replay_bitwise():
    U = I.sod_state(96, 64, seed=3)
    (a,), P, _ = gpu_godunov([U], 10, "sweep:reg:32x4")
    (b,), _, _ = gpu_godunov([U], 10, "sweep:reg:32x4", graph=True)
    (c,), _, _ = gpu_godunov([U], 10, "sweep:reg:32x4", graph=True)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def _host_state(ts):
    return np.stack([t.double().cpu().numpy() for t in ts])


@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "sweep:smem:64x4", "full:reg:32x4", "unfused"])
def test_plain_run_between_graph_replays(schedule):
    import torch
    UA = I.sod_state(96, 64, seed=4)
    UB = I.sod_state(96, 64, seed=5)
    refA = oracle.godunov(UA, 6)[0]
    refB = oracle.godunov(UB, 6)[0]
    inA = state_tensors(UA, torch.float64); outA = empty_like_state(inA)
    inB = state_tensors(UB, torch.float64); outB = empty_like_state(inB)
    P = H.Plan(H.godunov_dag(), [H.Grid.of(inA[0], 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC, schedule)
    P.run(inA, outA, 6, graph=True)
    torch.cuda.synchronize()
    check_fields(_host_state(outA), refA, 1e-12)
    for t in outA:
        t.fill_(float("nan"))
    P.run(inB, outB, 6)                 # rewrites the plain run's tables
    P.run(inA, outA, 6, graph=True)     # replays the graph captured for A
    torch.cuda.synchronize()
    check_fields(_host_state(outA), refA, 1e-12)
    check_fields(_host_state(outB), refB, 1e-12)


@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "sweep:hbm:32x4", "full:reg:32x4"])
def test_back_to_back_runs_on_a_side_stream(schedule):
    import torch
    U = I.sod_state(512, 256, seed=6)
    ref = oracle.godunov(U, 20)[0]
    side = torch.cuda.Stream()
    A = state_tensors(U, torch.float64)
    B = empty_like_state(A)
    P = H.Plan(H.godunov_dag(), [H.Grid.of(A[0], 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC, schedule)
    W = empty_like_state(A)
    P.run(A, W, 10, stream=side)        # allocates the plan's scratch (synchronising)
    side.synchronize()
    with torch.cuda.stream(side):
        P.run(A, B, 10, stream=side)    # A -> B
        P.run(B, A, 10, stream=side)    # B -> A, queued before the first run has finished
    side.synchronize()
    check_fields(_host_state(A), ref, 1e-12)


@pytest.mark.parametrize("dtype,tol", [(H.HFAV_F64, 1e-12), (H.HFAV_F32, 1e-4)])
@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "sweep:smem:64x4", "full:reg:32x4"])
def test_batch_of_uneven_grids(dtype, tol, schedule):
    sides = [(64, 40), (96, 96), (50, 30), (128, 33), (32, 160)]
    Us = [I.sod_state(nx, ny, seed=3, grid=g) for g, (nx, ny) in enumerate(sides)]
    got, P, s = gpu_godunov(Us, 10, schedule, dtype=dtype)
    for g, U in enumerate(Us):
        ref, _, _ = oracle.godunov(U, 10)
        check_fields(got[g], ref, tol)


def _golden4096():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "godunov4096_seed1_10steps.txt")
    dt = totals = absmax = None
    pts, vals = [], []
    for ln in open(path):
        if ln.startswith("#"):
            continue
        f = ln.split()
        if f[0] == "dt":
            dt = np.array([float(x) for x in f[1:]])
        elif f[0] == "totals":
            totals = np.array([float(x) for x in f[1:]])
        elif f[0] == "absmax":
            absmax = np.array([float(x) for x in f[1:]])
        else:
            pts.append((int(f[0]), int(f[1])))
            vals.append([float(x) for x in f[2:]])
    return dt, totals, absmax, np.array(pts), np.array(vals)


@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "sweep:hbm:32x4"])
def test_f32_bulk_4096_full_size_sampled(schedule):
    """The 4096^2 FP32-bulk workload at full size: sampled cells against the
    stored FP64 oracle result (tests/golden/make_godunov4096.py), 1e-4
    normwise per field; dt history and conserved totals."""
    import torch
    dt_ref, totals, absmax, pts, vals = _golden4096()
    U = I.sod_state(4096, 4096, seed=1)
    ins = state_tensors(U, torch.float32)
    outs = empty_like_state(ins)
    P = H.Plan(H.godunov_dag(), [H.Grid.of(ins[0], 0)], H.HFAV_F32, H.HFAV_BC_PERIODIC, schedule)
    P.run(ins, outs, 10)
    st = P.status()
    assert st["newton_nonconverged"] == 0 and st["nonphysical"] == 0
    assert np.allclose(st["dt"][:10], dt_ref, rtol=1e-5)
    jj = torch.from_numpy(pts[:, 0]).cuda(); ii = torch.from_numpy(pts[:, 1]).cuda()
    errs = []
    for f in range(4):
        got = outs[f][jj, ii].double().cpu().numpy()
        errs.append(np.max(np.abs(got - vals[:, f])) / absmax[f])
    print(f"\n4096^2 FP32 bulk {schedule}, 10 steps, sampled per-field error vs FP64 oracle "
          f"(rho, rho u, rho v, E): " + " ".join(f"{e:.2e}" for e in errs))
    assert max(errs) <= 1e-4, errs
    for f in (0, 3):
        tot = outs[f].double().sum().item()
        assert abs(tot - totals[f]) <= 1e-5 * abs(totals[f])


def _oracle_grid(args):
    nx, ny, seed, g, steps = args
    U = I.sod_state(nx, ny, seed=seed, grid=g)
    return oracle.godunov(U, steps)[0]


def test_batch64_full_size_eight_largest_grids_match_oracle():
    """The 64-grid FP32 batch at full size, 10 steps in one captured graph:
    the eight largest grids (1388 to 1928 rows, 2.3 to 3.5 M cells each)
    against the FP64 oracle, 1e-4 normwise per field.  The oracle runs in
    spawned processes, one per grid."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    sides = I.batch_sides(64, seed=3)
    Us = [I.sod_state(nx, ny, seed=3, grid=g) for g, (nx, ny) in enumerate(sides)]
    ins = [state_tensors(U, torch.float32) for U in Us]
    outs = [empty_like_state(t) for t in ins]
    P = H.Plan(H.godunov_dag(), [H.Grid.of(t[0], 0) for t in ins], H.HFAV_F32, H.HFAV_BC_PERIODIC,
               "sweep:reg:32x4")
    P.run(ins, outs, 10, graph=True)
    st = P.status()
    assert st["newton_nonconverged"] == 0 and st["nonphysical"] == 0
    big = sorted(range(64), key=lambda k: -sides[k][0] * sides[k][1])[:8]
    with cf.ProcessPoolExecutor(max_workers=8, mp_context=mp.get_context("spawn")) as ex:
        refs = list(ex.map(_oracle_grid, [(sides[g][0], sides[g][1], 3, g, 10) for g in big]))
    for g, ref in zip(big, refs):
        got = np.stack([o.double().cpu().numpy() for o in outs[g]])
        check_fields(got, ref, 1e-4)


def test_batch64_full_size_one_grid_and_conservation():
    """The 64-grid FP32 batch at full size, 100 steps through a captured graph:
    the smallest grid against the oracle (1e-4 normwise per field) and mass /
    energy conservation of every grid (FP32 bulk: 1e-5 relative)."""
    import math
    import torch
    sides = I.batch_sides(64, seed=3)
    Us = [I.sod_state(nx, ny, seed=3, grid=g) for g, (nx, ny) in enumerate(sides)]
    ins = [state_tensors(U, torch.float32) for U in Us]
    outs = [empty_like_state(t) for t in ins]
    P = H.Plan(H.godunov_dag(), [H.Grid.of(t[0], 0) for t in ins], H.HFAV_F32, H.HFAV_BC_PERIODIC,
               "sweep:reg:32x4")
    P.run(ins, outs, 100, graph=True)
    st = P.status()
    assert st["newton_nonconverged"] == 0 and st["nonphysical"] == 0
    g = min(range(64), key=lambda k: sides[k][0] * sides[k][1])
    ref, _, _ = oracle.godunov(Us[g], 100)
    got = np.stack([o.double().cpu().numpy() for o in outs[g]])
    errs = check_fields(got, ref, 1e-4)
    print(f"\nbatch of 64, FP32 bulk, 100 steps: grid {sides[g]} per-field error vs FP64 oracle "
          f"(rho, rho u, rho v, E): " + " ".join(f"{e:.2e}" for e in errs))
    for k in range(64):
        for f in (0, 3):
            t0 = math.fsum(Us[k][f].astype(np.float32).astype(np.float64).ravel().tolist())
            t1 = outs[k][f].double().sum().item()
            assert abs(t1 - t0) <= 1e-5 * abs(t0), (k, f)
