"""Status and failure paths of a run on the GPU, with the oracle as reference.

- A Godunov step at CFL 5 on an 8 x 8 grid overshoots (the oracle's own step
  gives rho < 0 and p < 0): hfav_status returns HFAV_ENONPHYSICAL with the
  count of bad cells; every loop in the kernels is bounded, so the run ends,
  and the same plan then runs a physical state correctly.
- Checkpoint / resume: 5 steps, the state copied to the host and back, then 5
  more steps equal 10 steps in one run bit for bit, and the oracle's 10 steps
  to 1e-12.
- The two-shock Newton iteration converges within its cap of 10 on every
  state tried (random states over 16 decades of density and 19 of pressure,
  collisions up to Mach 1e8; see the oracle pins), so physical data do not
  reach the cap; with the cap set to one iteration through the RIEMANN
  rule's parameter,
  hfav_status returns HFAV_WARN_NEWTON with the count of faces, and the
  default cap reports none.
- An injected allocation failure (hfav_inject_alloc_failure) makes the run
  that meets it return HFAV_ENOMEM, on the plan's first allocation and on a
  later one; the same plan then runs and matches the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I
from tests.gpu_util import empty_like_state, normwise, state_tensors

pytestmark = pytest.mark.gpu

ENOMEM, ENONPHYSICAL, WARN_NEWTON = -7, -10, 1


def _host(ts):
    return np.stack([t.double().cpu().numpy() for t in ts])


def _errs(got, ref):
    return [normwise(got[f], ref[f]) for f in range(4)]


@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "sweep:smem:32x4", "full:reg:32x4", "unfused"])
def test_cfl5_reports_nonphysical(schedule):
    import torch
    U = I.sod_state(8, 8, seed=1)
    W, _, _ = oracle.godunov(U, 1, cfl=5.0)
    rho = W[0]
    p = 0.4 * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / rho)
    assert rho.min() < 0 or p.min() < 0          # the scheme itself overshoots
    ins = state_tensors(U, torch.float64)
    outs = empty_like_state(ins)
    P = H.Plan(H.godunov_dag(cfl=5.0), [H.Grid.of(ins[0], 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC, schedule)
    P.run(ins, outs, 2)
    with pytest.raises(H.HfavError) as e:
        P.status()
    assert e.value.code == ENONPHYSICAL
    # the context is still usable: a physical run on a fresh plan is exact
    V = I.sod_state(40, 24, seed=2)
    ref = oracle.godunov(V, 4)[0]
    vin = state_tensors(V, torch.float64)
    vout = empty_like_state(vin)
    Q = H.Plan(H.godunov_dag(), [H.Grid.of(vin[0], 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC, schedule)
    Q.run(vin, vout, 4)
    s = Q.status()
    assert s["nonphysical"] == 0 and s["newton_nonconverged"] == 0
    assert max(_errs(_host(vout), ref)) <= 1e-12


@pytest.mark.parametrize("schedule,dtype", [("sweep:reg:32x4", H.HFAV_F64), ("full:smem:64x4", H.HFAV_F64),
                                            ("sweep:reg:32x4", H.HFAV_F32)])
def test_resume_five_plus_five_is_ten(schedule, dtype):
    import torch
    td = torch.float64 if dtype == H.HFAV_F64 else torch.float32
    U = I.sod_state(200, 120, seed=8)
    ins = state_tensors(U, td)
    P = H.Plan(H.godunov_dag(), [H.Grid.of(ins[0], 0)], dtype, H.HFAV_BC_PERIODIC, schedule)
    ten = empty_like_state(ins)
    P.run(ins, ten, 10)
    half = empty_like_state(ins)
    P.run(ins, half, 5)
    torch.cuda.synchronize()
    saved = [t.cpu().clone() for t in half]                 # the checkpoint
    resumed_in = [t.cuda() for t in saved]
    resumed = empty_like_state(ins)
    P.run(resumed_in, resumed, 5)
    torch.cuda.synchronize()
    for a, b in zip(ten, resumed):
        assert torch.equal(a, b)
    ref = oracle.godunov(U, 10)[0]
    assert max(_errs(_host(resumed), ref)) <= (1e-12 if dtype == H.HFAV_F64 else 1e-4)


@pytest.mark.parametrize("after", [0, 1, 3])
def test_injected_allocation_failure(after):
    import torch
    U = I.sod_state(64, 40, seed=9)
    ref = oracle.godunov(U, 3)[0]
    ins = state_tensors(U, torch.float64)
    outs = empty_like_state(ins)
    P = H.Plan(H.godunov_dag(), [H.Grid.of(ins[0], 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC, "sweep:hbm:32x4")
    L = H.load()
    L.hfav_inject_alloc_failure(after)
    try:
        with pytest.raises(H.HfavError) as e:
            P.run(ins, outs, 3)
        assert e.value.code == ENOMEM
    finally:
        L.hfav_inject_alloc_failure(-1)
    P.run(ins, outs, 3)
    s = P.status()
    assert s["nonphysical"] == 0
    assert max(_errs(_host(outs), ref)) <= 1e-12


@pytest.mark.parametrize("schedule", ["sweep:reg:32x4", "full:reg:32x4", "unfused"])
def test_newton_cap_reports_warning(schedule):
    import torch
    U = I.sod_state(64, 48, seed=3)
    ins = state_tensors(U, torch.float64)
    outs = empty_like_state(ins)
    P = H.Plan(H.godunov_dag(newton_max=1), [H.Grid.of(ins[0], 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC, schedule)
    P.run(ins, outs, 2)
    s = P.status()
    assert s["rc"] == WARN_NEWTON and s["newton_nonconverged"] > 0 and s["nonphysical"] == 0
    Q = H.Plan(H.godunov_dag(newton_max=10), [H.Grid.of(ins[0], 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC, schedule)
    Q.run(ins, outs, 2)
    s = Q.status()
    assert s["rc"] == 0 and s["newton_nonconverged"] == 0
    assert max(_errs(_host(outs), oracle.godunov(U, 2)[0])) <= 1e-12
