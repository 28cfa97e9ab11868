"""GPU parity of reductions, broadcasts and splits (Sec. 3.4) on generated
kernels, with the normalization example (Sec. 5.2), against oracle/expr.py.

- Normalization: fused (the split leaves two nests: 2 grid kernels and one
  finalization) and unfused (5 grid kernels and one finalization), FP64
  (<= 1e-12 normwise) and FP32 (<= 2e-5; the sum accumulates in FP64),
  ragged sizes, halo-given grids, bitwise repeatable runs, unit 2-norm.
- REDUCE_MAX broadcast back exactly; a goal that a later nest also reads.
- Seeded random DAGs with two reductions (sum, max), scalar rules and
  broadcast consumers, fused and unfused.
- The 16384^2 FP32 workload at full size: the output's 2-norm is 1 and
  sampled cells times the norm give the second difference of the input.
"""
import numpy as np
import pytest

from oracle import expr as E
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I
from tests import expr_dags as X
from tests.gpu_util import normwise, to_dev
from tests.test_gpu_codegen import run_plan

pytestmark = pytest.mark.gpu

SCHEDULES = ["full:smem:32x4", "full:smem:128x2", "unfused:hbm:32x4"]


def _norm_case(nx, ny, seed, h=1, fill=np.nan):
    u = I.chain2d_input(nx, seed=seed, ny=ny, halo=h, fill_halo=fill)
    return u, u[h:-h, h:-h]


@pytest.mark.parametrize("schedule", SCHEDULES + ["full:smem:64x4", "full:smem:32x8"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_normalization(schedule, dtype):
    u, core = _norm_case(200, 90, 1)
    (got,), P = run_plan(H.normalization_dag(), [u.astype(dtype)], 1, schedule, dtype)
    ref = E.evaluate(E.normalization_rules(), {"u": core.astype(dtype).astype(np.float64)})["out"]
    assert normwise(got, ref) <= (1e-12 if dtype == np.float64 else 2e-5)
    assert abs(np.sum(got * got) - 1) <= (1e-12 if dtype == np.float64 else 1e-5)
    assert P.status()["last_launches"] == (3 if schedule.startswith("full") else 6)


@pytest.mark.parametrize("shape", [(3, 2), (37, 29), (511, 7), (1021, 300)])
@pytest.mark.parametrize("schedule", ["full:smem:32x4", "unfused:hbm:32x4"])
def test_normalization_ragged(shape, schedule):
    u, core = _norm_case(*shape, seed=2)
    (got,), _ = run_plan(H.normalization_dag(), [u], 1, schedule)
    ref = E.evaluate(E.normalization_rules(), {"u": core})["out"]
    assert normwise(got, ref) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:smem:32x4", "unfused:hbm:64x4"])
def test_normalization_halo_given(schedule):
    rng = np.random.default_rng(4)
    u = rng.uniform(0, 1, (52, 77))          # the halo (width 1) holds values of its own
    (got,), _ = run_plan(H.normalization_dag(), [u], 1, schedule, bc=H.HFAV_BC_HALO_GIVEN)
    ref = E.evaluate_padded(E.normalization_rules(), {"u": u}, 1, ["out"])["out"]
    assert normwise(got, ref) <= 1e-12


def test_normalization_bitwise_repeatable():
    """The partials are combined in a fixed order: repeated runs agree bit for bit."""
    import torch
    u, _ = _norm_case(1000, 700, 5)
    ut = to_dev(u, torch.float32)
    outs = []
    P = H.Plan(H.normalization_dag(), [H.Grid.of(ut, 1)], H.HFAV_F32, H.HFAV_BC_PERIODIC, "full:smem:32x4")
    for _ in range(3):
        o = torch.full_like(ut, float("nan"))
        P.run([ut], [o])
        outs.append(o)
    torch.cuda.synchronize()
    assert all(torch.equal(outs[0][1:-1, 1:-1], o[1:-1, 1:-1]) for o in outs[1:])


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_max_broadcast_back_exactly(schedule):
    D = H.DagSpec(2)
    D.field("m", rank=0)
    D.rule("REDUCE_MAX", [("u", (1, -1))], ["m"])
    D.rule("EXPR", ["u", "m"], ["o"], expr="in0 - in1")
    D.axiom("u"); D.goal("o")
    rng = np.random.default_rng(6)
    core = rng.normal(size=(45, 70))
    u = np.full((47, 72), np.nan)
    u[1:-1, 1:-1] = core
    (got,), _ = run_plan(D, [u], 1, schedule)
    assert np.array_equal(got, core - core.max())


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_goal_read_after_the_split(schedule):
    """diff is both a goal and the input of the nest after the split."""
    D = H.normalization_dag()
    D.goal("diff")
    u, core = _norm_case(130, 40, 7)
    got, _ = run_plan(D, [u], 1, schedule, n_goals=2)
    ref = E.evaluate(E.normalization_rules(), {"u": core})
    assert normwise(got[0], ref["out"]) <= 1e-12
    assert np.array_equal(got[1], ref["diff"])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_random_reduce_dags(seed, schedule):
    rules, axioms, goals = X.random_reduce_dag(seed)
    D = X.to_spec_reduce(rules, axioms, goals)
    P0 = H.analyze(D)
    h = max(max(P0.field(a)["halo_lo"] + P0.field(a)["halo_hi"]) for a in axioms)
    shape = (53, 88)
    core = X.axiom_values(axioms, shape, seed + 3)
    padded = []
    for a in axioms:
        arr = np.full(tuple(n + 2 * h for n in shape), np.nan)
        arr[h:-h, h:-h] = core[a]
        padded.append(arr)
    got, _ = run_plan(D, padded, h, schedule, n_goals=len(goals))
    ref = E.evaluate(X.to_oracle_reduce(rules), core)
    for g, v in zip(goals, got):
        assert normwise(v, ref[g]) <= 1e-12, g


@pytest.mark.parametrize("schedule", ["full:smem:32x4", "full:smem:32x8"])
def test_normalization_16384_f32_full_size(schedule):
    """The bench's 16384^2 FP32 grid: sum of out^2 is 1 (to FP32 rounding of
    each term), and at sampled cells out * ||diff|| equals the input's second
    difference along i (the norm from the FP64 input, in row blocks)."""
    import torch
    n = 16384
    u = I.chain2d_input(n, seed=0, halo=1).astype(np.float32)
    ut = to_dev(u)
    op = torch.full_like(ut, float("nan"))
    P = H.Plan(H.normalization_dag(), [H.Grid.of(ut, 1)], H.HFAV_F32, H.HFAV_BC_PERIODIC, schedule)
    P.run([ut], [op])
    torch.cuda.synchronize()
    core = u[1:-1, 1:-1].astype(np.float64)
    ss = 0.0
    for j in range(0, n, 1024):
        blk = core[j:j + 1024]
        d = np.roll(blk, -1, axis=1) - 2 * blk + np.roll(blk, 1, axis=1)
        ss += float(np.sum(d * d))
    norm = np.sqrt(ss)
    out = op[1:-1, 1:-1]
    assert abs(float(out.double().pow(2).sum()) - 1) <= 1e-4
    rng = np.random.default_rng(9)
    pts = np.vstack([rng.integers(0, n, size=(400, 2)), [[0, 0], [n - 1, n - 1], [0, n - 1], [n - 1, 0]]])
    jj, ii = (torch.from_numpy(pts[:, x]).cuda() for x in range(2))
    got = out[jj, ii].double().cpu().numpy() * norm
    ref = np.array([core[j, (i + 1) % n] - 2 * core[j, i] + core[j, (i - 1) % n] for j, i in pts])
    assert normwise(got, ref) <= 2e-5
