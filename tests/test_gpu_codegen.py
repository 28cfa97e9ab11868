"""GPU parity of the generated kernels (DAGs with user rule bodies,
HFAV_OP_EXPR) against the oracle, through the C ABI.

- The 2D chain written as rule bodies against the chain's C oracle, every
  schedule, FP64 (<= 1e-12 normwise) and FP32 (<= 2e-5), ragged sizes, and at
  the bench's 16384^2 FP32 size on sampled cells.
- Seeded random DAGs (several axioms and goals, offsets in every direction,
  chains of up to 6 rules) against oracle/expr.py: fused and unfused, 2D and
  3D, periodic and halo-given, FP64 and FP32.
- Rule bodies mixed with builtin ops in one fused kernel; nested pointwise
  stages evaluated inside their readers; rings above the default 48 KB of
  shared memory; CUDA-graph replay; a body that does not compile fails the run
  cleanly.
FP32 bar: 2e-5 normwise -- a chain of up to 6 bodies of a few FP32 roundings
(relative 6e-8) each, on O(1) values whose bodies are Lipschitz with small
constants.
"""
import numpy as np
import pytest

import oracle
from oracle import expr as E
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I
from tests import expr_dags as X
from tests.gpu_util import normwise, to_dev
from tests.test_gpu_chain import _block_wrap, _sample_points

pytestmark = pytest.mark.gpu

SCHEDULES = [f"{f}:{t}" for f in ("full:smem", "full:reg", "unfused:hbm") for t in ("32x4", "64x4", "128x2", "32x8")]


def run_plan(spec, axioms, halo, schedule, dtype=np.float64, bc=H.HFAV_BC_PERIODIC, graph=False, n_goals=1):
    """Run a plan on halo-padded numpy axioms; returns the goals' interiors (FP64)."""
    import torch
    td = torch.float64 if dtype == np.float64 else torch.float32
    ts = [to_dev(a, td) for a in axioms]
    gs = [torch.full_like(ts[0], float("nan")) for _ in range(n_goals)]
    P = H.Plan(spec, [H.Grid.of(ts[0], halo)], H.HFAV_F64 if dtype == np.float64 else H.HFAV_F32, bc, schedule)
    P.run(ts, gs, graph=graph)
    torch.cuda.synchronize()
    crop = tuple(slice(halo, -halo) for _ in range(ts[0].dim()))
    return [g[crop].double().cpu().numpy() for g in gs], P


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_chain_as_rule_bodies_f64(schedule):
    u = I.chain2d_input(96, seed=0, ny=80)
    (got,), P = run_plan(H.chain2d_expr_dag(), [u], 2, schedule)
    assert P.dump()["pipeline"] == "codegen"
    assert normwise(got, oracle.chain2d(u)[2]) <= 1e-12


@pytest.mark.parametrize("shape", [(13, 7), (100, 37), (130, 67), (2, 2), (257, 3), (1000, 9)])
@pytest.mark.parametrize("schedule", ["full:smem:32x4", "full:smem:128x2", "full:reg:32x4", "full:reg:128x2",
                                      "unfused:hbm:32x4"])
def test_chain_as_rule_bodies_ragged(shape, schedule):
    nx, ny = shape
    u = I.chain2d_input(nx, seed=3, ny=ny)
    (got,), _ = run_plan(H.chain2d_expr_dag(), [u], 2, schedule)
    assert normwise(got, oracle.chain2d(u)[2]) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:smem:32x8", "full:reg:32x4", "unfused:hbm:32x4"])
def test_chain_as_rule_bodies_f32(schedule):
    u = I.chain2d_input(300, seed=4, ny=200)
    (got,), _ = run_plan(H.chain2d_expr_dag(), [u], 2, schedule, np.float32)
    ref = oracle.chain2d(u.astype(np.float32).astype(np.float64))[2]
    assert normwise(got, ref) <= 2e-5


def _random_case(ndim, seed, shape, n_rules=6, halo=None, fill=np.nan):
    rules, axioms, goals = X.random_dag(ndim, n_rules, seed)
    spec = X.to_spec(rules, axioms, goals, ndim, shuffle_seed=seed + 50)
    need = max(max(abs(v) for v in (P.field(a)["halo_lo"] + P.field(a)["halo_hi"])) for P in [H.analyze(spec)]
               for a in axioms)
    h = need if halo is None else halo
    core = X.axiom_values(axioms, shape, seed + 7)
    padded = []
    for a in axioms:
        arr = np.full(tuple(n + 2 * h for n in shape), fill)
        arr[tuple(slice(h, h + n) for n in shape)] = core[a]
        padded.append(arr)
    return rules, axioms, goals, spec, core, padded, h


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("schedule", ["full:smem:32x4", "full:smem:128x2", "full:smem:32x8", "unfused:hbm:32x4"])
def test_random_dags_2d_f64(seed, schedule):
    rules, axioms, goals, spec, core, padded, h = _random_case(2, seed, (45, 71))
    got, _ = run_plan(spec, padded, h, schedule, n_goals=len(goals))
    ref = E.evaluate(X.to_oracle(rules), core)
    for g, v in zip(goals, got):
        assert normwise(v, ref[g]) <= 1e-12, g


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("schedule", ["full:smem:64x4", "unfused:hbm:32x4"])
def test_random_dags_2d_f32(seed, schedule):
    rules, axioms, goals, spec, core, padded, h = _random_case(2, seed + 20, (130, 67))
    got, _ = run_plan(spec, [p.astype(np.float32) for p in padded], h, schedule, np.float32, n_goals=len(goals))
    ref = E.evaluate(X.to_oracle(rules), {a: core[a].astype(np.float32).astype(np.float64) for a in axioms})
    for g, v in zip(goals, got):
        assert normwise(v, ref[g]) <= 2e-5, g


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_random_dags_2d_warp_strips(seed, dtype):
    """Generated warp-strip kernels (full:reg) on the random DAGs they take
    (one fused part): against the oracle, and against the ring kernel to
    rounding (a stage's value stays in a register here, so the compiler may
    fuse its last product into a reader's sum: one rounding where the ring
    kernel, which stores the stage, has two)."""
    rules, axioms, goals, spec, core, padded, h = _random_case(2, seed + 80, (83, 57))
    import torch
    P = H.Plan(spec, [H.Grid.of(padded[0], h)])
    regs = [v for v in P.variants() if v.startswith("full:reg")]
    if not regs:
        pytest.skip("a DAG of several fused parts: warp strips do not apply")
    arrs = [p.astype(dtype) for p in padded]
    got, _ = run_plan(spec, arrs, h, "full:reg:32x4", dtype, n_goals=len(goals))
    ring, _ = run_plan(spec, arrs, h, "full:smem:32x4", dtype, n_goals=len(goals))
    ref = E.evaluate(X.to_oracle(rules), {a: core[a].astype(dtype).astype(np.float64) for a in axioms})
    for g, v, w in zip(goals, got, ring):
        assert normwise(v, ref[g]) <= (1e-12 if dtype == np.float64 else 2e-5), g
        assert normwise(v, w) <= (1e-13 if dtype == np.float64 else 1e-5), g


def test_warp_strips_take_most_random_dags():
    """Most random DAGs plan onto warp strips; the others (several fused
    parts, or row windows beyond the register budget) are refused with a
    reason."""
    taken = 0
    for seed in range(12):
        rules, axioms, goals = X.random_dag(2, 6, seed + 80)
        P = H.Plan(X.to_spec(rules, axioms, goals, 2), [H.Grid.of(np.zeros((60, 50)), 6)])
        if any(v.startswith("full:reg") for v in P.variants()):
            taken += 1
        else:
            with pytest.raises(H.HfavError) as e:
                P.schedule = "full:reg:32x4"
            assert "EUNSUPPORTED" in str(e.value) and ("one-part" in str(e.value) or "register" in str(e.value))
    assert taken >= 6


@pytest.mark.parametrize("seed", range(4))
def test_random_dags_3d_unfused(seed):
    rules, axioms, goals, spec, core, padded, h = _random_case(3, seed + 40, (9, 14, 23), n_rules=4)
    got, _ = run_plan(spec, padded, h, "unfused:hbm:32x4", n_goals=len(goals))
    ref = E.evaluate(X.to_oracle(rules), core)
    for g, v in zip(goals, got):
        assert normwise(v, ref[g]) <= 1e-12, g


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("schedule", ["full:smem:32x4", "full:reg:32x4", "unfused:hbm:64x4"])
def test_random_dags_halo_given(seed, schedule):
    """The caller's halo is read as given: random halo values, the oracle on the
    padded arrays cropped (exact while the halo covers the footprint)."""
    rules, axioms, goals = X.random_dag(2, 5, seed + 60)
    spec = X.to_spec(rules, axioms, goals, 2)
    P0 = H.analyze(spec)
    h = max(max(P0.field(a)["halo_lo"] + P0.field(a)["halo_hi"]) for a in axioms)
    shape = (33 + 2 * h, 50 + 2 * h)
    padded = X.axiom_values(axioms, shape, seed + 61)
    got, _ = run_plan(spec, [padded[a] for a in axioms], h, schedule, bc=H.HFAV_BC_HALO_GIVEN, n_goals=len(goals))
    ref = E.evaluate_padded(X.to_oracle(rules), padded, h, goals)
    for g, v in zip(goals, got):
        assert normwise(v, ref[g]) <= 1e-12, g


@pytest.mark.parametrize("schedule", ["full:smem:32x4", "full:smem:128x2", "full:reg:32x4", "unfused:hbm:32x4"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_nested_pointwise_stages(schedule, dtype):
    """Stages read only at offset 0 are evaluated inside their readers (two
    levels deep here); the goal goes straight from its rule to memory."""
    rules, axioms, goals = X.pointwise_dag()
    spec = X.to_spec(rules, axioms, goals, 2)
    shape, h = (67, 45), 3
    core = X.axiom_values(axioms, shape, 3)
    padded = []
    for a in axioms:
        arr = np.full(tuple(n + 2 * h for n in shape), np.nan)
        arr[h:-h, h:-h] = core[a]
        padded.append(arr.astype(dtype))
    (got,), _ = run_plan(spec, padded, h, schedule, dtype)
    ref = E.evaluate(X.to_oracle(rules), {a: core[a].astype(dtype).astype(np.float64) for a in axioms})["g"]
    assert normwise(got, ref) <= (1e-12 if dtype == np.float64 else 2e-5)


def test_rule_bodies_mixed_with_builtin_ops():
    D = H.DagSpec(2)
    D.rule("STENCIL_LINEAR", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))], ["L"],
           params=[1, 1, 1, 1, -4])
    D.rule("EXPR", [("L", (1, 0)), ("L", (-1, 0)), ("L", (0, 1)), ("L", (0, -1))], ["G"],
           expr="hypot(in0 - in1, in2 - in3) * (T)0.5")
    D.rule("SQUASH", ["G"], ["out"])
    D.axiom("u"); D.goal("out")
    u = I.chain2d_input(77, seed=9, ny=41)
    for sched in ("full:smem:32x4", "full:reg:32x4", "unfused:hbm:32x4"):
        (got,), _ = run_plan(D, [u], 2, sched)
        assert normwise(got, oracle.chain2d(u)[2]) <= 1e-12


@pytest.mark.parametrize("schedule", ["full:smem:32x8", "full:reg:32x8"])
def test_graph_replay_matches(schedule):
    rules, axioms, goals, spec, core, padded, h = _random_case(2, 3, (64, 40))
    a, _ = run_plan(spec, padded, h, schedule, n_goals=len(goals))
    b, _ = run_plan(spec, padded, h, schedule, graph=True, n_goals=len(goals))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_body_that_does_not_compile_fails_cleanly():
    import torch
    D = H.DagSpec(2)
    D.rule("EXPR", [("u", (0, 0))], ["o"], expr="in0 +* )")
    D.axiom("u"); D.goal("o")
    u = torch.zeros((12, 12), dtype=torch.float64, device="cuda")
    o = torch.zeros_like(u)
    P = H.Plan(D, [H.Grid.of(u, 1)], H.HFAV_F64, H.HFAV_BC_PERIODIC, "full:smem:32x4")
    with pytest.raises(H.HfavError) as e:
        P.run([u], [o])
    assert "does not compile" in str(e.value)
    # the context stays usable
    (got,), _ = run_plan(H.chain2d_expr_dag(), [I.chain2d_input(20, seed=1)], 2, "full:smem:32x4")
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("schedule", ["full:smem:32x8", "full:smem:128x2", "full:reg:32x4"])
def test_chain_as_rule_bodies_16384_f32_full_size_sampled(schedule):
    """The bench's 16384^2 FP32 grid: sampled cells (tile borders among them)
    against the chain's oracle on each cell's periodic 5 x 5 neighbourhood."""
    import torch
    n = 16384
    u = I.chain2d_input(n, seed=0).astype(np.float32)
    ut = to_dev(u)
    op = torch.full_like(ut, float("nan"))
    P = H.Plan(H.chain2d_expr_dag(), [H.Grid.of(ut, 2)], H.HFAV_F32, H.HFAV_BC_PERIODIC, schedule)
    P.run([ut], [op])
    torch.cuda.synchronize()
    pts = _sample_points(n, 2, 500, seed=12)
    jj, ii = (torch.from_numpy(pts[:, x] + 2).cuda() for x in range(2))
    got = op[jj, ii].double().cpu().numpy()
    interior = u[2:-2, 2:-2]
    ref = np.array([oracle.chain2d(np.pad(_block_wrap(interior, p, 2).astype(np.float64), 2))[2][2, 2] for p in pts])
    assert np.all(np.isfinite(got))
    assert normwise(got, ref) <= 2e-5


def test_rings_above_the_default_shared_memory_limit():
    """A DAG whose rings need more than 48 KB even at one column per thread
    (FP64, 256 threads, many wide fields) runs with the opt-in limit."""
    D = H.DagSpec(2)
    prev = "u"
    for k in range(7):
        refs = [(prev, (dx, dy)) for dx in (-2, 0, 2) for dy in (-2, 0, 2)]
        D.rule("EXPR", refs, [f"t{k}"], params=[0.1],
               expr="p0 * (in0 + in1 + in2 + in3 + in5 + in6 + in7 + in8) + (1 - 8 * p0) * in4")
        prev = f"t{k}"
    D.axiom("u"); D.goal(prev)
    rng = np.random.default_rng(8)
    core = rng.uniform(-1, 1, (200, 300))
    u = np.full((228, 328), np.nan)
    u[14:-14, 14:-14] = core
    (got,), _ = run_plan(D, [u], 14, "full:smem:128x2")
    rules = []
    prev = "u"
    for k in range(7):
        refs = [(prev, (dx, dy)) for dx in (-2, 0, 2) for dy in (-2, 0, 2)]
        rules.append((f"t{k}", refs, lambda *a: 0.1 * (sum(a[:4]) + sum(a[5:9])) + (1 - 0.8) * a[4], []))
        prev = f"t{k}"
    ref = E.evaluate(rules, {"u": core})[prev]
    assert normwise(got, ref) <= 1e-12
