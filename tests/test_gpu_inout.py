"""Declared in/out aliasing (Sec. 3.5 "In/out chaining") on the GPU: an
in-place run gives bit for bit the result of the out-of-place run, and both
equal the CPU oracle (oracle.chain2d for the chain, oracle/expr.py for rule
bodies and random DAGs, oracle.cosmo) within the FP64 bar (1e-12 normwise;
FP32 2e-5).

- Generated fused 2D kernels update in place, reading the halo bands at CTA
  boundaries from copies saved before the launch: the 2D chain as rule
  bodies and random DAGs on grids of several strips and chunks, periodic and
  halo-given, FP64 and FP32, and a pointwise rule (no bands needed).
- Every other path (hand-written chains, COSMO, unfused, split DAGs) copies
  the aliased axiom to a snapshot first.
- An alias that was not declared is refused; a CUDA-graph replay matches.
"""
import numpy as np
import pytest

import oracle
from oracle import expr as E
from paper_1710_08774_gb300 import hfav as H
from paper_1710_08774_gb300 import inputs as I
from tests import expr_dags as X
from tests.gpu_util import normwise, to_dev

pytestmark = pytest.mark.gpu


def _twice(spec, arrays, halo, schedule, dtype=np.float64, bc=H.HFAV_BC_PERIODIC, alias=0, graph=False, n_goals=1):
    """(out-of-place goals, in-place goals) after one run of each: in the
    in-place run the first goal overwrites axiom `alias`, the others get arrays
    of their own."""
    import torch
    td = torch.float64 if dtype == np.float64 else torch.float32
    hd = H.HFAV_F64 if dtype == np.float64 else H.HFAV_F32
    ts = [to_dev(a, td) for a in arrays]
    ref = [torch.full_like(ts[0], float("nan")) for _ in range(n_goals)]
    P = H.Plan(spec, [H.Grid.of(ts[0], halo)], hd, bc, schedule)
    P.run(ts, ref, graph=graph)
    ins = [t.clone() for t in ts]
    outs = [ins[alias]] + [torch.full_like(ts[0], float("nan")) for _ in range(n_goals - 1)]
    P2 = H.Plan(spec, [H.Grid.of(ts[0], halo)], hd, bc, schedule)
    P2.run(ins, outs, graph=graph)
    torch.cuda.synchronize()
    crop = (slice(halo, -halo), slice(halo, -halo))
    if n_goals == 1:
        return ref[0][crop].cpu().numpy(), outs[0][crop].cpu().numpy(), P2
    return [r[crop].cpu().numpy() for r in ref], [o[crop].cpu().numpy() for o in outs], P2


@pytest.mark.parametrize("schedule", ["full:smem:32x4", "full:smem:128x2", "full:smem:32x8", "full:reg:32x4",
                                      "unfused:hbm:32x4"])
@pytest.mark.parametrize("shape", [(1500, 700), (515, 1031), (37, 5)])
def test_chain_as_rule_bodies_in_place(schedule, shape):
    D = H.chain2d_expr_dag()
    D.inout("out", "u")
    u = I.chain2d_input(shape[0], seed=1, ny=shape[1])
    ref, got, P = _twice(D, [u], 2, schedule)
    if schedule.startswith("full:reg"):
        # the aliased run takes the ring kernel, the other the warp strips:
        # equal to rounding (the warp strips may fuse across stages)
        assert normwise(ref, got) <= 1e-13
    else:
        assert np.array_equal(ref, got)
    assert normwise(got, oracle.chain2d(u)[2]) <= 1e-12
    if schedule.startswith("full"):   # the two band kernels and the update, no snapshot copy
        assert P.status()["last_launches"] == 3


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("bc", [H.HFAV_BC_PERIODIC, H.HFAV_BC_HALO_GIVEN])
def test_chain_in_place_f32_and_halo_given(dtype, bc):
    D = H.chain2d_expr_dag()
    D.inout("out", "u")
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, (904, 1203)).astype(dtype)
    ref, got, _ = _twice(D, [u], 2, "full:smem:32x4", dtype, bc)
    assert np.array_equal(ref, got)
    want = oracle.chain2d(u.astype(np.float64), periodic=bc == H.HFAV_BC_PERIODIC)[2]
    assert normwise(got, want) <= (1e-12 if dtype == np.float64 else 2e-5)


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("schedule", ["full:smem:32x4", "full:smem:64x4"])
def test_random_dags_in_place(seed, schedule):
    """Random DAGs (offsets in every direction, several stages): the first goal
    overwrites the first axiom.  Seeds 70 and 74 form one fused kernel (band
    path), the others several (snapshot path)."""
    rules, axioms, goals = X.random_dag(2, 5, seed + 70)
    D = X.to_spec(rules, axioms, goals, 2)
    D.inout(goals[0], axioms[0])
    P0 = H.analyze(D)
    h = max(max(P0.field(a)["halo_lo"] + P0.field(a)["halo_hi"]) for a in axioms)
    shape = (811, 1290)
    core = X.axiom_values(axioms, shape, seed)
    arrs = []
    for a in axioms:
        arr = np.full(tuple(n + 2 * h for n in shape), np.nan)
        arr[h:-h, h:-h] = core[a]
        arrs.append(arr)
    ref, got, P = _twice(D, arrs, h, schedule, n_goals=len(goals))
    if len(goals) == 1:
        ref, got = [ref], [got]
    want = E.evaluate(X.to_oracle(rules), core)
    for r, g, name in zip(ref, got, goals):
        assert np.array_equal(r, g)
        assert normwise(g, want[name]) <= 1e-12, name


def test_pointwise_in_place():
    D = H.DagSpec(2)
    D.rule("EXPR", ["u", "v"], ["o"], params=[0.5], expr="in0 * p0 + sqrt(fabs(in1))")
    D.axiom("u", "v"); D.goal("o"); D.inout("o", "v")
    rng = np.random.default_rng(4)
    u, v = rng.normal(size=(302, 502)), rng.normal(size=(302, 502))
    ref, got, _ = _twice(D, [u, v], 1, "full:smem:32x4", alias=1)
    assert np.array_equal(ref, got)
    assert normwise(got, u[1:-1, 1:-1] * 0.5 + np.sqrt(np.abs(v[1:-1, 1:-1]))) <= 1e-12


@pytest.mark.parametrize("case", ["chain2d", "cosmo2d", "normalization"])
def test_snapshot_paths(case):
    """Hand-written pipelines and split DAGs take a snapshot of the axiom."""
    if case == "chain2d":
        D, u, h, sched = H.chain2d_dag(), I.chain2d_input(700, seed=5, ny=300), 2, "full:reg:32x4"
    elif case == "cosmo2d":
        D, u, h, sched = H.cosmo_dag(ndim=2), I.cosmo_input(400, 300, 1, seed=6)[2], 2, "full:reg:32x4"
    else:
        D, u, h, sched = H.normalization_dag(), I.chain2d_input(700, seed=5, ny=300, halo=1), 1, "full:smem:32x4"
    D.inout(D.names[D.goals[0]], D.names[D.axioms[0]])
    ref, got, _ = _twice(D, [u], h, sched)
    assert np.array_equal(ref, got)
    if case == "chain2d":
        want = oracle.chain2d(u)[2]
    elif case == "cosmo2d":
        want = oracle.cosmo(np.stack([u] * 5), 0.05)[3][0]   # one plane; the k halo is never read
    else:
        want = E.evaluate(E.normalization_rules(), {"u": u[1:-1, 1:-1]})["out"]
    assert normwise(got, want) <= 1e-12


def test_undeclared_alias_refused_and_graph_replay():
    import torch
    u = to_dev(I.chain2d_input(300, seed=2, ny=200))
    P = H.Plan(H.chain2d_expr_dag(), [H.Grid.of(u, 2)], H.HFAV_F64, H.HFAV_BC_PERIODIC, "full:smem:32x4")
    with pytest.raises(H.HfavError):
        P.run([u], [u])
    D = H.chain2d_expr_dag()
    D.inout("out", "u")
    u = I.chain2d_input(1100, seed=2, ny=600)
    ref, got, _ = _twice(D, [u], 2, "full:smem:32x4", graph=True)
    assert np.array_equal(ref, got)
    assert normwise(got, oracle.chain2d(u)[2]) <= 1e-12


def test_autotune_leaves_in_place_arrays_unchanged():
    import torch
    D = H.chain2d_expr_dag()
    D.inout("out", "u")
    u = to_dev(I.chain2d_input(600, seed=4, ny=300))
    keep = u.clone()
    P = H.Plan(D, [H.Grid.of(u, 2)], H.HFAV_F64, H.HFAV_BC_PERIODIC)
    P.autotune([u], [u], reps=1)
    torch.cuda.synchronize()
    assert torch.equal(u[2:-2, 2:-2], keep[2:-2, 2:-2])


def test_split_dag_with_reduction_in_place():
    """Rule bodies, a maximum broadcast back, and an in-place update (the
    README example): the split makes two parts, so the run reads a snapshot."""
    import torch
    from oracle import expr as E
    D = H.DagSpec(2)
    D.rule("EXPR", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))], ["lap"],
           params=[4.0], expr="in0 + in1 + in2 + in3 - p0 * in4")
    D.field("m", rank=0)
    D.rule("REDUCE_MAX", ["lap"], ["m"])
    D.rule("EXPR", ["u", "lap", "m"], ["out"], params=[0.1], expr="in0 + p0 * in1 / fmax(in2, (T)1)")
    D.axiom("u"); D.goal("out"); D.inout("out", "u")
    rng = np.random.default_rng(12)
    core = rng.uniform(0, 1, (300, 500))
    u = np.full((304, 504), np.nan)
    u[2:-2, 2:-2] = core
    ut = to_dev(u)
    P = H.Plan(D, [H.Grid.of(ut, 2)], H.HFAV_F64, H.HFAV_BC_PERIODIC, "full:smem:32x8")
    P.run([ut], [ut])
    torch.cuda.synchronize()
    rules = [("lap", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))],
              lambda a, b, c, d, e: a + b + c + d - 4.0 * e, []),
             ("m", [("lap", (0, 0))], "max", []),
             ("out", [("u", (0, 0)), ("lap", (0, 0)), ("m", (0, 0))], lambda a, b, c: a + 0.1 * b / np.maximum(c, 1.0), [])]
    ref = E.evaluate(rules, {"u": core})["out"]
    got = ut[2:-2, 2:-2].cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-12
