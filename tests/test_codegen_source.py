"""Runtime code generation on the host (no GPU): DAGs with user rule bodies
(HFAV_OP_EXPR) plan onto generated kernels, bad bodies are refused at plan
creation, and the CUDA source the plan emits compiles with NVRTC for sm_103a
in both precisions under every schedule."""
import ctypes
import os

import numpy as np
import pytest

from paper_1710_08774_gb300 import hfav as H
from tests import expr_dags as X


def _grid(shape, halo):
    return H.Grid.of(np.zeros(tuple(n + 2 * halo for n in shape)), halo)


def _nvrtc():
    for name in ("libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13", "libnvrtc.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    pytest.skip("libnvrtc not available")


def _compile(L, src):
    prog = ctypes.c_void_p()
    assert L.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"generated.cu", 0, None, None) == 0
    opts = (ctypes.c_char_p * 2)(b"--gpu-architecture=sm_103a", b"--std=c++17")
    rc = L.nvrtcCompileProgram(prog, 2, opts)
    n = ctypes.c_size_t()
    L.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(max(1, n.value))
    L.nvrtcGetProgramLog(prog, log)
    L.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(errors="replace")


def _units(src):
    """The separately compiled units of a plan's source (each after a '// ---- kernel' line)."""
    return [u.split("\n", 1)[1] for u in src.split("// ---- kernel ")[1:]]


def test_expr_dag_plans_onto_generated_kernels():
    rules, axioms, goals = X.random_dag(2, 5, 0)
    P = H.Plan(X.to_spec(rules, axioms, goals, 2), [_grid((40, 30), 6)])
    assert P.dump()["pipeline"] == "codegen"
    assert P.schedule == "full:smem:32x8"          # the default in 2D
    assert set(P.variants()) == {f"{f}:{t}" for f in ("full:smem", "full:reg", "unfused:hbm")
                                 for t in ("32x4", "64x4", "128x2", "32x8")}
    with pytest.raises(H.HfavError):
        P.schedule = "full:hbm:32x4"
    with pytest.raises(H.HfavError):
        P.schedule = "sweep:smem:32x4"
    rules3, ax3, go3 = X.random_dag(3, 3, 1)
    P3 = H.Plan(X.to_spec(rules3, ax3, go3, 3), [_grid((12, 10, 8), 4)])
    assert P3.schedule.startswith("unfused")      # 3D: one generated kernel per rule
    assert P3.variants() == [f"unfused:hbm:{t}" for t in ("32x4", "64x4", "128x2", "32x8")]


BAD = [("in0; in1", "character ';'"), ("in2", "input"), ("p1", "parameter"), ("in0 // x", "comments"),
       ("#define X", "character '#'"), ("hfav_wrap(in0, 1)", "math function"), ("in0 + 'a'", "character"),
       ("", "1 to 4096"), ("x" * 5000, "1 to 4096"), ("in0 {", "character '{'"), ("*(&in0 + 9)", "'&'"),
       ("__trap()", "math function"), ("threadIdx.x", "math function"), ("in0[3]", "character '['"),
       ("printf(in0)", "math function"), ("asm(in0)", "math function")]


@pytest.mark.parametrize("body,why", BAD)
def test_bad_bodies_refused_at_plan_creation(body, why):
    D = H.DagSpec(2)
    D.rule("EXPR", [("u", (0, 0)), ("u", (1, 0))], ["o"], params=[1.0], expr=body)
    D.axiom("u"); D.goal("o")
    with pytest.raises(H.HfavError) as e:
        H.analyze(D)
    assert e.value.args and "EINVAL" in str(e.value) and why in str(e.value)


def test_good_bodies_accepted():
    for body in ("in0 + 1.5e-3 * p0", "fmax(in0, in1) > 0 && in1 < 2 ? (T)1 : (float)0.5f", "-in0 % 1 == 0 ? 1 : 2",
                 "pow(fabs(in0), 1.5) + hypot(in0, in1) + atan2(in1, 1 + in0 * in0)"):
        D = H.DagSpec(2)
        D.rule("EXPR", [("u", (0, 0)), ("u", (1, 0))], ["o"], params=[1.0], expr=body)
        D.axiom("u"); D.goal("o")
        H.analyze(D)


def test_builtin_plans_have_no_source():
    P = H.Plan(H.chain2d_dag(), [_grid((64, 64), 2)])
    with pytest.raises(H.HfavError):
        P.source()


@pytest.mark.parametrize("dtype", [H.HFAV_F64, H.HFAV_F32])
@pytest.mark.parametrize("seed", range(4))
def test_generated_source_compiles_with_nvrtc(dtype, seed):
    L = _nvrtc()
    rules, axioms, goals = X.random_dag(2, 6, seed)
    P = H.Plan(X.to_spec(rules, axioms, goals, 2), [_grid((50, 40), 8)], dtype)
    for sched in ("full:smem:32x4", "full:smem:128x2", "full:reg:32x4", "unfused:hbm:32x4"):
        if sched not in P.variants():
            continue   # warp strips take one-part DAGs only
        P.schedule = sched
        src = P.source()
        for body in {r["c"] for r in rules}:
            assert body in src
        units = _units(src)
        assert units
        for u in units:
            rc, log = _compile(L, u)
            assert rc == 0, log


def test_source_is_deterministic_and_mixes_catalogue_ops():
    D = H.DagSpec(2)
    D.rule("STENCIL_LINEAR", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))], ["L"],
           params=[1, 1, 1, 1, -4])
    D.rule("EXPR", [("L", (1, 0)), ("L", (0, 0))], ["d"], params=[0.5], expr="p0 * (in0 - in1)")
    D.rule("SQUASH", ["d"], ["o"])
    D.axiom("u"); D.goal("o")
    a = H.Plan(D, [_grid((64, 64), 2)]).source()
    b = H.Plan(D, [_grid((64, 64), 2)]).source()
    assert a == b and "hfav_cg_part" in a
    L = _nvrtc()
    for u in _units(a):
        rc, log = _compile(L, u)
        assert rc == 0, log


def test_pointwise_stages_are_inlined_and_the_goal_written_directly():
    """t0 and t1 (read only at offset 0, over their readers' tiles) get no
    shared tile; t2 (read at offsets) and the axiom a0 do; the goal is stored
    from its rule.  The source still compiles."""
    rules, axioms, goals = X.pointwise_dag()
    P = H.Plan(X.to_spec(rules, axioms, goals, 2), [_grid((64, 64), 3)], H.HFAV_F32, H.HFAV_BC_PERIODIC,
               "full:smem:32x4")
    src = P.source()
    names = P.spec.names
    tiles = {names[int(k)] for k in __import__("re").findall(r"T\* s(\d+) = ", src)}
    assert tiles == {"a0", "a1", "t2"}
    assert "hfav_body1(hfav_body0(" in src
    L = _nvrtc()
    for u in _units(src):
        rc, log = _compile(L, u)
        assert rc == 0, log


@pytest.mark.parametrize("dtype", [H.HFAV_F64, H.HFAV_F32])
@pytest.mark.parametrize("schedule", ["full:smem:32x4", "unfused:hbm:32x4"])
def test_reduction_sources_compile_with_nvrtc(dtype, schedule):
    """The normalization example and random DAGs with reductions: per-part
    kernels and finalizations all compile; the fused form has 2 grid kernels
    and 1 finalization for the normalization example, the unfused form 5 and 1."""
    L = _nvrtc()
    P = H.Plan(H.normalization_dag(), [_grid((64, 48), 1)], dtype, H.HFAV_BC_PERIODIC, schedule)
    src = P.source()
    heads = [l for l in src.splitlines() if l.startswith("// ---- kernel")]
    assert len(heads) == (3 if schedule.startswith("full") else 6)
    assert sum(h.endswith("finalize") for h in heads) == 1
    for seed in range(3):
        rules, axioms, goals = X.random_reduce_dag(seed)
        Q = H.Plan(X.to_spec_reduce(rules, axioms, goals), [_grid((64, 48), 6)], dtype, H.HFAV_BC_PERIODIC, schedule)
        src += "// ---- kernel x\n" + Q.source()
    for u in _units(src):
        rc, log = _compile(L, u)
        assert rc == 0, log


def test_inout_declarations_validated():
    D = H.DagSpec(2)
    D.rule("EXPR", [("u", (1, 0)), ("u", (-1, 0))], ["o"], expr="in0 - in1")
    D.axiom("u"); D.goal("o"); D.inout("o", "u")
    H.analyze(D)
    bad = H.DagSpec(2, feedback=True)
    bad.rule("EXPR", [("u", (1, 0))], ["o"], expr="in0")
    bad.axiom("u"); bad.goal("o"); bad.inout("o", "u")
    with pytest.raises(H.HfavError):
        H.analyze(bad)


@pytest.mark.parametrize("dtype", [H.HFAV_F64, H.HFAV_F32])
def test_inplace_sources_compile_with_nvrtc(dtype):
    """A declared in/out pair makes the fused 2D kernel read its halo bands
    from saved copies; the source compiles."""
    L = _nvrtc()
    D = H.chain2d_expr_dag()
    D.inout("out", "u")
    P = H.Plan(D, [_grid((64, 64), 2)], dtype, H.HFAV_BC_PERIODIC, "full:smem:32x4")
    src = P.source()
    assert "cb0" in src and "rb0" in src and "wint" in src
    for u in _units(src):
        rc, log = _compile(L, u)
        assert rc == 0, log


def test_non_finite_and_extreme_parameters_compile():
    """Parameters are baked in as literals: infinities, NaN, subnormals and
    integers all give a valid, exact literal."""
    L = _nvrtc()
    D = H.DagSpec(2)
    D.rule("EXPR", [("u", (0, 0))], ["o"], params=[float("inf"), float("nan"), 5e-324, 3.0, -float("inf")],
           expr="fmin(in0, p0) + (p1 != p1 ? p2 : 0) + p3 * in0 + fmax(p4, in0)")
    D.axiom("u"); D.goal("o")
    for dt in (H.HFAV_F64, H.HFAV_F32):
        src = H.Plan(D, [_grid((40, 30), 1)], dt, H.HFAV_BC_PERIODIC, "full:smem:32x4").source()
        assert "__longlong_as_double(0x7ff0000000000000ULL)" in src and "4.9406564584124654e-324" in src
        for u in _units(src):
            rc, log = _compile(L, u)
            assert rc == 0, log


def test_unsupported_scalar_forms_refused():
    """A grid field from scalars alone, a scalar read at an offset, a scalar
    goal, and a reduction in 3D have no generated kernels (EUNSUPPORTED)."""
    def dag(build, ndim=2):
        D = H.DagSpec(ndim)
        D.field("s", rank=0)
        build(D)
        return D
    cases = [
        lambda D: (D.rule("REDUCE_SUM", ["u"], ["s"]), D.rule("EXPR", ["s"], ["o"], expr="in0"), D.axiom("u"), D.goal("o")),
        lambda D: (D.rule("REDUCE_SUM", ["u"], ["s"]), D.rule("EXPR", ["u", ("s", (1, 0))], ["o"], expr="in0 + in1"),
                   D.axiom("u"), D.goal("o")),
        lambda D: (D.rule("REDUCE_SUM", ["u"], ["s"]), D.axiom("u"), D.goal("s")),
    ]
    for build in cases:
        with pytest.raises(H.HfavError):
            H.Plan(dag(build), [_grid((32, 32), 1)])
    D3 = H.DagSpec(3)
    D3.field("s", rank=0)
    D3.rule("REDUCE_SUM", ["u"], ["s"]); D3.rule("EXPR", ["u", "s"], ["o"], expr="in0 - in1")
    D3.axiom("u"); D3.goal("o")
    with pytest.raises(H.HfavError):
        H.Plan(D3, [H.Grid.of(np.zeros((10, 10, 10)), 1)])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("schedule", ["full:smem:32x4", "unfused:hbm:32x4"])
def test_generated_units_run_in_dependency_order(seed, schedule):
    """In the emitted program every scalar a kernel reads (sv<f>) is written by
    an earlier finalization (scal[f] = ...), and every finalization follows the
    kernel whose partials it combines."""
    import re
    rules, axioms, goals = X.random_reduce_dag(seed)
    P = H.Plan(X.to_spec_reduce(rules, axioms, goals), [_grid((64, 48), 6)], H.HFAV_F64, H.HFAV_BC_PERIODIC, schedule)
    src = P.source()
    units = src.split("// ---- kernel ")[1:]
    known = set()
    for k, u in enumerate(units):
        head = u.split("\n", 1)[0]
        body = u.split("\n", 1)[1]
        if head.endswith("finalize"):
            assert k > 0 and not units[k - 1].split("\n", 1)[0].endswith("finalize")
            assert "part[" in units[k - 1]          # the preceding kernel writes partials
            known |= {int(f) for f in re.findall(r"scal\[(\d+)\] = ", body)}
        else:
            for f in re.findall(r"\(T\)scal\[(\d+)\]", body):
                assert int(f) in known, (k, f)
    assert len(known) == sum(1 for r in rules if r["out"].startswith(("acc", "sc")))


def test_warp_strip_source_keeps_windows_in_registers():
    """The warp-strip form of the 2D chain written as rule bodies: no shared
    memory, no barrier, i-neighbours by shuffle, 16-byte loads and stores on
    the aligned path; it compiles in both precisions."""
    L = _nvrtc()
    for dt in (H.HFAV_F32, H.HFAV_F64):
        P = H.Plan(H.chain2d_expr_dag(), [_grid((256, 256), 2)], dt, H.HFAV_BC_PERIODIC, "full:reg:32x4")
        src = P.source()
        assert "hfav_cg_wstrip" in src and "__shared__" not in src and "__syncthreads" not in src
        assert "__shfl_up_sync" in src and "__shfl_down_sync" in src
        assert ("float4" if dt == H.HFAV_F32 else "double2") in src
        for u in _units(src):
            rc, log = _compile(L, u)
            assert rc == 0, log
