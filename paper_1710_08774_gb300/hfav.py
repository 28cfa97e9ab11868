"""Thin ctypes binding of libhfav.so (include/hfav.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Functions keep the C names (``hfav_plan``, ``hfav_run``,
``hfav_status``, ``hfav_free`` ...); ``Plan`` wraps a plan handle and takes
torch tensors (their ``data_ptr()`` and the current CUDA stream).

There is no CPU fallback: ``load()`` raises when the library is missing.
"""
import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfav.so")

HFAV_OK = 0
HFAV_WARN_NEWTON = 1
ERRORS = {-1: "EINVAL", -2: "ECYCLE", -3: "EPRODUCER", -4: "EMISSING", -5: "EHALO", -6: "EALIGN",
          -7: "ENOMEM", -8: "ECUDA", -9: "ETIMEOUT", -10: "ENONPHYSICAL", -11: "EUNSUPPORTED"}
HFAV_F64, HFAV_F32 = 0, 1
HFAV_BC_PERIODIC, HFAV_BC_HALO_GIVEN = 0, 1
OP = dict(STENCIL_LINEAR=1, GRADMAG_HALF=2, SQUASH=3, GENERIC=4, LIMFLUX=5, DIFFUSE=6, EXPR=7, CONSTOPRIM=10, EOS=11, SLOPE=12, TRACE=13,
          QLEFTRIGHT=14, RIEMANN=15, CMPFLX=16, UPDATE=17, CFL_DT=20, REDUCE_SUM=21, BROADCAST=22, REDUCE_MAX=23)
STORAGE = ["axiom", "goal", "hbm", "rolling", "scalar"]
N_FEATURES = 16

# every symbol include/hfav.h declares
SYMBOLS = ["hfav_plan", "hfav_analyze", "hfav_plan_groups", "hfav_plan_field", "hfav_plan_order",
           "hfav_plan_set_schedule", "hfav_plan_schedule", "hfav_plan_dump", "hfav_plan_source", "hfav_plan_features", "hfav_run",
           "hfav_run_graph", "hfav_status", "hfav_autotune", "hfav_plan_variants", "hfav_free", "hfav_last_error",
           "hfav_version", "hfav_mlp_n_params", "hfav_mlp_forward", "hfav_mlp_work_floats", "hfav_mlp_loss_grad",
           "hfav_mlp_adam", "hfav_mlp_train", "hfav_model_choose", "hfav_plan_timing", "hfav_kernel_times",
           "hfav_chain2d_static", "hfav_selftest_arith", "hfav_selftest_rsqrt", "hfav_selftest_half", "hfav_selftest_convert", "hfav_inject_alloc_failure",
           "hfav_probe_peaks"]


class HfavError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Ref(ctypes.Structure):
    _fields_ = [("field", ctypes.c_int), ("off", ctypes.c_int * 3)]


class Rule(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("axis", ctypes.c_int), ("n_in", ctypes.c_int), ("in_", ctypes.POINTER(Ref)),
                ("n_out", ctypes.c_int), ("out", ctypes.POINTER(ctypes.c_int)), ("n_params", ctypes.c_int),
                ("params", ctypes.POINTER(ctypes.c_double)), ("expr", ctypes.c_char_p)]


class Dag(ctypes.Structure):
    _fields_ = [("n_fields", ctypes.c_int), ("field_rank", ctypes.POINTER(ctypes.c_int)), ("n_rules", ctypes.c_int),
                ("rules", ctypes.POINTER(Rule)), ("n_axioms", ctypes.c_int), ("axioms", ctypes.POINTER(ctypes.c_int)),
                ("n_goals", ctypes.c_int), ("goals", ctypes.POINTER(ctypes.c_int)), ("ndim", ctypes.c_int),
                ("stream_axis", ctypes.c_int), ("feedback", ctypes.c_int), ("inout", ctypes.POINTER(ctypes.c_int))]


class Grid(ctypes.Structure):
    _fields_ = [("extent", ctypes.c_int64 * 3), ("pitch", ctypes.c_int64 * 3), ("halo", ctypes.c_int)]

    @staticmethod
    def make(extent, pitch, halo):
        g = Grid()
        e = list(extent) + [1] * (3 - len(extent))
        p = list(pitch) + [0] * (3 - len(pitch))
        for a in range(3):
            g.extent[a] = int(e[a])
            g.pitch[a] = int(p[a])
        g.halo = int(halo)
        return g

    @staticmethod
    def of(t, halo):
        """Grid of a halo-padded tensor / array laid out (..., j, i), i contiguous."""
        shape = list(t.shape)
        strides = list(t.stride()) if hasattr(t, "stride") and callable(t.stride) else \
            [s // t.itemsize for s in t.strides]
        if strides[-1] != 1:
            raise ValueError("axis i must be contiguous")
        nd = len(shape)
        ext = [shape[nd - 1 - a] - 2 * halo for a in range(nd)]
        pitch = [1] + [strides[nd - 1 - a] for a in range(1, nd)]
        return Grid.make(ext, pitch, halo)


class FieldInfo(ctypes.Structure):
    _fields_ = [("producer", ctypes.c_int), ("group", ctypes.c_int), ("storage", ctypes.c_int),
                ("halo_lo", ctypes.c_int * 3), ("halo_hi", ctypes.c_int * 3), ("window", ctypes.c_int * 3),
                ("stage_window", ctypes.c_int * 3), ("storage_elems", ctypes.c_int64), ("n_reuse", ctypes.c_int),
                ("reuse", (ctypes.c_int * 3) * 27)]


class RunStats(ctypes.Structure):
    _fields_ = [("newton_nonconverged", ctypes.c_int64), ("nonphysical", ctypes.c_int64), ("n_dt", ctypes.c_int),
                ("dt", ctypes.c_double * 64), ("last_ms", ctypes.c_double), ("last_launches", ctypes.c_int)]


_lib = None


def load(path=None):
    """Load libhfav.so (built by ``paper_1710_08774_gb300.build``).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_1710_08774_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    ip = ctypes.POINTER(ctypes.c_int)
    fp = ctypes.POINTER(ctypes.c_float)
    sig = {
        "hfav_plan": ([ctypes.POINTER(Dag), ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                       ctypes.c_char_p, ctypes.POINTER(P)], ctypes.c_int),
        "hfav_analyze": ([ctypes.POINTER(Dag), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(P)], ctypes.c_int),
        "hfav_plan_groups": ([P, ip, ip, ctypes.c_int], ctypes.c_int),
        "hfav_plan_field": ([P, ctypes.c_int, ctypes.POINTER(FieldInfo)], ctypes.c_int),
        "hfav_plan_order": ([P, ip, ctypes.c_int], ctypes.c_int),
        "hfav_plan_set_schedule": ([P, ctypes.c_char_p], ctypes.c_int),
        "hfav_plan_schedule": ([P, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "hfav_plan_dump": ([P, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "hfav_plan_source": ([P, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "hfav_plan_features": ([P, ctypes.c_char_p, fp], ctypes.c_int),
        "hfav_run": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int, P], ctypes.c_int),
        "hfav_run_graph": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int, P], ctypes.c_int),
        "hfav_status": ([P, ctypes.POINTER(RunStats)], ctypes.c_int),
        "hfav_autotune": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, P, fp, ctypes.c_int],
                          ctypes.c_int),
        "hfav_plan_variants": ([P, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "hfav_free": ([P], None),
        "hfav_last_error": ([], ctypes.c_char_p),
        "hfav_version": ([], ctypes.c_int),
        "hfav_mlp_n_params": ([ctypes.c_int, ctypes.c_int], ctypes.c_int64),
        "hfav_mlp_forward": ([P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P], ctypes.c_int),
        "hfav_mlp_work_floats": ([ctypes.c_int, ctypes.c_int], ctypes.c_int64),
        "hfav_mlp_loss_grad": ([P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P], ctypes.c_int),
        "hfav_mlp_adam": ([P, P, P, P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, ctypes.c_int, P], ctypes.c_int),
        "hfav_mlp_train": ([P, P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                            P, P, P, P], ctypes.c_int),
        "hfav_model_choose": ([P, P, ctypes.c_int, ctypes.c_int, fp, fp, fp, ctypes.c_int, ctypes.c_char_p,
                               ctypes.c_size_t], ctypes.c_int),
        "hfav_plan_timing": ([P, ctypes.c_int], ctypes.c_int),
        "hfav_selftest_arith": ([P, ctypes.c_int64, P, P, P], ctypes.c_int),
        "hfav_selftest_rsqrt": ([P, ctypes.c_int64, P, P], ctypes.c_int),
        "hfav_selftest_half": ([P, ctypes.c_int64, P, P], ctypes.c_int),
        "hfav_selftest_convert": ([P, P, ctypes.c_int64, P, P, P], ctypes.c_int),
        "hfav_chain2d_static": ([P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_double), P, P], ctypes.c_int),
        "hfav_kernel_times": ([P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double), ip,
                               ctypes.c_int], ctypes.c_int),
        "hfav_inject_alloc_failure": ([ctypes.c_int], ctypes.c_int),
        "hfav_probe_peaks": ([ctypes.POINTER(ctypes.c_double), ctypes.c_int, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def check(rc):
    if rc < 0:
        raise HfavError(rc, load().hfav_last_error().decode())
    return rc


# ---------------------------------------------------------------------------
# rule DAGs (the front-end: the paper's axioms, goals and production rules)
# ---------------------------------------------------------------------------
class DagSpec:
    """Builder of an hfav_dag.  Fields are named; refs are (name, (di, dj, dk))."""

    def __init__(self, ndim, stream_axis=None, feedback=False):
        self.ndim = ndim
        self.stream_axis = ndim - 1 if stream_axis is None else stream_axis
        self.feedback = int(bool(feedback))
        self.names, self.rank = [], []
        self.rules = []
        self.axioms, self.goals = [], []

    def field(self, name, rank=None):
        if name not in self.names:
            self.names.append(name)
            self.rank.append(self.ndim if rank is None else rank)
        return self.names.index(name)

    def rule(self, op, ins, outs, params=(), axis=0, expr=None):
        """A rule; `expr` is the C body of an EXPR rule (over in0 .., p0 ..)."""
        refs = []
        for r in ins:
            name, off = (r, (0, 0, 0)) if isinstance(r, str) else r
            off = tuple(off) + (0,) * (3 - len(off))
            refs.append((self.field(name), off))
        out = [self.field(o) for o in outs]
        self.rules.append((OP[op] if isinstance(op, str) else op, axis, refs, out, list(params), expr))
        return len(self.rules) - 1

    def axiom(self, *names):
        self.axioms += [self.field(n) for n in names]

    def goal(self, *names):
        self.goals += [self.field(n) for n in names]

    def inout(self, goal, axiom):
        """Declare that `goal`'s array may be `axiom`'s array (an in-place update)."""
        self.aliases = getattr(self, "aliases", {})
        self.aliases[self.field(goal)] = self.field(axiom)

    def c(self):
        """The hfav_dag struct (kept alive by this object)."""
        keep = []
        rules = (Rule * len(self.rules))()
        for k, (op, axis, refs, out, params, expr) in enumerate(self.rules):
            R = rules[k]
            R.op, R.axis = op, axis
            ra = (Ref * max(1, len(refs)))()
            for m, (f, off) in enumerate(refs):
                ra[m].field = f
                for a in range(3):
                    ra[m].off[a] = off[a]
            oa = (ctypes.c_int * len(out))(*out)
            pa = (ctypes.c_double * max(1, len(params)))(*params)
            keep += [ra, oa, pa]
            R.n_in, R.in_ = len(refs), ra
            R.n_out, R.out = len(out), oa
            R.n_params, R.params = len(params), pa
            if expr is not None:
                eb = ctypes.create_string_buffer(expr.encode())
                keep.append(eb)
                R.expr = ctypes.cast(eb, ctypes.c_char_p)
        d = Dag()
        rk = (ctypes.c_int * len(self.rank))(*self.rank)
        ax = (ctypes.c_int * max(1, len(self.axioms)))(*self.axioms)
        go = (ctypes.c_int * max(1, len(self.goals)))(*self.goals)
        keep += [rules, rk, ax, go]
        d.n_fields, d.field_rank = len(self.rank), rk
        d.n_rules, d.rules = len(self.rules), rules
        d.n_axioms, d.axioms = len(self.axioms), ax
        d.n_goals, d.goals = len(self.goals), go
        d.ndim, d.stream_axis, d.feedback = self.ndim, self.stream_axis, self.feedback
        aliases = getattr(self, "aliases", {})
        if aliases:
            io = (ctypes.c_int * len(self.goals))(*[self.axioms.index(aliases[g]) if g in aliases else -1
                                                   for g in self.goals])
            keep.append(io)
            d.inout = io
        self._keep = keep
        self._c = d
        return d


def _off(axis, d):
    o = [0, 0, 0]
    o[axis] = d
    return tuple(o)


def chain2d_dag():
    """L = u(i+1)+u(i-1)+u(j+1)+u(j-1)-4u; G = |central grad L|/2; out = G/(1+G)."""
    D = DagSpec(2, stream_axis=1)
    D.rule("STENCIL_LINEAR", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))], ["L"],
           params=[1, 1, 1, 1, -4])
    D.rule("GRADMAG_HALF", [("L", (1, 0)), ("L", (-1, 0)), ("L", (0, 1)), ("L", (0, -1))], ["G"])
    D.rule("SQUASH", ["G"], ["out"])
    D.axiom("u")
    D.goal("out")
    return D


def chain2d_expr_dag():
    """The 2D chain of chain2d_dag written as user rule bodies (EXPR): runs on
    kernels generated and compiled at run time instead of the builtin ones."""
    D = DagSpec(2, stream_axis=1)
    D.rule("EXPR", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))], ["L"],
           params=[4.0], expr="in0 + in1 + in2 + in3 - p0 * in4")
    D.rule("EXPR", [("L", (1, 0)), ("L", (-1, 0)), ("L", (0, 1)), ("L", (0, -1))], ["G"],
           expr="sqrt((in0 - in1) * (in0 - in1) + (in2 - in3) * (in2 - in3)) * (T)0.5")
    D.rule("EXPR", ["G"], ["out"], expr="in0 / (1 + in0)")
    D.axiom("u")
    D.goal("out")
    return D


def normalization_dag():
    """The normalization example (Sec. 5.2) as rule bodies: flux = u(i+1) - u(i),
    diff = flux(i) - flux(i-1), the norm accumulation acc = sum of diff^2 (a
    reduction), its root, out = diff / root (a broadcast).  The reduction feeding
    the broadcast splits the DAG into two nests."""
    D = DagSpec(2, stream_axis=1)
    D.rule("EXPR", [("u", (1, 0)), ("u", (0, 0))], ["flux"], expr="in0 - in1")
    D.rule("EXPR", [("flux", (0, 0)), ("flux", (-1, 0))], ["diff"], expr="in0 - in1")
    D.rule("EXPR", ["diff"], ["sq"], expr="in0 * in0")
    D.field("acc", rank=0)
    D.field("root", rank=0)
    D.rule("REDUCE_SUM", ["sq"], ["acc"])
    D.rule("EXPR", ["acc"], ["root"], expr="sqrt(in0)")
    D.rule("EXPR", ["diff", "root"], ["out"], expr="in0 / in1")
    D.axiom("u")
    D.goal("out")
    return D


def chain3d_dag():
    """s1 = D7 u; s2 = D7 s1; s3 = |central grad s2|/2; out = s3/(1+s3)."""
    D = DagSpec(3, stream_axis=2)
    star = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (0, 0, 0)]
    w = [1, 1, 1, 1, 1, 1, -6]
    D.rule("STENCIL_LINEAR", [("u", o) for o in star], ["s1"], params=w)
    D.rule("STENCIL_LINEAR", [("s1", o) for o in star], ["s2"], params=w)
    D.rule("GRADMAG_HALF", [("s2", o) for o in star[:6]], ["s3"])
    D.rule("SQUASH", ["s3"], ["out"])
    D.axiom("u")
    D.goal("out")
    return D


def cosmo_dag(c=0.05, ndim=3):
    """COSMO horizontal diffusion (Sec. 5.3): ulapstage (5-point Laplacian of
    u), flux_x / flux_y (limited Laplacian differences across the faces i+1/2,
    j+1/2), ustage (u minus c times the flux divergence); no dependency in k."""
    D = DagSpec(ndim, stream_axis=ndim - 1)
    z = (0,) * (ndim - 2)
    D.rule("STENCIL_LINEAR", [("u", (1, 0) + z), ("u", (-1, 0) + z), ("u", (0, 1) + z), ("u", (0, -1) + z),
                              ("u", (0, 0) + z)], ["lap"], params=[1, 1, 1, 1, -4])
    D.rule("LIMFLUX", [("u", (0, 0) + z), ("u", (1, 0) + z), ("lap", (0, 0) + z), ("lap", (1, 0) + z)], ["flx"],
           axis=0)
    D.rule("LIMFLUX", [("u", (0, 0) + z), ("u", (0, 1) + z), ("lap", (0, 0) + z), ("lap", (0, 1) + z)], ["fly"],
           axis=1)
    D.rule("DIFFUSE", [("u", (0, 0) + z), ("flx", (-1, 0) + z), ("flx", (0, 0) + z), ("fly", (0, -1) + z),
                       ("fly", (0, 0) + z)], ["out"], params=[c])
    D.axiom("u")
    D.goal("out")
    return D


def godunov_dag(gamma=1.4, cfl=0.5, axes=(0, 1), newton_max=None):
    """Directionally split Godunov step: the Hydro2D kernels once per pass
    (x then y), the CFL time step as a reduction of the state entering the
    step, and the goals fed back as next step's axioms.  newton_max (1..10)
    caps the Riemann solver's Newton iterations (default 10)."""
    D = DagSpec(2, stream_axis=1, feedback=True)
    U = ["U0", "U1", "U2", "U3"]
    D.field("dt", rank=0)
    D.rule("CFL_DT", U, ["dt"], params=[cfl, gamma])
    cur = U
    for n, a in enumerate(axes):
        s = "xy"[a]
        f = lambda base: f"{base}_{s}"
        D.rule("CONSTOPRIM", cur, [f("r"), f("un"), f("ut"), f("e")], params=[gamma], axis=a)
        D.rule("EOS", [f("r"), f("e")], [f("p"), f("c")], params=[gamma], axis=a)
        prim = [f("r"), f("un"), f("ut"), f("p")]
        D.rule("SLOPE", [(q, _off(a, d)) for q in prim for d in (-1, 0, 1)],
               [f("dr"), f("dun"), f("dut"), f("dp")], params=[gamma], axis=a)
        qm = [f(f"qm{k}") for k in range(4)]
        qp = [f(f"qp{k}") for k in range(4)]
        D.rule("TRACE", prim + [f("c"), f("dr"), f("dun"), f("dut"), f("dp"), "dt"], qm + qp, params=[gamma], axis=a)
        qL = [f(f"qL{k}") for k in range(4)]
        qR = [f(f"qR{k}") for k in range(4)]
        D.rule("QLEFTRIGHT", [(q, (0, 0)) for q in qp] + [(q, _off(a, 1)) for q in qm], qL + qR, params=[gamma],
               axis=a)
        g = [f(f"g{k}") for k in range(4)]
        D.rule("RIEMANN", qL + qR, g, params=[gamma] if newton_max is None else [gamma, newton_max], axis=a)
        F = [f(f"F{k}") for k in range(4)]
        D.rule("CMPFLX", g, F, params=[gamma], axis=a)
        nxt = [f"U{k}_{s}" for k in range(4)]
        D.rule("UPDATE", cur + F + [(q, _off(a, -1)) for q in F] + ["dt"], nxt, params=[gamma], axis=a)
        cur = nxt
    D.axiom(*U)
    D.goal(*cur)
    return D


# ---------------------------------------------------------------------------
# plans
# ---------------------------------------------------------------------------
def _ptr(x):
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Plan:
    """An hfav_plan_t: analysis (always) plus, with grids, an executable schedule."""

    def __init__(self, dag, grids=None, dtype=HFAV_F64, bc=HFAV_BC_PERIODIC, schedule=None, extent=None):
        L = load()
        self.spec = dag
        self._dag = dag.c()
        self.h = ctypes.c_void_p()
        if grids is None:
            ext = None
            if extent is not None:
                ext = (ctypes.c_int64 * 3)(*(list(extent) + [1] * (3 - len(extent))))
            check(L.hfav_analyze(ctypes.byref(self._dag), ext, ctypes.byref(self.h)))
            self.n_grids = 0
        else:
            ga = (Grid * len(grids))(*grids)
            self._grids = ga
            check(L.hfav_plan(ctypes.byref(self._dag), ga, len(grids), dtype, bc,
                              None if schedule is None else schedule.encode(), ctypes.byref(self.h)))
            self.n_grids = len(grids)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None) and self.h.value:
            load().hfav_free(self.h)
            self.h = ctypes.c_void_p()

    # -- analysis -----------------------------------------------------------
    def groups(self):
        n = ctypes.c_int()
        rg = (ctypes.c_int * len(self.spec.rules))()
        check(load().hfav_plan_groups(self.h, ctypes.byref(n), rg, len(self.spec.rules)))
        return n.value, list(rg)

    def order(self):
        o = (ctypes.c_int * len(self.spec.rules))()
        check(load().hfav_plan_order(self.h, o, len(self.spec.rules)))
        return list(o)

    def field(self, name):
        fid = self.spec.names.index(name) if isinstance(name, str) else name
        fi = FieldInfo()
        check(load().hfav_plan_field(self.h, fid, ctypes.byref(fi)))
        return dict(producer=fi.producer, group=fi.group, storage=STORAGE[fi.storage],
                    halo_lo=list(fi.halo_lo), halo_hi=list(fi.halo_hi), window=list(fi.window),
                    stage_window=list(fi.stage_window), storage_elems=fi.storage_elems,
                    reuse=[tuple(fi.reuse[k]) for k in range(fi.n_reuse)])

    def dump(self):
        buf = ctypes.create_string_buffer(1 << 20)
        check(load().hfav_plan_dump(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def source(self):
        """CUDA source of the plan's generated kernels (DAGs with EXPR rules)."""
        buf = ctypes.create_string_buffer(1 << 22)
        check(load().hfav_plan_source(self.h, buf, len(buf)))
        return buf.value.decode()

    # -- schedule -------------------------------------------------------------
    @property
    def schedule(self):
        buf = ctypes.create_string_buffer(128)
        check(load().hfav_plan_schedule(self.h, buf, len(buf)))
        return buf.value.decode()

    @schedule.setter
    def schedule(self, s):
        check(load().hfav_plan_set_schedule(self.h, s.encode()))

    def variants(self):
        buf = ctypes.create_string_buffer(1 << 14)
        check(load().hfav_plan_variants(self.h, buf, len(buf)))
        return [v for v in buf.value.decode().split("\n") if v]

    def features(self, schedule=None):
        f = (ctypes.c_float * N_FEATURES)()
        check(load().hfav_plan_features(self.h, None if schedule is None else schedule.encode(), f))
        return np.array(list(f), dtype=np.float32)

    # -- execution ------------------------------------------------------------
    @staticmethod
    def _table(ts):
        flat = []
        for t in ts:
            flat += list(t) if isinstance(t, (list, tuple)) else [t]
        return (ctypes.c_void_p * len(flat))(*[_ptr(t) for t in flat])

    def run(self, axioms, goals, n_steps=1, stream=None, graph=False):
        """axioms / goals: tensors, grid-major (grid 0's fields, then grid 1's ...)."""
        a, g = self._table(axioms), self._table(goals)
        fn = load().hfav_run_graph if graph else load().hfav_run
        check(fn(self.h, a, g, n_steps, _stream(stream)))

    def status(self):
        st = RunStats()
        rc = check(load().hfav_status(self.h, ctypes.byref(st)))
        return dict(rc=rc, newton_nonconverged=st.newton_nonconverged, nonphysical=st.nonphysical,
                    dt=list(st.dt[:st.n_dt]), last_ms=st.last_ms, last_launches=st.last_launches)

    def timing(self, on=True):
        check(load().hfav_plan_timing(self.h, int(bool(on))))

    def kernel_times(self):
        """{kernel name: (total ms, launches)} of the last run with timing on."""
        names = ctypes.create_string_buffer(1 << 14)
        ms = (ctypes.c_double * 64)()
        cnt = (ctypes.c_int * 64)()
        n = check(load().hfav_kernel_times(self.h, names, len(names), ms, cnt, 64))
        nm = names.value.decode().split("\n")
        return {nm[k]: (ms[k], cnt[k]) for k in range(n)}

    def autotune(self, axioms, goals, n_steps=1, reps=3, stream=None):
        vs = self.variants()
        times = (ctypes.c_float * len(vs))()
        check(load().hfav_autotune(self.h, self._table(axioms), self._table(goals), n_steps, reps, _stream(stream),
                                   times, len(vs)))
        return dict(zip(vs, [float(t) for t in times]))

    def model_choose(self, params, hidden, shift=None, scale=None, n_models=1):
        vs = self.variants()
        pred = (ctypes.c_float * len(vs))()
        best = ctypes.create_string_buffer(128)
        fp = ctypes.POINTER(ctypes.c_float)
        sh = None if shift is None else (ctypes.c_float * N_FEATURES)(*[float(x) for x in shift])
        sc = None if scale is None else (ctypes.c_float * N_FEATURES)(*[float(x) for x in scale])
        check(load().hfav_model_choose(self.h, _ptr(params), n_models, hidden, sh, sc, pred, len(vs), best,
                                       len(best)))
        return best.value.decode(), dict(zip(vs, [float(x) for x in pred]))


def analyze(dag, extent=None):
    return Plan(dag, extent=extent)


# ---------------------------------------------------------------------------
# MLP kernels
# ---------------------------------------------------------------------------
def probe_peaks(stream=None):
    """Measured peaks of the current device: FP64 FMA/s (the FP64 pipe's issue
    rate), FP64 divide/s, sqrt/s, rsqrt/s and FP32 FMA/s (per second, whole
    GPU)."""
    r = (ctypes.c_double * 5)()
    check(load().hfav_probe_peaks(r, 5, _stream(stream)))
    return dict(dfma=r[0], ddiv=r[1], dsqrt=r[2], drsqrt=r[3], ffma=r[4])


def mlp_n_params(n_in, hidden):
    return int(load().hfav_mlp_n_params(n_in, hidden))


def mlp_forward(params, X, hidden, y, stream=None):
    n, n_in = X.shape
    check(load().hfav_mlp_forward(_ptr(params), n_in, hidden, _ptr(X), n, _ptr(y), _stream(stream)))


def mlp_loss_grad(params, X, t, hidden, grad, loss, work, stream=None):
    n, n_in = X.shape
    check(load().hfav_mlp_loss_grad(_ptr(params), n_in, hidden, _ptr(X), _ptr(t), n, _ptr(grad), _ptr(loss),
                                    _ptr(work), _stream(stream)))


def mlp_work_floats(n, hidden):
    return int(load().hfav_mlp_work_floats(n, hidden))


def mlp_adam(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(load().hfav_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), lr, beta1, beta2, eps,
                               step, _stream(stream)))


def mlp_train(params, m, v, X, t, hidden, epochs, lr, work, grad, loss_hist, stream=None):
    n, n_in = X.shape
    check(load().hfav_mlp_train(_ptr(params), _ptr(m), _ptr(v), n_in, hidden, _ptr(X), _ptr(t), n, epochs, lr,
                                _ptr(work), _ptr(grad), _ptr(loss_hist), _stream(stream)))
