"""Seeded random DAGs of user rule bodies (HFAV_OP_EXPR) for the tests.

Each rule body is given twice: as the C expression the library compiles and
as the numpy function the oracle evaluates -- the same user kernel written for
each side, so neither side's arithmetic comes from the other.  The bodies are
continuous in their inputs (so an FP32 run and the FP64 oracle take no
different branch at a near-tie) and keep values O(1) along a chain.
"""
import numpy as np

# (C body, numpy body, number of inputs, parameter range or None per parameter)
BODIES = [
    ("p0 * in0 + p1 * in1", lambda a, b, p0, p1: p0 * a + p1 * b, 2, [(-0.9, 0.9), (-0.9, 0.9)]),
    ("fmax(in0, in1) - p0 * in2", lambda a, b, c, p0: np.maximum(a, b) - p0 * c, 3, [(0.1, 0.6)]),
    ("in0 > in1 ? in0 - in1 : p0 * (in0 - in1)", lambda a, b, p0: np.where(a > b, a - b, p0 * (a - b)), 2,
     [(0.2, 0.8)]),
    ("sqrt(in0 * in0 + p0)", lambda a, p0: np.sqrt(a * a + p0), 1, [(0.1, 1.0)]),
    ("in0 / (1 + fabs(in1))", lambda a, b: a / (1 + np.abs(b)), 2, []),
    ("exp(-in0 * in0) * in1 + p0 * in2", lambda a, b, c, p0: np.exp(-a * a) * b + p0 * c, 3, [(-0.5, 0.5)]),
    ("fmin(in0, in1) * p0 + tanh(in2)", lambda a, b, c, p0: np.minimum(a, b) * p0 + np.tanh(c), 3, [(0.3, 0.9)]),
    ("(in0 + in1 + in2 + in3 - 4 * in4) * p0", lambda a, b, c, d, e, p0: (a + b + c + d - 4 * e) * p0, 5,
     [(0.1, 0.3)]),
]


def random_dag(ndim, n_rules, seed, radius=1, n_axioms=2):
    """Rules as dicts {out, refs, c, fn, params}; axioms; goals (the outputs no
    later rule reads).  Offsets are drawn within `radius` on every axis."""
    rng = np.random.default_rng(seed)
    axioms = [f"a{k}" for k in range(n_axioms)]
    fields = list(axioms)
    rules, read = [], set()
    for r in range(n_rules):
        c, fn, n_in, prange = BODIES[rng.integers(len(BODIES))]
        refs = []
        for k in range(n_in):
            # favour recent fields so chains grow deep
            f = fields[max(0, len(fields) - 1 - int(rng.integers(0, 3)))] if rng.random() < 0.7 else \
                fields[int(rng.integers(len(fields)))]
            off = tuple(int(rng.integers(-radius, radius + 1)) for _ in range(ndim)) + (0,) * (3 - ndim)
            refs.append((f, off))
            read.add(f)
        params = [float(rng.uniform(lo, hi)) for lo, hi in prange]
        out = f"t{r}"
        rules.append(dict(out=out, refs=refs, c=c, fn=fn, params=params))
        fields.append(out)
    goals = [r["out"] for r in rules if r["out"] not in read]
    return rules, axioms, goals


def to_spec(rules, axioms, goals, ndim, shuffle_seed=None):
    """The DAG as an hfav DagSpec of EXPR rules (optionally in shuffled order)."""
    from paper_1710_08774_gb300 import hfav as H
    D = H.DagSpec(ndim)
    for a in axioms:
        D.field(a)
    order = list(range(len(rules)))
    if shuffle_seed is not None:
        np.random.default_rng(shuffle_seed).shuffle(order)
    for k in order:
        r = rules[k]
        D.rule("EXPR", [(f, off[:ndim]) for f, off in r["refs"]], [r["out"]], params=r["params"], expr=r["c"])
    D.axiom(*axioms)
    D.goal(*goals)
    return D


def to_oracle(rules):
    """The DAG in the oracle's form: (out, refs, numpy body, params)."""
    return [(r["out"], r["refs"], r["fn"], r["params"]) for r in rules]


def axiom_values(axioms, shape, seed):
    """Smooth-plus-noise O(1) axiom fields of the given numpy shape (..., j, i)."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    vals = {}
    for k, a in enumerate(axioms):
        smooth = sum(np.sin(2 * np.pi * (k + 1 + d) * g / n) for d, (g, n) in enumerate(zip(grids, shape)))
        vals[a] = 0.5 * smooth / len(shape) + 0.5 * rng.uniform(-1, 1, shape)
    return vals


def pointwise_dag():
    """A DAG whose pointwise stages (read only at offset 0) nest: t0 a stencil
    of a0, t1 = f(t0), t2 = g(t1, t0, a1), t3 a stencil of t2, goal = h(t3)."""
    z = (0, 0, 0)
    star = [((1, 0, 0)), ((-1, 0, 0)), ((0, 1, 0)), ((0, -1, 0)), z]
    rules = [
        dict(out="t0", refs=[("a0", o) for o in star], c=BODIES[7][0], fn=BODIES[7][1], params=[0.25]),
        dict(out="t1", refs=[("t0", z)], c="sqrt(in0 * in0 + p0)", fn=lambda a, p0: np.sqrt(a * a + p0),
             params=[0.5]),
        dict(out="t2", refs=[("t1", z), ("t0", z), ("a1", z)], c="fmax(in0, in1) - p0 * in2",
             fn=lambda a, b, c, p0: np.maximum(a, b) - p0 * c, params=[0.3]),
        dict(out="t3", refs=[("t2", (1, 1, 0)), ("t2", (-1, 0, 0)), ("t2", (0, -1, 0))],
             c="p0 * in0 + p1 * (in1 - in2)", fn=lambda a, b, c, p0, p1: p0 * a + p1 * (b - c), params=[0.7, 0.4]),
        dict(out="g", refs=[("t3", z)], c="in0 / (1 + fabs(in0))", fn=lambda a: a / (1 + np.abs(a)), params=[]),
    ]
    return rules, ["a0", "a1"], ["g"]


# scalar finalization bodies (C, numpy, n_in, parameter ranges) and broadcast
# consumers (a grid field and a scalar)
SCALAR_BODIES = [
    ("sqrt(fabs(in0) + p0)", lambda a, p0: np.sqrt(np.abs(a) + p0), 1, [(0.5, 2.0)]),
    ("in0 * p0 + 1", lambda a, p0: a * p0 + 1, 1, [(-0.01, 0.01)]),
]
BROADCAST_BODIES = [
    ("in0 / in1", lambda a, b: a / b, [(0.0, 0.0)]),
    ("in0 - p0 * in1", lambda a, b, p0: a - p0 * b, [(0.001, 0.01)]),
]


def random_reduce_dag(seed, n_grid=4):
    """A random grid DAG (as random_dag), reductions (sum or max) of two of its
    fields, a scalar rule on each, and broadcast consumers: a split between a
    nest that reduces and one that reads the scalars.  Returns rules in the
    tests' dict form with `op` set for reductions, the axioms and goals."""
    rng = np.random.default_rng(1000 + seed)
    rules, axioms, _ = random_dag(2, n_grid, seed)
    grid_fields = [r["out"] for r in rules]
    extra = []
    for k, f in enumerate(rng.choice(grid_fields, size=2, replace=False)):
        op = "sum" if k == 0 else "max"
        extra.append(dict(out=f"acc{k}", refs=[(str(f), (0, 0, 0))], op=op))
        c, fn, _, prange = SCALAR_BODIES[k]
        params = [float(rng.uniform(lo, hi)) for lo, hi in prange]
        extra.append(dict(out=f"sc{k}", refs=[(f"acc{k}", (0, 0, 0))], c=c, fn=fn, params=params))
    for k in range(2):
        c, fn, prange = BROADCAST_BODIES[k]
        params = [float(rng.uniform(lo, hi)) for lo, hi in prange if hi > 0]
        src = str(rng.choice(grid_fields))
        off = tuple(int(v) for v in rng.integers(-1, 2, size=2)) + (0,)
        extra.append(dict(out=f"b{k}", refs=[(src, off), (f"sc{k}", (0, 0, 0))], c=c, fn=fn, params=params))
    rules = rules + extra
    read = {f for r in rules for f, _ in r["refs"]}
    goals = [r["out"] for r in rules if r["out"] not in read and not r["out"].startswith(("acc", "sc"))]
    return rules, axioms, goals


def to_spec_reduce(rules, axioms, goals):
    """DagSpec of random_reduce_dag's rules (scalars rank 0)."""
    from paper_1710_08774_gb300 import hfav as H
    D = H.DagSpec(2)
    for a in axioms:
        D.field(a)
    for r in rules:
        if r["out"].startswith(("acc", "sc")):
            D.field(r["out"], rank=0)
    for r in rules:
        refs = [(f, off[:2]) for f, off in r["refs"]]
        if "op" in r:
            D.rule("REDUCE_SUM" if r["op"] == "sum" else "REDUCE_MAX", refs, [r["out"]])
        else:
            D.rule("EXPR", refs, [r["out"]], params=r["params"], expr=r["c"])
    D.axiom(*axioms)
    D.goal(*goals)
    return D


def to_oracle_reduce(rules):
    return [(r["out"], r["refs"], r["op"], []) if "op" in r else (r["out"], r["refs"], r["fn"], r["params"])
            for r in rules]
