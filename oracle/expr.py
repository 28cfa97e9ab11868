"""Plain numpy FP64 evaluation of a DAG of user rules (test infrastructure
only: like the rest of this package, only the tests, the smoke check and the
benchmark's CPU legs may import it; it shares no code with the CUDA path).

A rule is a side-effect-free kernel that reads fields at relative offsets and
writes one field at offset 0 (Sec. 3.1).  The DAG is the dataflow between
rules (Sec. 3.2): a rule runs once every field it reads exists.  Here each
rule runs over the whole periodic grid at once,

    out[x] = f(in_0[x + o_0], in_1[x + o_1], ..., p_0, p_1, ...),

with no fusion, footprint or contraction: on a periodic grid every field is
periodic, so the full-grid evaluation is the plain definition of what a fused
nest with halos computes (fusion and contraction do not change values, Sec.
3.1).  For grids whose halo the caller gives, `evaluate_padded` evaluates on
the padded array and crops: a cell of the interior depends only on cells
within the DAG's footprint, which the halo covers, so the wrap at the padded
array's edge never reaches it.

Parity: pinned by tests/test_oracle_expr.py -- brute force with explicit
modular indices on tiny grids, Fourier eigenmodes of a Laplacian rule, order
independence and the DAG errors, and agreement with the separately pinned C
oracle of the 2D chain.
"""
import numpy as np


def shifted(a, off):
    """The field a read at offset off = (di, dj, dk): a[x + off], periodically.

    a is laid out (..., j, i) with i the last numpy axis."""
    nd = a.ndim
    out = a
    for axis, o in enumerate(tuple(off)[:nd]):
        if o:
            out = np.roll(out, -int(o), axis=nd - 1 - axis)
    return out


def evaluate(rules, axioms, halo=0):
    """Run a DAG of rules to completion.

    rules:  list of (out, refs, fn, params): out a field name, refs a list of
            (field, offset) read in this order, fn(*inputs, *params) -> array.
            fn may instead be the string "sum" or "max": a reduction (Sec.
            3.4) of its one input over the whole grid to a scalar.  Scalars
            read by a grid rule take the same value at every cell (a
            broadcast); offsets on them are ignored.
    axioms: dict field -> array (..., j, i); every other field is produced by
            exactly one rule.
    halo:   with halo-padded axioms (see evaluate_padded), the reductions run
            over the interior only.
    Returns a dict with every field (axioms included) as an FP64 array
    (0-d for scalars)."""
    vals = {k: np.asarray(v, dtype=np.float64) for k, v in axioms.items()}
    outs = [r[0] for r in rules]
    if len(set(outs)) != len(outs) or set(outs) & set(vals):
        raise ValueError("a field has two producers")
    pending = list(range(len(rules)))
    while pending:
        ready = [r for r in pending if all(f in vals for f, _ in rules[r][1])]
        if not ready:
            raise ValueError("the rules read a field nothing produces, or form a cycle")
        for r in ready:
            out, refs, fn, params = rules[r]
            ins = [shifted(vals[f], off) for f, off in refs]
            if isinstance(fn, str):
                red = {"sum": np.sum, "max": np.max}[fn]
                a = ins[0][tuple(slice(halo, n - halo) for n in ins[0].shape)] if halo else ins[0]
                vals[out] = np.asarray(red(a), dtype=np.float64)
                continue
            # the output has the shape of the largest input (a grid rule that
            # reads scalars, or ignores its inputs, still yields a field)
            shape = max((a.shape for a in ins), key=len)
            vals[out] = np.broadcast_to(np.asarray(fn(*ins, *params), dtype=np.float64), shape).copy()
        pending = [r for r in pending if r not in ready]
    return vals


def evaluate_padded(rules, axioms_padded, halo, fields):
    """The given fields on the interior of halo-padded axioms (halo given by
    the caller, not periodic): evaluate on the padded arrays, crop `halo`
    cells off every axis; reductions run over the interior.  Exact when the
    halo covers the DAG's footprint."""
    vals = evaluate(rules, axioms_padded, halo)
    crop = lambda a: a[tuple(slice(halo, s - halo) for s in a.shape)]
    return {f: crop(vals[f]) for f in fields}


def chain2d_rules():
    """The synthetic three-stage 2D chain (5-point Laplacian L, half gradient
    magnitude G of L, squash out = G / (1 + G)) as rule bodies."""
    lap = ("L", [("u", (1, 0)), ("u", (-1, 0)), ("u", (0, 1)), ("u", (0, -1)), ("u", (0, 0))],
           lambda a, b, c, d, e, p0: a + b + c + d - p0 * e, [4.0])
    grad = ("G", [("L", (1, 0)), ("L", (-1, 0)), ("L", (0, 1)), ("L", (0, -1))],
            lambda a, b, c, d: np.sqrt((a - b) * (a - b) + (c - d) * (c - d)) * 0.5, [])
    squash = ("out", [("G", (0, 0))], lambda g: g / (1 + g), [])
    return [lap, grad, squash]


def normalization_rules():
    """The normalization example (Sec. 5.2) in the reading taken here: flux =
    u(i+1) - u(i), diff = flux(i) - flux(i-1), the norm accumulation acc =
    sum of diff^2 over the grid, the norm root = sqrt(acc), out = diff / root."""
    return [
        ("flux", [("u", (1, 0)), ("u", (0, 0))], lambda a, b: a - b, []),
        ("diff", [("flux", (0, 0)), ("flux", (-1, 0))], lambda a, b: a - b, []),
        ("sq", [("diff", (0, 0))], lambda a: a * a, []),
        ("acc", [("sq", (0, 0))], "sum", []),
        ("root", [("acc", (0, 0))], lambda a: np.sqrt(a), []),
        ("out", [("diff", (0, 0)), ("root", (0, 0))], lambda a, b: a / b, []),
    ]
