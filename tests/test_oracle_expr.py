"""The expression-DAG oracle (oracle/expr.py) pinned by facts outside itself.

- Brute force: random DAGs on tiny 2D and 3D grids against a loop over cells
  with explicit modular indices (pins the direction of every offset and the
  order of evaluation).
- Closed form: the 5-point Laplacian rule on a Fourier mode sin(w i) sin(v j)
  gives -(4 sin^2(w/2) + 4 sin^2(v/2)) times the mode; applied twice, the
  square of that eigenvalue.
- Order independence (rules are order agnostic, Sec. 3.1) and the DAG errors
  (two producers, a missing input, a cycle).
- The 2D chain written as three rule bodies equals the C oracle of the chain,
  itself pinned separately.
- Reductions and broadcasts: sums and maxima with closed forms (a constant,
  the index i, a full period of a sine), brute force with a loop, and the
  normalization example's invariants (unit 2-norm, invariance under scaling
  and shifting u, the second difference of a quadratic).
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import expr as E
from tests import expr_dags as X


def _brute(rules, axioms, shape):
    vals = {k: np.asarray(v, dtype=np.float64) for k, v in axioms.items()}
    nd = len(shape)
    for r in rules:   # generated in dependency order
        out = np.empty(shape)
        for cell in itertools.product(*[range(n) for n in shape]):
            # cell is (..., j, i); offsets are (di, dj, dk)
            ins = []
            for f, off in r["refs"]:
                src = tuple((cell[a] + off[nd - 1 - a]) % shape[a] for a in range(nd))
                ins.append(vals[f][src])
            out[cell] = r["fn"](*ins, *r["params"])
        vals[r["out"]] = out
    return vals


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(4, 5), (3, 4, 5)])
def test_brute_force_tiny_grids(seed, shape):
    nd = len(shape)
    rules, axioms, goals = X.random_dag(nd, 5, seed)
    ax = X.axiom_values(axioms, shape, seed + 100)
    got = E.evaluate(X.to_oracle(rules), ax)
    ref = _brute(rules, ax, shape)
    for g in goals:
        assert np.allclose(got[g], ref[g], rtol=0, atol=1e-14)


def _lap_rule(src, out):
    return (out, [(src, (1, 0)), (src, (-1, 0)), (src, (0, 1)), (src, (0, -1)), (src, (0, 0))],
            lambda a, b, c, d, e: a + b + c + d - 4 * e, [])


def test_laplacian_eigenmode_and_its_square():
    ny, nx = 24, 40
    w, v = 2 * np.pi * 3 / nx, 2 * np.pi * 5 / ny
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    mode = np.sin(w * i) * np.sin(v * j)
    lam = 4 * np.sin(w / 2) ** 2 + 4 * np.sin(v / 2) ** 2
    vals = E.evaluate([_lap_rule("u", "l1"), _lap_rule("l1", "l2")], {"u": mode})
    assert np.max(np.abs(vals["l1"] + lam * mode)) < 1e-13
    assert np.max(np.abs(vals["l2"] - lam * lam * mode)) < 1e-12


def test_offsets_read_the_named_neighbour():
    """x[i + 1] at i is the next column: on u = i the rule in0 - in1 with refs
    (+1, 0), (0, 0) is 1 except at the wrap, where it is 1 - n."""
    ny, nx = 3, 7
    u = np.broadcast_to(np.arange(nx, dtype=float), (ny, nx))
    d = E.evaluate([("d", [("u", (1, 0)), ("u", (0, 0))], lambda a, b: a - b, [])], {"u": u})["d"]
    assert np.all(d[:, :-1] == 1) and np.all(d[:, -1] == 1 - nx)
    dj = E.evaluate([("d", [("u", (0, -1)), ("u", (0, 0))], lambda a, b: a - b, [])], {"u": u.T.copy()})["d"]
    assert np.all(dj[1:, :] == -1) and np.all(dj[0, :] == nx - 1)


def test_order_independent_and_dag_errors():
    rules, axioms, goals = X.random_dag(2, 6, 3)
    ax = X.axiom_values(axioms, (9, 11), 1)
    a = E.evaluate(X.to_oracle(rules), ax)
    b = E.evaluate(X.to_oracle(rules)[::-1], ax)
    for g in goals:
        assert np.array_equal(a[g], b[g])
    one = ("o", [("u", (0, 0))], lambda x: x, [])
    with pytest.raises(ValueError):
        E.evaluate([one, one], {"u": np.zeros((3, 3))})
    with pytest.raises(ValueError):
        E.evaluate([("o", [("missing", (0, 0))], lambda x: x, [])], {"u": np.zeros((3, 3))})
    with pytest.raises(ValueError):
        E.evaluate([("a", [("b", (0, 0))], lambda x: x, []), ("b", [("a", (0, 0))], lambda x: x, [])],
                   {"u": np.zeros((3, 3))})


def test_chain_as_rule_bodies_equals_c_oracle():
    rng = np.random.default_rng(5)
    ny, nx = 20, 33
    core = rng.uniform(-1, 1, (ny, nx))
    up = np.pad(core, 2, mode="wrap")
    ref = oracle.chain2d(up)[2]
    got = E.evaluate(E.chain2d_rules(), {"u": core})["out"]
    assert np.max(np.abs(got - ref)) < 1e-14


def test_reductions_closed_forms():
    ny, nx = 12, 20
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    u = i.astype(float)
    v = E.evaluate([("s", [("u", (0, 0))], "sum", []), ("m", [("u", (0, 0))], "max", []),
                    ("c", [("u", (0, 0))], lambda a: 0 * a + 2.5, []), ("sc", [("c", (0, 0))], "sum", []),
                    ("w", [("u", (1, 0))], lambda a: np.sin(2 * np.pi * a / nx), []), ("sw", [("w", (0, 0))], "sum", [])],
                   {"u": u})
    assert v["s"] == ny * nx * (nx - 1) / 2 and v["m"] == nx - 1
    assert v["sc"] == 2.5 * nx * ny
    assert abs(v["sw"]) < 1e-12
    assert v["s"].shape == () and v["w"].shape == (ny, nx)


def test_broadcast_and_reduction_brute_force():
    rng = np.random.default_rng(11)
    ny, nx = 4, 5
    u = rng.uniform(-1, 1, (ny, nx))
    rules = [("d", [("u", (1, 0)), ("u", (0, -1))], lambda a, b: a - 2 * b, []),
             ("m", [("d", (0, 1))], "max", []), ("s", [("d", (-1, 0))], "sum", []),
             ("k", [("m", (0, 0)), ("s", (0, 0))], lambda a, b: a * b + 1, []),
             ("o", [("d", (0, 0)), ("k", (0, 0)), ("u", (-1, 1))], lambda a, b, c: a * b - c, [])]
    got = E.evaluate(rules, {"u": u})
    d = np.array([[u[jj, (ii + 1) % nx] - 2 * u[(jj - 1) % ny, ii] for ii in range(nx)] for jj in range(ny)])
    m = max(d[(jj + 1) % ny, ii] for jj in range(ny) for ii in range(nx))
    s = sum(d[jj, (ii - 1) % nx] for jj in range(ny) for ii in range(nx))
    k = m * s + 1
    o = np.array([[d[jj, ii] * k - u[(jj + 1) % ny, (ii - 1) % nx] for ii in range(nx)] for jj in range(ny)])
    assert got["m"] == m and abs(got["s"] - s) < 1e-13 and np.allclose(got["o"], o, rtol=0, atol=1e-13)


def test_normalization_invariants():
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, (16, 24))
    out = E.evaluate(E.normalization_rules(), {"u": u})["out"]
    assert abs(np.sum(out * out) - 1) < 1e-13
    for v in (7.5 * u, u + 3.0):
        assert np.allclose(E.evaluate(E.normalization_rules(), {"u": v})["out"], out, rtol=0, atol=1e-13)
    # u = i^2 along i (periodic wrap aside): the second difference is 2 in the interior columns
    q = np.broadcast_to((np.arange(24.0) ** 2), (16, 24)).copy()
    diff = E.evaluate(E.normalization_rules(), {"u": q})["diff"]
    assert np.all(diff[:, 1:-1] == 2)


def test_padded_evaluation_reduces_over_the_interior():
    """Halo-given grids: the reduction sees only the interior (the halo holds
    a value that would change every sum); the broadcast reaches every cell."""
    rng = np.random.default_rng(5)
    core = rng.uniform(-1, 1, (6, 9))
    pad = np.pad(core, 2, constant_values=100.0)
    rules = [("s", [("u", (0, 0))], "sum", []), ("o", [("u", (0, 0)), ("s", (0, 0))], lambda a, b: a - b, [])]
    got = E.evaluate_padded(rules, {"u": pad}, 2, ["o"])["o"]
    assert np.allclose(got, core - core.sum(), rtol=0, atol=1e-13)
