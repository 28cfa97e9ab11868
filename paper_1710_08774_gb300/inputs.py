"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module holds no arithmetic of the method: it only draws numbers and lays
out initial states.  Neither the oracle nor the CUDA library imports it; the
tests and bench.py call it and hand the arrays to both sides.

Random numbers: counter-based SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; output mixer of Vigna's
splitmix64).  Value n of stream s under seed k is
    mix(base(k, s) + (n + 1) * GOLDEN),  base(k, s) = mix(mix(k + GOLDEN) ^ (s * GOLDEN))
and a uniform double in [0, 1) is (value >> 11) * 2**-53.  Normals use the
Box-Muller transform on two consecutive uniforms.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
GAMMA = 1.4


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _base(seed, stream):
    with np.errstate(over="ignore"):
        k = _mix(np.array([np.uint64(seed) + GOLDEN], dtype=np.uint64))
        s = np.array([np.uint64(stream)], dtype=np.uint64) * GOLDEN
        return _mix(k ^ s)[0]


def uniform(seed, stream, n, offset=0):
    """n uniforms in [0, 1) from counters offset .. offset+n-1 of (seed, stream)."""
    ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(_base(seed, stream) + ctr * GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed, stream, n):
    """n standard normals via Box-Muller on uniform pairs (2k, 2k+1)."""
    u = uniform(seed, stream, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def chain2d_input(n=256, seed=0, halo=2, ny=None, fill_halo=np.nan):
    """u ~ U[0,1) on an n x ny interior inside a (ny+2h, n+2h) FP64 array.

    The halo is filled with ``fill_halo`` (NaN by default): with periodic
    boundaries nothing may read it."""
    ny = n if ny is None else ny
    u = np.full((ny + 2 * halo, n + 2 * halo), fill_halo, dtype=np.float64)
    u[halo:halo + ny, halo:halo + n] = uniform(seed, 0, n * ny).reshape(ny, n)
    return u


def chain3d_input(n=64, seed=4, halo=3, dtype=np.float64, fill_halo=np.nan):
    """u ~ N(0,1) on an n^3 interior inside an (n+2h)^3 array (interior at h)."""
    u = np.full((n + 2 * halo,) * 3, fill_halo, dtype=dtype)
    u[halo:halo + n, halo:halo + n, halo:halo + n] = normal(seed, 0, n ** 3).reshape(n, n, n)
    return u


def cosmo_input(nx, ny, nz, seed=7, halo=2, dtype=np.float64, fill_halo=np.nan):
    """u ~ U[0,1) on an nx x ny x nz interior inside an (nz+2h, ny+2h, nx+2h)
    array (interior at h); the COSMO diffusion reads no k neighbours, the k
    halo only keeps one halo width for every axis."""
    u = np.full((nz + 2 * halo, ny + 2 * halo, nx + 2 * halo), fill_halo, dtype=dtype)
    u[halo:halo + nz, halo:halo + ny, halo:halo + nx] = uniform(seed, 0, nx * ny * nz).reshape(nz, ny, nx)
    return u


def sod_state(nx, ny, seed=1, grid=0, perturb=0.01, gamma=GAMMA):
    """Sod-like conserved state (4, ny, nx) FP64 on [0,1] x [0, ny/nx], dx = 1/nx.

    Cells with centre x < 0.5 get (rho, p) = (1, 1), the rest (0.125, 0.1);
    then rho *= 1 + perturb*xi1, p *= 1 + perturb*xi2, u = perturb*xi3,
    v = perturb*xi4 with xi ~ U[-1, 1) drawn per (seed, grid, field, cell).
    perturb = 0 gives the plain Sod states at rest."""
    x = (np.arange(nx, dtype=np.float64) + 0.5) / nx
    left = np.broadcast_to(x < 0.5, (ny, nx))
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    n = nx * ny
    xi = [2.0 * uniform(seed, grid * 16 + f, n).reshape(ny, nx) - 1.0 for f in range(4)]
    rho = rho * (1.0 + perturb * xi[0])
    p = p * (1.0 + perturb * xi[1])
    u = perturb * xi[2]
    v = perturb * xi[3]
    U = np.empty((4, ny, nx), dtype=np.float64)
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return U


def batch_sides(n_grids=64, seed=3, lo=128, hi=2048, multiple=4):
    """Grid sides (nx, ny), each independently ~ U{lo..hi}, rounded down to a multiple."""
    u = uniform(seed, 1000, 2 * n_grids)
    s = lo + np.floor(u * (hi - lo + 1)).astype(np.int64)
    s = np.maximum(lo, (s // multiple) * multiple)
    return [(int(s[2 * g]), int(s[2 * g + 1])) for g in range(n_grids)]


def pad(a, halo, fill=np.nan, pitch_multiple=1):
    """Place an interior array into a halo-padded array (last axis optionally pitch-rounded)."""
    shape = [s + 2 * halo for s in a.shape]
    if pitch_multiple > 1:
        shape[-1] = -(-shape[-1] // pitch_multiple) * pitch_multiple
    out = np.full(shape, fill, dtype=a.dtype)
    sl = tuple(slice(halo, halo + s) for s in a.shape)
    out[sl] = a
    return out
