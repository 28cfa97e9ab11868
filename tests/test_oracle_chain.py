"""Pins of the oracle's stencil chains (CPU only).

oracle.chain2d: pinned by (1) the exact discrete Laplacian of integer
quadratics (L = 2a + 2b bitwise, so G = out = 0), (2) cubics (L = 6i, G = 6,
out = 6/7 exactly), (3) the periodic sine closed form, (4) brute force with
np.roll on 8x8 and 13x7 grids.
oracle.chain3d: pinned by quadratics (out = 0), u = i^5 (s1 = 20i^3 + 10i,
s2 = 120 i, s3 = 120, out = 120/121) and np.roll brute force.
"""
import numpy as np
import pytest

import oracle
from paper_1710_08774_gb300 import inputs as I


def _grid2(nx, ny):
    j, i = np.meshgrid(np.arange(-2, ny + 2), np.arange(-2, nx + 2), indexing="ij")
    return i.astype(np.float64), j.astype(np.float64)


@pytest.mark.parametrize("coef", [(1, 2, 3, 4, 5, 6), (-3, 7, 0, 1, -2, 9), (5, -4, -6, 0, 0, 1)])
def test_chain2d_quadratic_exact(coef):
    a, b, c, d, e, f = coef
    i, j = _grid2(13, 9)
    u = a * i * i + b * j * j + c * i * j + d * i + e * j + f
    L, G, out = oracle.chain2d(u, periodic=False)
    assert np.all(L == 2 * a + 2 * b)
    assert np.all(G == 0.0) and np.all(out == 0.0)


def test_chain2d_cubic_exact():
    i, j = _grid2(11, 7)
    L, G, out = oracle.chain2d(i ** 3, periodic=False)
    ii = np.arange(-1, 12, dtype=np.float64)
    assert np.all(L == 6.0 * ii[None, :])
    assert np.all(G == 6.0) and np.all(out == 6.0 / 7.0)
    # two-axis cubic: L = 6i + 6j, G = 6 sqrt(2)
    L, G, out = oracle.chain2d(i ** 3 + j ** 3, periodic=False)
    assert np.allclose(G, 6.0 * np.sqrt(2.0), rtol=0, atol=1e-13)
    assert np.allclose(out, 6 * np.sqrt(2) / (1 + 6 * np.sqrt(2)), rtol=0, atol=1e-15)


@pytest.mark.parametrize("N,k", [(32, 1), (64, 3), (40, 7)])
def test_chain2d_periodic_sine_closed_form(N, k):
    th = 2 * np.pi * k / N
    ii = np.arange(N)
    interior = np.tile(np.sin(th * ii), (N, 1))
    u = I.pad(interior, 2)          # NaN halo: periodic mode must not read it
    L, G, out = oracle.chain2d(u, periodic=True)
    Lx = (2 * np.cos(th) - 2) * np.sin(th * ii)
    assert np.allclose(L[1:-1, 1:-1], Lx[None, :], rtol=0, atol=1e-14)
    Gx = abs(2 * np.cos(th) - 2) * np.abs(np.cos(th * ii)) * np.sin(th)
    assert np.allclose(G, Gx[None, :], rtol=0, atol=1e-14)
    assert np.allclose(out, Gx / (1 + Gx), rtol=0, atol=1e-14)


@pytest.mark.parametrize("nx,ny", [(8, 8), (13, 7)])
def test_chain2d_bruteforce_roll(nx, ny):
    u = I.chain2d_input(nx, seed=5, ny=ny)
    c = u[2:-2, 2:-2]
    r = lambda a, dj, di: np.roll(np.roll(a, -dj, axis=0), -di, axis=1)   # a(i+di, j+dj)
    L = r(c, 0, 1) + r(c, 0, -1) + r(c, 1, 0) + r(c, -1, 0) - 4 * c
    G = np.hypot(r(L, 0, 1) - r(L, 0, -1), r(L, 1, 0) - r(L, -1, 0)) / 2
    _, Go, out = oracle.chain2d(u, periodic=True)
    assert np.allclose(Go, G, rtol=1e-14, atol=1e-14)
    assert np.allclose(out, G / (1 + G), rtol=1e-14, atol=1e-15)


def _grid3(n):
    k, j, i = np.meshgrid(*(np.arange(-3, n + 3),) * 3, indexing="ij")
    return i.astype(np.float64), j.astype(np.float64), k.astype(np.float64)


def test_chain3d_quadratic_zero():
    i, j, k = _grid3(6)
    u = 3 * i * i - 2 * j * j + k * k + 4 * i * j - k * i + 7 * j + 2
    assert np.all(oracle.chain3d(u, periodic=False) == 0.0)


def test_chain3d_quintic_exact():
    i, j, k = _grid3(7)
    out = oracle.chain3d(i ** 5, periodic=False)
    assert np.all(out == 120.0 / 121.0)


def test_chain3d_bruteforce_roll():
    n = 9
    u = I.chain3d_input(n, seed=11)
    c = u[3:-3, 3:-3, 3:-3]

    def lap(a):
        s = -6 * a
        for ax in range(3):
            s = s + np.roll(a, 1, axis=ax) + np.roll(a, -1, axis=ax)
        return s
    s2 = lap(lap(c))
    g2 = sum((np.roll(s2, -1, axis=ax) - np.roll(s2, 1, axis=ax)) ** 2 for ax in range(3))
    s3 = np.sqrt(g2) / 2
    out = oracle.chain3d(u, periodic=True)
    assert np.allclose(out, s3 / (1 + s3), rtol=1e-13, atol=1e-14)


def test_neighbourhood_block_gives_the_whole_domain_value():
    """The full-size GPU tests check sampled cells against the oracle run on
    each cell's periodic neighbourhood (radius 3 in 3D, 2 in 2D).  That block
    fixes the cell: on small grids it reproduces the whole-domain oracle."""
    from tests.test_gpu_chain import _block_wrap, _sample_points
    u = I.chain3d_input(20, seed=4)
    full = oracle.chain3d(u)
    interior = u[3:-3, 3:-3, 3:-3]
    for p in _sample_points(20, 3, 20, 1):
        b = oracle.chain3d(np.pad(_block_wrap(interior, p, 3), 3))[3, 3, 3]
        assert abs(b - full[tuple(p)]) <= 1e-14 * max(1.0, abs(full[tuple(p)]))
    u2 = I.chain2d_input(24, seed=0)
    _, _, f2 = oracle.chain2d(u2)
    interior2 = u2[2:-2, 2:-2]
    for p in _sample_points(24, 2, 30, 2):
        assert oracle.chain2d(np.pad(_block_wrap(interior2, p, 2), 2))[2][2, 2] == f2[tuple(p)]
