"""Pins of the COSMO horizontal-diffusion oracle (Sec. 5.3) against closed forms.

* A periodic Fourier mode u = sin(w i) sin(v j) is an eigenfunction of every
  stage: the discrete Laplacian gives -(lx + ly) u with lx = 4 sin^2(w/2),
  ly = 4 sin^2(v/2); each flux is -(lx + ly) times the difference of u across
  its face, so flux * du <= 0 and the limiter never acts; the update gives
  out = (1 - c (lx + ly)^2) u.  A dropped term, a wrong sign or a shifted
  face index changes that factor.
* u = i^4 (halo given) makes every flux_x counter-gradient (flux and du have
  the same sign), so the limiter zeroes all of them and out = u exactly; the
  unlimited value would be u - 24 c.
* u = j^4 does the same to every flux_y, the limiter along j; the
  unlimited value would again be u - 24 c.
* Quadratics have a constant Laplacian, hence zero fluxes and out = u exactly.
* Periodic data: the update is in flux form, so the sum over a plane is
  conserved (to rounding).
* No dependency in k: planes are computed on their own.
"""
import numpy as np

import oracle
from paper_1710_08774_gb300 import inputs as I


def padded(core, halo=2):
    """(nz, ny, nx) interior -> (nz+4, ny+4, nx+4) with a NaN halo (periodic mode must not read it)."""
    nz, ny, nx = core.shape
    u = np.full((nz + 2 * halo, ny + 2 * halo, nx + 2 * halo), np.nan)
    u[halo:halo + nz, halo:halo + ny, halo:halo + nx] = core
    return u


def test_fourier_mode_is_an_eigenfunction():
    nx, ny, nz, c = 48, 40, 2, 0.03
    for mx, my in ((1, 0), (0, 3), (5, 2), (11, 7)):
        w, v = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
        j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        # a mode with no wave along an axis is constant (1) along it
        ui = np.sin(w * i) if mx else np.ones_like(i, dtype=float)
        uj = np.sin(v * j) if my else np.ones_like(j, dtype=float)
        core = np.broadcast_to(ui * uj, (nz, ny, nx)).copy()
        lam = 4 * np.sin(w / 2) ** 2 + 4 * np.sin(v / 2) ** 2
        lap, flx, fly, out = oracle.cosmo(padded(core), c)
        assert np.max(np.abs(lap[:, 1:-1, 1:-1] + lam * core)) <= 1e-12
        assert np.max(np.abs(out - (1 - c * lam * lam) * core)) <= 1e-12


def test_limiter_zeroes_counter_gradient_fluxes():
    nx, ny, nz, c = 20, 6, 1, 0.1
    k, j, i = np.meshgrid(np.arange(-2, nz + 2), np.arange(-2, ny + 2), np.arange(-2, nx + 2), indexing="ij")
    u = (i.astype(np.float64)) ** 4
    lap, flx, fly, out = oracle.cosmo(u, c, periodic=False)
    assert np.all(lap[:, 1:-1, 1:-1] == 12.0 * (np.arange(nx) ** 2) + 2.0)
    assert np.all(flx == 0.0) and np.all(fly == 0.0)
    assert np.all(out == u[2:-2, 2:-2, 2:-2])


def test_limiter_zeroes_counter_gradient_fluxes_in_j():
    nx, ny, nz, c = 7, 18, 2, 0.1
    k, j, i = np.meshgrid(np.arange(-2, nz + 2), np.arange(-2, ny + 2), np.arange(-2, nx + 2), indexing="ij")
    u = (j.astype(np.float64)) ** 4
    lap, flx, fly, out = oracle.cosmo(u, c, periodic=False)
    assert np.all(lap[:, 1:-1, 1:-1] == (12.0 * (np.arange(ny) ** 2) + 2.0)[None, :, None])
    assert np.all(flx == 0.0) and np.all(fly == 0.0)
    assert np.all(out == u[2:-2, 2:-2, 2:-2])


def test_quadratics_give_zero_fluxes():
    nx, ny, nz, c = 17, 13, 2, 0.2
    k, j, i = np.meshgrid(np.arange(-2, nz + 2), np.arange(-2, ny + 2), np.arange(-2, nx + 2), indexing="ij")
    u = 3.0 * i * i - 2.0 * j * j + 5.0 * i * j + i - 7.0 * j + 11.0 + k
    lap, flx, fly, out = oracle.cosmo(u, c, periodic=False)
    assert np.all(lap == 2.0)
    assert np.all(flx == 0.0) and np.all(fly == 0.0)
    assert np.all(out == u[2:-2, 2:-2, 2:-2])


def test_periodic_planes_conserve_their_sum():
    u = I.cosmo_input(64, 48, 3, seed=5)
    _, _, _, out = oracle.cosmo(u, 0.05)
    for k in range(3):
        a = u[k + 2, 2:-2, 2:-2]
        assert abs(out[k].sum() - a.sum()) <= 1e-12 * np.abs(a).sum()
    # and the limiter did act somewhere on this input
    _, flx, _, _ = oracle.cosmo(u, 0.05)
    assert np.any(flx == 0.0) and np.any(flx != 0.0)


def test_planes_are_independent():
    u = I.cosmo_input(24, 20, 4, seed=6)
    _, _, _, out = oracle.cosmo(u, 0.05)
    perm = [2, 0, 3, 1]
    v = u.copy()
    v[2:-2] = u[2:-2][perm]
    _, _, _, out2 = oracle.cosmo(v, 0.05)
    assert np.array_equal(out2, out[perm])


def test_neighbourhood_block_gives_the_whole_domain_value():
    """The full-size GPU test checks sampled cells against the oracle run on
    each cell's periodic 5 x 5 neighbourhood in its plane: that block fixes the
    cell (the composed stencil reaches two cells in i and j)."""
    from tests.test_gpu_chain import _block_wrap, _sample_points
    u = I.cosmo_input(24, 20, 2, seed=3)
    full = oracle.cosmo(u, 0.05)[3]
    for kq in range(2):
        plane = u[kq + 2, 2:-2, 2:-2]
        for p in _sample_points(20, 2, 25, 4):
            blk = _block_wrap(plane, p, 2)[None]
            assert oracle.cosmo(np.pad(blk, 2), 0.05)[3][0, 2, 2] == full[kq][tuple(p)]
