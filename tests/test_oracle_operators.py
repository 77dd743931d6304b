"""Pins of the oracle's staggered operators, FFT solves, advection and noise.

The checks use properties the mathematics fixes rather than the oracle's own
formulas: adjointness, exact Fourier eigenvalues, an FFT-independent real-space
residual of the Helmholtz/projection solve (divergence-free + curl-free residual),
conservation laws of the advection operator (Sec. II.B: conservative in momentum
and energy), its continuum limit, and published Philox known answers.
"""
import os

import numpy as np
import pytest

from oracle import icm, philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dot(a, b):
    return float(np.sum(a * b))


def test_gradient_is_minus_divergence_transpose():
    rng = np.random.default_rng(1)
    shape = (6, 7, 8)
    v = rng.standard_normal((3,) + shape)
    p = rng.standard_normal(shape)
    h = 0.3
    assert _dot(icm.divergence(v, h), p) == pytest.approx(-_dot(v, icm.gradient(p, h)), rel=1e-13)


def test_div_grad_is_cell_laplacian():
    rng = np.random.default_rng(2)
    p = rng.standard_normal((6, 5, 8))
    np.testing.assert_allclose(icm.divergence(icm.gradient(p, 0.5), 0.5), icm.laplacian(p, 0.5), atol=1e-11)


def test_laplacian_fourier_eigenvalue():
    n = (8, 12, 6)    # Nx, Ny, Nz
    h = 0.4
    kvec = (3, 5, 1)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    phase = 2 * np.pi * (kvec[0] * i / n[0] + kvec[1] * j / n[1] + kvec[2] * k / n[2])
    f = np.cos(phase)
    lam = -sum(4 * np.sin(np.pi * kvec[a] / n[a]) ** 2 for a in range(3)) / h ** 2
    np.testing.assert_allclose(icm.laplacian(f, h), lam * f, atol=1e-11)


def _curl(w, h):
    """Edge-centred discrete curl of a face field (zero iff w is a discrete gradient + const)."""
    out = []
    for a, b in ((0, 1), (0, 2), (1, 2)):
        out.append((w[b] - icm.shift(w[b], a, -1)) / h - (w[a] - icm.shift(w[a], b, -1)) / h)
    return np.stack(out)


@pytest.mark.parametrize("ab", [(20.0, 0.5), (1.0, 0.0), (1.0, 0.025)])
@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 12, 9)])
def test_spectral_solve_real_space_residual(ab, shape):
    """x = solve(r) iff D x = 0, and r - (a - b L) x is a gradient with zero mean.

    On the periodic MAC grid a face field with zero curl and zero mean is a discrete
    gradient, so these three conditions fix x uniquely, independently of any FFT.
    """
    a, b = ab
    h = 0.9
    rng = np.random.default_rng(3)
    r = rng.standard_normal((3,) + shape)
    x = icm.spectral_solve(r, a, b, h)
    scale = np.abs(r).max()
    assert np.abs(icm.divergence(x, h)).max() < 1e-12 * scale / h
    resid = r - (a * x - b * icm.vector_laplacian(x, h))
    assert np.abs(_curl(resid, h)).max() < 1e-11 * scale
    np.testing.assert_allclose(resid.reshape(3, -1).mean(axis=1), 0.0, atol=1e-13 * scale)


def test_naive_dft_closed_forms():
    """The plain DFT sums: a delta at the origin transforms to all ones, a constant to
    N at k = 0 only, a single plane wave to N at its own wave vector; and idft3 undoes
    dft3 on random data (sides 8, 6 and 12 and a mixed grid)."""
    for shape in ((8, 8, 8), (6, 6, 6), (12, 12, 12), (6, 8, 12)):
        n = int(np.prod(shape))
        delta = np.zeros(shape)
        delta[0, 0, 0] = 1.0
        np.testing.assert_allclose(icm.dft3(delta), np.ones(shape), atol=1e-13)
        const = icm.dft3(np.ones(shape))
        assert const[0, 0, 0] == pytest.approx(n, rel=1e-13)
        const[0, 0, 0] = 0.0
        assert np.abs(const).max() < 1e-10
        kz, ky, kx = 1, shape[1] - 2, 3 % shape[2]
        z, y, x = np.indices(shape)
        wave = np.exp(2j * np.pi * (kz * z / shape[0] + ky * y / shape[1] + kx * x / shape[2]))
        spec = icm.dft3(wave)
        assert spec[kz, ky, kx] == pytest.approx(n, rel=1e-12)
        spec[kz, ky, kx] = 0.0
        assert np.abs(spec).max() < 1e-9
        rng = np.random.default_rng(n)
        f = rng.standard_normal(shape)
        np.testing.assert_allclose(icm.idft3(icm.dft3(f)).real, f, atol=1e-12)


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 6, 6), (12, 12, 12), (6, 8, 12)])
def test_fft_solve_equals_naive_dft_solve(shape):
    """numpy's FFT, the library transform of the oracle's solves, against the plain
    O(N^2) DFT sums, through the whole Helmholtz / projection solve on 8^3, 6^3 and 12^3
    grids (radix 2 and 3) and a mixed one."""
    rng = np.random.default_rng(5)
    r = rng.standard_normal((3,) + shape)
    for a, b in ((20.0, 0.5), (1.0, 0.0), (0.0, 0.8)):
        want = icm.spectral_solve_dft(r, a, b, 0.9)
        np.testing.assert_allclose(icm.spectral_solve(r, a, b, 0.9), want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_projection_is_orthogonal_projector():
    rng = np.random.default_rng(4)
    shape = (6, 8, 10)
    u = rng.standard_normal((3,) + shape)
    w = rng.standard_normal((3,) + shape)
    pu = icm.spectral_solve(u, 1.0, 0.0, 1.0)
    pw = icm.spectral_solve(w, 1.0, 0.0, 1.0)
    np.testing.assert_allclose(icm.spectral_solve(pu, 1.0, 0.0, 1.0), pu, atol=1e-12)
    assert _dot(pu, w) == pytest.approx(_dot(u, pw), rel=1e-12)
    # the mean flow is left alone (P = I at k = 0)
    np.testing.assert_allclose(pu.reshape(3, -1).mean(1), u.reshape(3, -1).mean(1), atol=1e-14)


def test_advection_conserves_momentum():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((3, 7, 8, 9))
    a = icm.advection(v, 1.3, 0.6)
    np.testing.assert_allclose(a.reshape(3, -1).sum(axis=1), 0.0, atol=1e-11)


def test_advection_conserves_energy_for_divergence_free_fields():
    """Skew-adjointness (Sec. II.B): sum v . A(v) = 0 when D v = 0."""
    rng = np.random.default_rng(6)
    v = icm.spectral_solve(rng.standard_normal((3, 8, 10, 12)), 1.0, 0.0, 1.0)
    a = icm.advection(v, 1.0, 1.0)
    assert abs(_dot(v, a)) < 1e-12 * np.sqrt(_dot(a, a) * _dot(v, v))


def test_advection_continuum_limit_second_order():
    """A -> div(v v^T) for a smooth field; error falls ~4x per halving of h."""
    L = 2 * np.pi
    errs = []
    for n in (16, 32):
        h = L / n
        k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        v = np.zeros((3, n, n, n))
        exact = np.zeros_like(v)
        for c in range(3):
            off = icm.component_offsets(c)
            x, y, z = (i + off[0]) * h, (j + off[1]) * h, (k + off[2]) * h
            # v = (sin y + cos z, sin z + cos x, sin x + cos y): divergence free
            if c == 0:
                v[c] = np.sin(y) + np.cos(z)
                vy, vz = np.sin(z) + np.cos(x), np.sin(x) + np.cos(y)
                exact[c] = vy * np.cos(y) - vz * np.sin(z)          # v . grad v_x
            elif c == 1:
                v[c] = np.sin(z) + np.cos(x)
                vx, vz = np.sin(y) + np.cos(z), np.sin(x) + np.cos(y)
                exact[c] = -vx * np.sin(x) + vz * np.cos(z)
            else:
                v[c] = np.sin(x) + np.cos(y)
                vx, vy = np.sin(y) + np.cos(z), np.sin(z) + np.cos(x)
                exact[c] = vx * np.cos(x) - vy * np.sin(y)
        errs.append(np.abs(icm.advection(v, 1.0, h) - exact).max())
    assert errs[1] < errs[0] / 3.5


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        vals = [int(x, 16) for x in row]
        got = philox.philox4x32(vals[0:4], vals[4:6])
        assert [int(x) for x in got] == vals[6:10]


def test_stress_normals_moments_and_independence():
    plane = 500   # 400 planes of 500 cells
    z = philox.stress_normals(seed=77, step=3, ncell=200_000, plane=plane)
    assert z.shape == (6, 200_000)
    np.testing.assert_allclose(z.mean(axis=1), 0.0, atol=0.01)
    np.testing.assert_allclose(z.var(axis=1), 1.0, atol=0.01)
    c = np.corrcoef(z)
    assert np.abs(c - np.eye(6)).max() < 0.01
    # fourth moment of a unit normal is 3
    np.testing.assert_allclose((z ** 4).mean(axis=1), 3.0, atol=0.06)
    # the off-diagonal normals of planes 2m and 2m + 1 (one Philox call) are uncorrelated
    zz = z.reshape(6, 400, plane)
    for a in (4, 5):
        for b in (4, 5):
            r = np.corrcoef(zz[a, 0::2].ravel(), zz[b, 1::2].ravel())[0, 1]
            assert abs(r) < 0.01, (a, b, r)
    # a new step or seed gives new numbers
    assert not np.allclose(z, philox.stress_normals(seed=77, step=4, ncell=200_000, plane=plane))
    assert not np.allclose(z, philox.stress_normals(seed=78, step=3, ncell=200_000, plane=plane))


def test_stress_normals_counter_layout():
    """The normals are Box-Muller pairs of the Philox words of the counters the layout
    names, recomputed here for single cells from the generator (pinned by the Random123
    known-answer vectors): call 0 at (cell, step, 0, 0) gives (Z_xx, Z_yy) and (Z_zz,
    Z_xy); call 1 at (cell of plane 2m, step, 1, 0) gives (Z_xz, Z_yz) of that cell from
    words 0-1 and of the cell above it (plane 2m + 1) from words 2-3.  Five planes of
    4 x 5 cells: cells on even and odd planes and on the last, unpaired, plane."""
    nx, ny, nz = 4, 5, 5
    plane, ncell, seed, step = nx * ny, nx * ny * nz, (1 << 33) + 9, 21
    z = philox.stress_normals(seed, step, ncell, plane)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for cell in (0, 3, 27, 39, 45, 61, 99):
        k = cell // plane
        a = [int(w) for w in philox.philox4x32((cell, step, 0, 0), key)]
        b = [int(w) for w in philox.philox4x32((cell - (k % 2) * plane, step, 1, 0), key)]
        pair = b[2:4] if k % 2 else b[0:2]
        want = list(philox.box_muller(np.array([a[0]]), np.array([a[1]])))
        want += list(philox.box_muller(np.array([a[2]]), np.array([a[3]])))
        want += list(philox.box_muller(np.array([pair[0]]), np.array([pair[1]])))
        np.testing.assert_array_equal(z[:, cell], np.concatenate(want))
    # the pairs of a call: plane 1's off-diagonal normals are not plane 0's
    assert not np.allclose(z[4:, plane:2 * plane], z[4:, :plane])


def test_box_muller_special_values():
    # word 0xffffffff is u = 1 - 2^-33: radius ~ sqrt(2^-32); word 0 for the angle gives cos ~ 1
    c, s = philox.box_muller(np.array([0xFFFFFFFF]), np.array([0]))
    assert c[0] == pytest.approx(np.sqrt(2 * 2.0 ** -33), rel=1e-6)
    assert abs(s[0]) < 1e-13


def test_stochastic_flux_is_divergence_of_symmetric_stress():
    """Discrete Gauss theorem: the flux divergence sums to zero over the box."""
    z = philox.stress_normals(seed=5, step=0, ncell=6 * 7 * 8, plane=7 * 8)
    f = icm.stochastic_flux_divergence(z, 0.7, 0.5, (6, 7, 8))
    np.testing.assert_allclose(f.reshape(3, -1).sum(axis=1), 0.0, atol=1e-11)
