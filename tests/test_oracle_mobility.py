"""Pins of the oracle's blob-grid operators of Sec. III.A.2 (translational invariance
of J P S, pair coupling J_i P S_j, single-blob mobility and hydrodynamic radius) and of
the Stokes limit (a = 0) of the spectral solve they use."""
import numpy as np
import pytest

from oracle import icm

from test_oracle_operators import _curl


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 12, 9)])
def test_stokes_solve_real_space_residual(shape):
    """a = 0: x = solve(r) iff D x = 0, mean(x) = 0 and r - mean(r) + eta L x is a
    gradient with zero mean (the mean mode has no solution and is dropped)."""
    h, eta = 0.9, 1.7
    r = np.random.default_rng(4).standard_normal((3,) + shape)
    x = icm.spectral_solve(r, 0.0, eta, h)
    scale = np.abs(r).max()
    assert np.abs(icm.divergence(x, h)).max() < 1e-12 * scale / h
    np.testing.assert_allclose(x.reshape(3, -1).mean(axis=1), 0.0, atol=1e-13 * scale)
    resid = r - r.reshape(3, -1).mean(axis=1)[:, None, None, None] + eta * icm.vector_laplacian(x, h)
    assert np.abs(_curl(resid, h)).max() < 1e-11 * scale
    np.testing.assert_allclose(resid.reshape(3, -1).mean(axis=1), 0.0, atol=1e-13 * scale)


def test_three_point_hydrodynamic_radius_matches_paper():
    """Sec. III.A.2: R_H ~ 0.91 dx for the three-point kernel (infinite system; here from
    the 32^3 periodic mobility with the lattice correction, averaged over positions)."""
    rng = np.random.default_rng(11)
    mus = [np.trace(icm.mobility(rng.uniform(0, 32, size=3), (32, 32, 32), 3, 1.0, 1.0)) / 3 for _ in range(4)]
    rh = icm.hydrodynamic_radius(np.mean(mus), 1.0, 32.0)
    assert rh == pytest.approx(0.91, rel=0.02)


def test_mobility_symmetric_and_nearly_isotropic():
    """-J L^-1 S is symmetric (J = dV_f S^T); off-diagonal terms are a small fraction."""
    mu = icm.mobility([3.3, 7.9, 11.2], (16, 16, 16), 4, 1.0, 1.0)
    np.testing.assert_allclose(mu, mu.T, rtol=0, atol=1e-14)
    assert np.abs(mu - np.diag(np.diag(mu))).max() < 0.01 * np.diag(mu).min()


@pytest.mark.parametrize("direction", [(1.0, 0.0, 0.0), (1.0, 1.0, 1.0)])
def test_pair_coupling_small_beyond_five_cells(direction):
    """Sec. III.A.2, Fig. JPS right (three-point kernel, 32^3): 3 dV J_i P S_j / 2 falls
    below 0.01 for l >~ 5 dx; at l = 0 it is ~I.  Beyond the supports it is the dipolar
    far field of P, ~ (3/2) dV 2 / (4 pi l^3) along the line of centres."""
    u = np.asarray(direction) / np.linalg.norm(direction)
    qj = np.array([9.3, 10.6, 12.1])
    dv = icm.blob_volume(3, 1.0)
    near = 1.5 * dv * icm.coupling_matrix(qj, qj, (32, 32, 32), 3, 1.0)
    assert np.abs(np.diag(near) - 1.0).max() < 0.05
    far = 1.5 * dv * icm.coupling_matrix(qj + 6.0 * u, qj, (32, 32, 32), 3, 1.0)
    assert np.abs(far).max() < 0.01
    assert np.abs(far).max() > 0.25 * 1.5 * dv * 2 / (4 * np.pi * 6.0 ** 3)


def test_disjoint_kernels_do_not_couple_without_projection():
    """J_i S_j = 0 exactly when the supports are disjoint (distance >= w cells along x)."""
    shape = (16, 16, 16)
    F = np.array([[1.0, -2.0, 0.5]])
    f = icm.spread(F, [[3.2, 5.0, 5.0]], 4, 1.0, shape)
    assert np.abs(icm.interpolate(f, [[7.3, 5.0, 5.0]], 4, 1.0)).max() == 0.0
    assert np.abs(icm.interpolate(f, [[5.9, 5.0, 5.0]], 4, 1.0)).max() > 0.0
