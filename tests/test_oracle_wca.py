"""Pins of the oracle's WCA pair forces (Sec. IV.A, Eq. WCA): the force is minus the
gradient of the pair energy (finite differences), the potential and force vanish at
the cut-off 2^(1/6) sigma, pairs obey Newton's third law, and the step conserves
momentum with them."""
import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm


def _prm(**kw):
    return icm.Params((12, 10, 14), wca_epsilon=0.7, wca_sigma=1.6, **kw)


def _cluster(seed, n=12):
    rng = np.random.default_rng(seed)
    # a loose cluster that straddles the periodic seam: many pairs inside the cut-off
    return np.mod(rng.uniform(-2.5, 2.5, size=(n, 3)) + [0.5, 9.5, 7.0], [12.0, 10.0, 14.0])


def test_force_is_minus_gradient_of_the_energy():
    prm = _prm()
    q = _cluster(1)
    f = icm.wca_force(q, prm)
    assert np.abs(f).max() > 1e-2
    eps = 1e-6
    for i in range(q.shape[0]):
        for a in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, a] += eps
            qm[i, a] -= eps
            fd = -(icm.wca_energy(qp, prm) - icm.wca_energy(qm, prm)) / (2 * eps)
            assert f[i, a] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(f).max())


def test_newton_third_law_and_cutoff():
    prm = _prm()
    f = icm.wca_force(_cluster(2, 20), prm)
    np.testing.assert_allclose(f.sum(axis=0), 0.0, atol=1e-13 * np.abs(f).max())
    rc = 2.0 ** (1.0 / 6.0) * 1.6
    for r in (rc * (1 - 1e-9), rc * (1 + 1e-9)):
        pair = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        assert np.abs(icm.wca_force(pair, prm)).max() < 1e-7
        assert icm.wca_energy(pair, prm) < 1e-8
    # at r = sigma: V = eps, |F| = 24 eps / sigma
    pair = np.array([[1.0, 1.0, 1.0], [2.6, 1.0, 1.0]])
    assert icm.wca_energy(pair, prm) == pytest.approx(0.7, rel=1e-12)
    assert icm.wca_force(pair, prm)[0, 0] == pytest.approx(-24 * 0.7 / 1.6, rel=1e-12)


def test_step_with_wca_conserves_momentum():
    grid = (12, 10, 14)
    prm = icm.Params(grid, kT=1e-3, dt=0.05, wca_epsilon=1e-2, wca_sigma=1.6)
    q = _cluster(3, 10)
    rng = np.random.default_rng(3)
    st = icm.State(wl.random_fluid(grid, 0.02, 4), q, 0.01 * rng.standard_normal((10, 3)),
                   rng.uniform(-0.5, 2.0, size=10), np.zeros((10, 3)))
    tr = {}
    st1 = icm.icm_step(st, prm, tr)
    assert np.abs(tr["force_half"]).max() > 1e-3
    p0, p1 = icm.total_momentum(st, prm), icm.total_momentum(st1, prm)
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-15 + 1e-13 * np.abs(tr["force_half"]).max())
