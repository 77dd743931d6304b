"""Pins of the oracle's thermal drift forcing (Appendix B.2, Eq. thermal_drift): the
Peskin kernel derivatives, the drift field against finite differences of the pinned
spreading operator, and the conservation laws it keeps."""
import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm


@pytest.mark.parametrize("kernel", [3, 4])
def test_kernel_derivative_against_finite_differences(kernel):
    r = np.random.default_rng(1).uniform(-2.2, 2.2, size=4000)
    eps = 1e-6
    fd = (icm.phi(kernel, r + eps) - icm.phi(kernel, r - eps)) / (2 * eps)
    np.testing.assert_allclose(icm.dphi(kernel, r), fd, rtol=0, atol=2e-6)


@pytest.mark.parametrize("kernel", [3, 4])
def test_kernel_derivative_moment_rules(kernel):
    """d/dr of sum_k phi(r-k) = 1 and sum_k (r-k) phi(r-k) = 0: sum phi' = 0, sum (r-k) phi' = -1."""
    r = np.random.default_rng(2).uniform(0, 1, size=2000)[:, None] - np.arange(-3, 4)[None, :]
    d = icm.dphi(kernel, r)
    np.testing.assert_allclose(d.sum(axis=1), 0.0, atol=1e-14)
    np.testing.assert_allclose((r * d).sum(axis=1), -1.0, atol=1e-14)


@pytest.mark.parametrize("kernel", [3, 4])
def test_drift_field_is_the_position_derivative_of_the_spread(kernel):
    """Component a of the drift field = d/dq_a of component a of S(q) e_a."""
    shape, h = (10, 12, 9), 0.8
    rng = np.random.default_rng(kernel)
    q = rng.uniform(0, 1, size=(3, 3)) * np.array([9, 12, 10]) * h
    coef = np.array([0.7, -1.3, 2.0])
    got = icm.spread_drift(coef, q, kernel, h, shape)
    eps = 1e-6
    want = np.zeros_like(got)
    for a in range(3):
        F = np.zeros((3, 3))
        F[:, a] = coef
        dq = np.zeros(3)
        dq[a] = eps
        want[a] = (icm.spread(F, q + dq, kernel, h, shape)[a] - icm.spread(F, q - dq, kernel, h, shape)[a]) / (2 * eps)
    assert np.abs(got - want).max() < 1e-7 * np.abs(got).max()
    # and it integrates to zero (no net force)
    np.testing.assert_allclose(got.reshape(3, -1).sum(axis=1), 0.0, atol=1e-12 * np.abs(got).max())


def test_step_with_drift_conserves_momentum_and_changes_only_through_the_drift():
    grid = (12, 12, 12)
    rng = np.random.default_rng(9)
    q = wl.random_sequential_addition(4, grid, 1.0, 3.0, 9)
    st = icm.State(wl.random_fluid(grid, 0.02, 10), q, 0.01 * rng.standard_normal((4, 3)),
                   rng.uniform(-0.5, 2.0, size=4), np.zeros((4, 3)))
    on = icm.Params(grid, kT=1e-3, dt=0.05, thermal_drift=True)
    off = icm.Params(grid, kT=1e-3, dt=0.05, thermal_drift=False)
    p0 = icm.total_momentum(st, on)
    tr_on, tr_off = {}, {}
    s_on = icm.icm_step(st, on, tr_on)
    icm.icm_step(st, off, tr_off)
    np.testing.assert_allclose(icm.total_momentum(s_on, on), p0, rtol=0, atol=1e-14 * np.abs(st.v).sum())
    mtf = icm.fluid_dragged_mass(4, 1.0, 1.0)
    drift = icm.spread_drift(1e-3 * mtf / (mtf + st.me), tr_on["q_half"], 4, 1.0, (12, 12, 12))
    assert np.abs(drift).max() > 0
    np.testing.assert_allclose(tr_on["rhs"] - tr_off["rhs"], drift, rtol=0, atol=1e-15)
