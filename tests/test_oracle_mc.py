"""Pins of the Monte Carlo reference sampler (oracle/mc_wca.c) used for the equilibrium
radial distribution function of Sec. IV.A: g(r) = 1 for an ideal gas, and
g(r) -> exp(-V(r)/kT) at low density (the exact zero-density limit)."""
import numpy as np

from oracle import mc


def _wca(r, sigma, eps):
    rc = 2.0 ** (1.0 / 6.0) * sigma
    s6 = (sigma / r) ** 6
    return np.where(r < rc, 4.0 * eps * (s6 * s6 - s6) + eps, 0.0)


def test_ideal_gas_is_uniform():
    r, g, _ = mc.wca_rdf(200, (12.0, 12.0, 12.0), 1.0, 0.0, 1.0, 1500, 100, 5, 11, 0.25, 5.0)
    sel = r > 1.0
    assert np.abs(g[sel] - 1.0).max() < 0.08
    assert abs(g[sel].mean() - 1.0) < 0.02


def test_low_density_limit_is_the_boltzmann_factor():
    sigma, eps, kT = 2.0, 1.0, 1.0
    r, g, acc = mc.wca_rdf(64, (20.0, 20.0, 20.0), sigma, eps, kT, 20000, 500, 2, 12, 0.1, 6.0)
    want = np.exp(-_wca(r, sigma, eps) / kT)
    sel = (r > 1.85) & (r < 3.0)
    assert 0.1 < acc < 0.9
    np.testing.assert_allclose(g[sel], want[sel], atol=0.08)
    assert np.all(g[r < 1.6] == 0.0)
