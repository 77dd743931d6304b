"""GPU path of the WCA pair forces (Sec. IV.A, Eq. WCA; cell list at q^{n+1/2}): per-step
parity with the oracle's all-pairs forces, and the equilibrium g(r) of the inertial
coupling dynamics against the Monte Carlo reference of tests/golden/wca_rdf_mc.txt."""
import os

import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm as oracle

from _gpu_helpers import TOL, compare_states, make_sim, read_oracle_state

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wca_rdf_mc.txt")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1212_6427_gb300 import build
    build.build_library()


def _cluster(grid, n, seed, centre, spacing, side):
    """n points in a cube of the given side around centre, no two closer than spacing
    (nearest image): many pairs inside the cut-off, none deep inside the core."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = np.mod(centre + rng.uniform(-0.5 * side, 0.5 * side, size=3), grid)
        ok = True
        for o in pts:
            d = p - o
            d -= grid * np.round(d / grid)
            ok &= np.sqrt((d * d).sum()) >= spacing
        if ok:
            pts.append(p)
    return np.array(pts)


WCA_CASES = [
    # (grid, n, kernel, seed, me_scale, eps, sigma, trap_k)
    ((16, 16, 16), 12, 4, 81, 1.0, 0.02, 1.6, 0.0),
    ((12, 18, 9), 8, 3, 82, 0.0, 0.05, 1.2, 0.0),         # few cells per axis
    ((32, 32, 16), 14, 4, 83, 1.0, 0.01, 1.8, 0.02),      # x passes with blob work; with the trap
]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", WCA_CASES, ids=[str(i) for i in range(len(WCA_CASES))])
def test_step_parity_with_wca(precision, case):
    grid, n, kernel, seed, me_scale, eps, sigma, k = case
    prm = oracle.Params(grid, kT=1e-3, dt=0.05, kernel=kernel, seed=seed, wca_epsilon=eps, wca_sigma=sigma,
                        trap_k=k, trap_center=(16.0, 16.0, 8.0))
    rng = np.random.default_rng(seed)
    q = _cluster(np.array(grid, float), n, seed, np.array([0.5, 1.0, 0.5]) * np.array(grid) - [0, 1.0, 0],
                 0.95 * sigma, 1.3 * sigma * n ** (1.0 / 3.0))
    st = oracle.State(wl.random_fluid(grid, 0.02, seed + 1), q, 0.01 * rng.standard_normal((n, 3)),
                      me_scale * rng.uniform(-0.5, 2.0, size=n), 0.005 * rng.standard_normal((n, 3)))
    tr = {}
    oracle.icm_step(st, prm, tr)
    assert np.abs(oracle.wca_force(tr["q_half"], prm)).max() > 1e-4     # the pair forces are active
    sim = make_sim(prm, st, precision)
    state = st
    worst = {}
    for _ in range(4):
        q_prev = state.q.copy()
        want = oracle.icm_step(state, prm)
        sim.write(state.q, state.u, state.v.ravel(), None if state.adv_prev is None else state.adv_prev.ravel(),
                  state.slip_g, state.step)
        sim.step(1)
        got, mom = read_oracle_state(sim, prm, state.me, state.force)
        err = compare_states(got, want, prm, q_prev)
        scale = prm.rho * prm.h ** 3 * np.abs(want.v).sum() + np.abs(want.me[:, None] * want.u).sum()
        err["P"] = float(np.abs(mom - oracle.total_momentum(want, prm)).max() / scale)
        for key, e in err.items():
            worst[key] = max(worst.get(key, 0.0), e)
        state = got
    sim.close()
    for key, e in worst.items():
        assert e < TOL[precision], (key, e, worst)


def test_wca_input_errors():
    import paper_1212_6427_gb300 as icm
    sim = icm.Simulation((16, 16, 16), kT=0.0, kernel=4, precision=64)
    with pytest.raises(icm.IcmError):
        sim.set_wca(-1.0, 1.0)
    with pytest.raises(icm.IcmError):
        sim.set_wca(1.0, 0.0)
    with pytest.raises(icm.IcmError):
        sim.set_wca(1.0, 8.0)          # cut-off 8.98 > half the box
    sim.set_wca(0.0, 1.0)
    sim.close()


def test_equilibrium_rdf_matches_monte_carlo():
    """Sec. IV.A, Fig. RDF (m_e = 0, Table tableRDF parameters, dt = 1): the g(r) of the
    dynamics agrees with Monte Carlo sampling of exp(-U/kT)."""
    from paper_1212_6427_gb300 import experiments
    ref = np.loadtxt(GOLDEN)
    res = experiments.rdf(steps=100000, burn=10000, sample_every=50)
    r, g = np.array(res["r"]), np.array(res["g"])
    np.testing.assert_allclose(r, ref[:, 0], atol=1e-9)
    sel = (r > 1.8) & (r < 7.9)
    # 100k steps hold ~10 decorrelated configurations: a few percent of noise per bin
    assert np.abs(g[sel] - ref[sel, 1]).max() < 0.12
    assert abs(g.max() - ref[:, 1].max()) < 0.08
    assert np.all(g[r < 1.5] == 0.0)
