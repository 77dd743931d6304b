"""GPU parity of the step with the thermal drift forcing (Appendix B.2, Eq.
thermal_drift, ICM_FLAG_THERMAL_DRIFT) against the oracle, per step."""
import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm as oracle

from _gpu_helpers import TOL, compare_states, make_sim, read_oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1212_6427_gb300 import build
    build.build_library()


DRIFT_CASES = [
    # (grid, nblobs, kernel, seed, me_scale, kT)
    ((16, 16, 16), 5, 4, 71, 1.0, 2e-3),
    ((12, 18, 9), 4, 3, 72, 0.0, 5e-3),
    ((32, 32, 16), 8, 4, 73, 1.0, 1e-3),     # blob work inside the x passes
    ((48, 24, 12), 6, 3, 74, 1.0, 1e-3),
]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", DRIFT_CASES, ids=[str(i) for i in range(len(DRIFT_CASES))])
def test_step_parity_with_thermal_drift(precision, case):
    grid, nb, kernel, seed, me_scale, kT = case
    prm = oracle.Params(grid, kT=kT, dt=0.05, kernel=kernel, seed=seed, thermal_drift=True)
    rng = np.random.default_rng(seed)
    q = wl.random_sequential_addition(nb, grid, 1.0, 2.0, seed)
    st = oracle.State(wl.random_fluid(grid, 0.05, seed + 1), q, 0.05 * rng.standard_normal((nb, 3)),
                      me_scale * rng.uniform(-0.5, 2.0, size=nb), 0.01 * rng.standard_normal((nb, 3)))
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


def test_drift_flag_changes_the_step_only_with_noise():
    """With kT = 0 the flag is a no-op (the drift is proportional to kT)."""
    import paper_1212_6427_gb300 as icm
    grid = (16, 16, 16)
    q = wl.random_sequential_addition(4, grid, 1.0, 2.0, 5)
    out = []
    for flags in (0, icm.FLAG_THERMAL_DRIFT):
        sim = icm.Simulation(grid, 1.0, 1.0, 1.0, 0.0, 0.05, 4, 1, 64, flags)
        sim.add_blobs(q, None, [0.0, 1.0, 2.0, 0.5])
        sim.set_forces(np.full((4, 3), 0.01))
        sim.step(3)
        out.append(sim.read(fluid=True))
        sim.close()
    np.testing.assert_array_equal(out[0]["pos"], out[1]["pos"])
    np.testing.assert_array_equal(out[0]["fluid"], out[1]["fluid"])
