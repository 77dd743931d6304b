"""GPU path of the harmonic trap (the temporal accuracy test of Sec. III.D): per-step
parity with the oracle, and the error E(dt) of Eq. E_dt_definition on the GPU."""
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


TRAP_CASES = [
    # (grid, nblobs, kernel, seed, me_scale, trap_k, centre)
    ((16, 16, 16), 4, 4, 61, 1.0, 0.05, (8.0, 8.0, 8.0)),
    ((16, 12, 18), 3, 3, 62, 0.0, 0.2, (0.0, 11.5, 2.0)),
    ((32, 32, 16), 6, 4, 63, 1.0, 0.03, (31.0, 0.5, 8.0)),     # blob work inside the x passes
]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", TRAP_CASES, ids=[str(i) for i in range(len(TRAP_CASES))])
def test_step_parity_with_trap(precision, case):
    grid, nb, kernel, seed, me_scale, k, centre = case
    prm = oracle.Params(grid, kT=1e-3, dt=0.05, kernel=kernel, seed=seed, trap_k=k, trap_center=centre)
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


def _gpu_trajectory(dt, T, precision, me=0.0, k=0.01):
    import paper_1212_6427_gb300 as icm
    sim = icm.Simulation((16, 16, 16), 1.0, 1.0, 1.0, 0.0, dt, 4, 1, precision, 0)
    sim.add_blobs([[10.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]], [me])
    sim.set_forces([[0.0, 0.0, 0.0]])
    sim.set_trap(k, (0.0, 0.0, 0.0))
    out = []
    for _ in range(int(round(T / dt))):
        sim.step(1)
        out.append(sim.read()["pos"][0].copy())
    sim.close()
    return np.array(out)


def _e_dt(qa, qb, box=16.0):
    d = qa - qb[1::2]
    d -= box * np.round(d / box)
    return np.linalg.norm(d, axis=1).mean()


@pytest.mark.parametrize("precision", [64, 32])
def test_trap_error_second_order_on_gpu(precision):
    """Eq. E_dt_definition for a neutrally buoyant blob released from rest 10 cells from
    the centre (16^3, k = 0.01, kT = 0): the GPU's E(dt) falls ~4x per halving of dt and
    equals the oracle's."""
    T = 16.0
    dts = (1.0, 0.5, 0.25)
    q = {dt: _gpu_trajectory(dt, T, precision) for dt in dts}
    e = [_e_dt(q[a], q[b]) for a, b in zip(dts[:-1], dts[1:])]
    assert 3.2 < e[0] / e[1] < 4.8
    # the oracle's trajectories of the same setup
    def orc(dt):
        prm = oracle.Params((16, 16, 16), kT=0.0, dt=dt, kernel=4, trap_k=0.01)
        st = oracle.State(np.zeros((3, 16, 16, 16)), [[10.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]], [0.0], [[0.0, 0.0, 0.0]])
        out = []
        for _ in range(int(round(T / dt))):
            st = oracle.icm_step(st, prm)
            out.append(st.q[0].copy())
        return np.array(out)
    qo = {dt: orc(dt) for dt in dts}
    eo = [_e_dt(qo[a], qo[b]) for a, b in zip(dts[:-1], dts[1:])]
    tol = 1e-6 if precision == 64 else 5e-2
    np.testing.assert_allclose(e, eo, rtol=tol)


def test_trap_input_errors():
    import paper_1212_6427_gb300 as icm
    sim = icm.Simulation((16, 16, 16), kT=0.0, kernel=4, precision=64)
    with pytest.raises(icm.IcmError):
        sim.set_trap(-1.0, (0.0, 0.0, 0.0))
    with pytest.raises(icm.IcmError):
        sim.set_trap(1.0, (np.nan, 0.0, 0.0))
    sim.set_trap(0.0, (0.0, 0.0, 0.0))
    sim.close()
