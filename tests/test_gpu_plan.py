"""Execution plans (icm_plan) and the autotuner: every plan choice gives the oracle's
step (parity per step), tuning leaves the state untouched, and a tuned plan is shared
by simulations with the same key."""
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


PLANS = [
    dict(fused_blobs=1, tma_z=1, rhs_kz=16, fork=1, fused_xy=1, z_split=0),
    dict(fused_blobs=0, tma_z=1, rhs_kz=16, fork=1, fused_xy=1, z_split=0),   # separate blob kernels, fused-capable side
    dict(fused_blobs=1, tma_z=0, rhs_kz=8, fork=0, fused_xy=0, z_split=0),    # one block per z tile, short RHS march
    dict(fused_blobs=0, tma_z=0, rhs_kz=32, fork=0, fused_xy=0, z_split=0),
    dict(fused_blobs=1, tma_z=1, rhs_kz=0, fork=1, fused_xy=0, z_split=0),    # persistent RHS blocks
    dict(fused_blobs=1, tma_z=1, rhs_kz=4, fork=1, fused_xy=0, z_split=0),
    dict(fused_blobs=1, tma_z=1, rhs_kz=0, fork=1, fused_xy=0, z_split=1),    # the other z split, TMA z pass
    dict(fused_blobs=1, tma_z=0, rhs_kz=16, fork=1, fused_xy=0, z_split=1),   # the other z split, plain z pass
]


def _case(grid, nb, seed):
    prm = oracle.Params(grid, kT=1e-3, dt=0.05, kernel=4, seed=seed)
    rng = np.random.default_rng(seed)
    q = wl.random_sequential_addition(nb, grid, 1.0, 2.0, seed)
    st = oracle.State(wl.random_fluid(grid, 0.05, seed + 1), q, 0.05 * rng.standard_normal((nb, 3)),
                      rng.uniform(-0.5, 2.0, size=nb), 0.01 * rng.standard_normal((nb, 3)))
    return prm, st


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("plan", PLANS, ids=[str(i) for i in range(len(PLANS))])
@pytest.mark.parametrize("grid", [(32, 32, 48), (24, 16, 64), (16, 24, 96), (16, 8, 256)])
def test_every_plan_matches_the_oracle(precision, plan, grid):
    import paper_1212_6427_gb300 as icm
    prm, st = _case(grid, 10, 91)
    sim = make_sim(prm, st, precision)
    icm.icm_set_plan(sim.handle, **plan)
    assert icm.icm_get_plan(sim.handle) == plan
    state = st
    worst = {}
    for _ in range(3):
        q_prev = state.q.copy()
        want = oracle.icm_step(state, prm)
        sim.write(state.q, state.u, state.v.ravel(), None if state.adv_prev is None else state.adv_prev.ravel(),
                  state.slip_g, state.step)
        sim.step(1)
        got, mom = read_oracle_state(sim, prm, state.me, state.force)
        err = compare_states(got, want, prm, q_prev)
        for key, e in err.items():
            worst[key] = max(worst.get(key, 0.0), e)
        state = got
    sim.close()
    for key, e in worst.items():
        assert e < TOL[precision], (key, e, worst, plan)


def test_autotune_keeps_the_state_and_shares_its_plan():
    import paper_1212_6427_gb300 as icm
    prm, st = _case((32, 32, 48), 10, 92)
    sim = make_sim(prm, st, 32)
    sim.step(2)
    before = sim.read(fluid=True)
    plan, ms = icm.icm_autotune(sim.handle, 2)
    assert ms > 0 and (plan["rhs_kz"] == 0 or 4 <= plan["rhs_kz"] <= 64)
    after = sim.read(fluid=True)
    for k in ("pos", "vel", "fluid", "momentum"):
        np.testing.assert_array_equal(before[k], after[k])
    assert before["step"] == after["step"]
    assert icm.icm_get_plan(sim.handle) == plan
    # a new simulation with the same key takes the tuned plan when it captures its step
    other = make_sim(prm, st, 32)
    other.step(1)
    assert icm.icm_get_plan(other.handle) == plan
    sim.close()
    other.close()


def test_plan_input_errors():
    import paper_1212_6427_gb300 as icm
    sim = icm.Simulation((16, 16, 16), kT=0.0, kernel=4, precision=64)
    with pytest.raises(icm.IcmError):
        icm.icm_set_plan(sim.handle, rhs_kz=2)
    with pytest.raises(icm.IcmError):
        icm.icm_autotune(sim.handle, 0)
    sim.close()
