"""GPU parity of the full ICM step (Sec. III.C) against the FP64 oracle, per step,
through the C ABI: the GPU state after each step is loaded into the oracle, which
advances one step from it, and every output (v, u, q, momentum) is compared."""
import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm as oracle

from _gpu_helpers import TOL, compare_states, make_sim, read_oracle_state, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1212_6427_gb300 import build
    build.build_library()


def _case(grid, nb, kernel, seed, me_scale=1.0, force=0.0, kT=1e-3, dt=0.05, vamp=0.05, slip="visc",
          advection=True, h=1.0):
    prm = oracle.Params(grid, h=h, rho=1.0, eta=1.0, kT=kT, dt=dt, kernel=kernel, seed=seed, slip=slip,
                        advection=advection)
    rng = np.random.default_rng(seed)
    q = wl.random_sequential_addition(nb, grid, h, 2.0 * h, seed)
    st = oracle.State(wl.random_fluid(grid, vamp, seed + 1), q, 0.05 * rng.standard_normal((nb, 3)),
                      me_scale * rng.uniform(-0.5, 2.0, size=nb), force * rng.standard_normal((nb, 3)))
    return prm, st


def _run_parity(prm, st0, precision, nsteps, plan=None):
    sim = make_sim(prm, st0, precision)
    if plan is not None:
        import paper_1212_6427_gb300 as icm
        icm.icm_set_plan(sim.handle, **plan)
    state = st0.copy()
    worst = {}
    for _ in range(nsteps):
        q_prev = state.q.copy()
        want = oracle.icm_step(state, prm)
        sim.write(state.q, state.u, state.v.ravel(), None if state.adv_prev is None else state.adv_prev.ravel(),
                  state.slip_g, state.step)
        sim.step(1)
        got, mom = read_oracle_state(sim, prm, state.me, state.force)
        err = compare_states(got, want, prm, q_prev)
        # momentum against its natural scale rho dV_f sum|v| + sum|m_e u| (P itself may be ~0)
        scale = prm.rho * prm.h ** 3 * np.abs(want.v).sum() + np.abs(want.me[:, None] * want.u).sum()
        err["P"] = float(np.abs(mom - oracle.total_momentum(want, prm)).max() / scale)
        for k, e in err.items():
            worst[k] = max(worst.get(k, 0.0), e)
        assert got.step == want.step
        state = got      # continue from the GPU's own state
    sim.close()
    return worst


CASES = [
    # (grid, nblobs, kernel, seed, me_scale, force, kT, slip, advection)
    ((16, 16, 16), 6, 4, 11, 1.0, 0.05, 1e-3, "visc", True),
    ((16, 16, 16), 6, 3, 12, 1.0, 0.0, 1e-3, "zero", True),
    ((24, 16, 12), 5, 3, 13, 1.0, 0.02, 0.0, "full", True),
    ((32, 12, 18), 9, 4, 14, 0.0, 0.05, 1e-3, "visc", True),      # neutrally buoyant: steps 4-8 skipped
    ((9, 18, 16), 4, 4, 15, 2.0, 0.01, 5e-3, "visc", False),
    ((16, 16, 16), 0, 4, 16, 1.0, 0.0, 1e-3, "visc", True),       # fluid only
    # x sides with register FFT passes: the blob work runs inside the x passes
    ((32, 32, 16), 8, 4, 17, 1.0, 0.05, 1e-3, "visc", True),      # Ny % 32 == 0: one z plane per row block
    ((32, 64, 8), 10, 3, 20, 1.0, 0.03, 1e-3, "visc", True),      # 3-point, 7-node span on an 8-node side
    ((48, 24, 12), 7, 3, 18, 1.0, 0.02, 1e-3, "full", True),      # row blocks straddle z planes
    ((64, 12, 9), 6, 4, 19, 2.0, 0.0, 2e-3, "zero", True),        # several z planes per row block
    ((96, 32, 12), 9, 4, 22, 1.0, 0.04, 0.0, "visc", False),
    # dense: ~150 blob tasks per row block, past the staged records of an x-pass block
    ((32, 32, 16), 600, 4, 23, 1.0, 0.02, 1e-3, "visc", True),
    ((64, 32, 8), 800, 3, 24, 1.0, 0.02, 1e-3, "full", True),     # ~300 per block: past the inverse pass too
    # Nx = Ny: run with the x and y forward passes fused on clusters of Ny/32 blocks (FP32)
    ((64, 64, 8), 20, 4, 25, 1.0, 0.02, 1e-3, "visc", True),
    ((128, 128, 8), 30, 3, 26, 1.0, 0.02, 1e-3, "full", True),
    ((256, 256, 8), 40, 4, 27, 1.0, 0.02, 1e-3, "visc", True),
]
SEAM = {6, 7, 8, 9, 13}    # cases that also put blobs on the periodic seams and corners
XY = {13, 14, 15}          # cases stepped with the fused x-y plan


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_step_parity(precision, case):
    grid, nb, kernel, seed, me_scale, force, kT, slip, adv = case
    prm, st = _case(grid, nb, kernel, seed, me_scale, force, kT, slip=slip, advection=adv)
    if CASES.index(case) in SEAM:
        L = np.array(grid, dtype=float) * prm.h
        st.q[0] = [0.0, 0.0, 0.0]
        st.q[1] = L - 0.3 * prm.h
        st.q[2] = [0.5 * prm.h, L[1] - 0.25 * prm.h, 1e-12]
        st.q[3] = [L[0] - 0.5 * prm.h, 0.5 * prm.h, L[2] - 0.5 * prm.h]
    plan = dict(fused_xy=1) if CASES.index(case) in XY else None
    worst = _run_parity(prm, st, precision, nsteps=4, plan=plan)
    for k, e in worst.items():
        assert e < TOL[precision], (k, e, worst)


@pytest.mark.parametrize("precision", [64, 32])
def test_plain_config_100_steps(precision):
    """The 32^3 FP64 plain configuration (one neutral blob, 4-point kernel), every step."""
    w = wl.workload("plain")
    prm = oracle.Params(w["grid"], h=w["h"], rho=w["rho"], eta=w["eta"], kT=w["kT"], dt=w["dt"],
                        kernel=w["kernel"], seed=w["seed"])
    st = oracle.State(np.zeros((3, 32, 32, 32)), w["q"], w["u"], w["me"], w["force"])
    worst = _run_parity(prm, st, precision, nsteps=100 if precision == 64 else 20)
    for k, e in worst.items():
        assert e < TOL[precision], (k, e, worst)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("grid", [(24, 24, 24), (32, 32, 24)])
def test_momentum_conservation_and_impulse(precision, grid):
    prm, st = _case(grid, 12, 4, 21, 1.0, 0.0, kT=1e-3)
    st.v += 0.01      # a nonzero total momentum
    sim = make_sim(prm, st, precision)
    p0 = sim.read()["momentum"]
    sim.step(20)
    p1 = sim.read()["momentum"]
    assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(p0).max()
    # with forces: P^{n+1} - P^n = dt sum F
    F = np.random.default_rng(5).standard_normal((12, 3)) * 0.01
    sim.set_forces(F)
    sim.step(10)
    p2 = sim.read()["momentum"]
    np.testing.assert_allclose(p2 - p1, 10 * prm.dt * F.sum(axis=0), rtol=1e-10, atol=1e-13 * np.abs(p1).max())
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_no_slip_exact_for_neutral_blobs(precision):
    import paper_1212_6427_gb300 as icm
    grid = (16, 16, 16)
    prm, st = _case(grid, 5, 4, 31, me_scale=0.0, force=0.05)
    sim = make_sim(prm, st, precision)
    sim.step(3)
    r = sim.read(fluid=True)
    # u^{n+1} = J^{n+1/2} v^{n+1}; q^{n+1/2} is not exported, so check through the oracle's
    # predictor from the state one step earlier
    sim.write(r["pos"], r["vel"], r["fluid"], None, None, r["step"])
    tr = {}
    stp = oracle.State(r["fluid"].reshape((3, 16, 16, 16)), r["pos"], r["vel"], st.me, st.force, None, None, r["step"])
    oracle.icm_step(stp, prm, tr)
    sim.step(1)
    r2 = sim.read(fluid=True)
    ju = icm.icm_op_interpolate(sim.handle, tr["q_half"], r2["fluid"])
    assert rel(r2["vel"], ju) < 10 * TOL[precision]
    sim.close()


def test_cfl_violation_is_reported():
    import paper_1212_6427_gb300 as icm
    grid = (16, 16, 16)
    prm, st = _case(grid, 2, 4, 41, me_scale=0.0)
    st.v[0] += 30.0          # |u| dt / h = 1.5
    sim = make_sim(prm, st, 64)
    sim.step(1)
    with pytest.raises(icm.IcmError) as ei:
        sim.sync()
    assert ei.value.status == icm.ICM_ECFL
    sim.close()


def test_invalid_blob_input():
    import paper_1212_6427_gb300 as icm
    sim = icm.Simulation((16, 16, 16), kT=0.0, kernel=3, precision=32)
    with pytest.raises(icm.IcmError):
        sim.add_blobs([[1.0, 2.0, 3.0]], None, [-13.0])      # m_e <= -m~_f = -12
    with pytest.raises(icm.IcmError):
        sim.add_blobs([[np.nan, 2.0, 3.0]], None, [0.0])
    with pytest.raises(icm.IcmError):
        sim.add_blobs([[1.0, 2.0, 3.0]], [[30.0, 0.0, 0.0]], [0.0])   # |u| dt / h > 1
    sim.add_blobs([[1.0, 2.0, 3.0]], None, [0.5])
    assert icm.icm_num_blobs(sim.handle) == 1
    sim.close()


def test_checkpoint_resume_matches_uninterrupted_run():
    grid = (16, 16, 16)
    prm, st = _case(grid, 6, 4, 51, 1.0, 0.02)
    a = make_sim(prm, st, 64)
    a.step(6)
    ra = a.read(fluid=True)
    b = make_sim(prm, st, 64)
    b.step(3)
    r = b.read(fluid=True)
    adv, g, hist = b.read_aux()
    b.close()
    c = make_sim(prm, st, 64)
    c.write(r["pos"], r["vel"], r["fluid"], adv if hist else None, g, r["step"])
    c.step(3)
    rc = c.read(fluid=True)
    assert rc["step"] == ra["step"] == 6
    assert rel(rc["fluid"], ra["fluid"]) < 1e-13
    assert rel(rc["pos"], ra["pos"]) < 1e-15
    assert rel(rc["vel"], ra["vel"]) < 1e-12
    a.close()
    c.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_bulk_config_sampled_parity(precision):
    """The 128^3 bulk configuration (2000 blobs, 3-point kernel, dt = 0.02) for 1000
    steps; at each of the first 10 steps and then every 100th, the GPU's state is
    loaded into the oracle, advanced one step, and compared with the GPU's next state."""
    w = wl.workload("bulk")
    prm = oracle.Params(w["grid"], h=w["h"], rho=w["rho"], eta=w["eta"], kT=w["kT"], dt=w["dt"],
                        kernel=w["kernel"], seed=w["seed"])
    st0 = oracle.State(np.zeros((3,) + prm.shape), w["q"], w["u"], w["me"], w["force"])
    sim = make_sim(prm, st0, precision)
    nsteps = w["steps"]
    samples = sorted(set(range(10)) | set(range(100, nsteps, 100)))
    worst = {}
    n = 0
    for s in samples:
        if s > n:
            sim.step(s - n)
        cur, _ = read_oracle_state(sim, prm, w["me"], w["force"])
        assert cur.step == s
        want = oracle.icm_step(cur, prm)
        sim.step(1)
        got, mom = read_oracle_state(sim, prm, w["me"], w["force"])
        err = compare_states(got, want, prm, cur.q)
        scale = prm.rho * prm.h ** 3 * np.abs(want.v).sum() + np.abs(want.me[:, None] * want.u).sum()
        err["P"] = float(np.abs(mom - oracle.total_momentum(want, prm)).max() / scale)
        for k, e in err.items():
            worst[k] = max(worst.get(k, 0.0), e)
        n = s + 1
    sim.step(nsteps - n)
    assert sim.read()["step"] == nsteps
    sim.close()
    for k, e in worst.items():
        assert e < TOL[precision], (k, e, worst)
