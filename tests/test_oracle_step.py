"""Pins of the oracle's full ICM step (Sec. III.C) against what the paper fixes.

* exact conservation of total fluid + blob momentum without external force, and
  P^{n+1} - P^n = dt sum F with it (Sec. II; Appendix C, Eq. dv_eq_modified);
* the no-slip constraint u^{n+1} = J^{n+1/2} v^{n+1} exactly for m_e = 0 and
  a slip of O(m_e dt^2) otherwise (Appendix C, after Eq. u_np1_modified);
* second-order temporal accuracy for neutrally buoyant blobs (Sec. III.D);
* fluctuation-dissipation: equilibrium variance of the fluid, exact for any dt
  (Sec. III, the fluid solver of the scheme), and of a passive blob, (kT/rho) J P S;
* J P S ~ (2/3) dV^-1 I within a few percent (Sec. III.A.2, Fig. JPS);
* the harmonic trap of the temporal accuracy test (Sec. III.D): the force at
  q^{n+1/2} against hand values, its impulse, and the second-order decay of the
  error E(dt) of Eq. E_dt_definition for a neutrally buoyant blob.
"""
import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm


def _prm(grid, **kw):
    return icm.Params(grid, **kw)


def _state(grid, nb, seed, me_scale=1.0, vamp=0.05, force=0.0, kernel=4):
    rng = np.random.default_rng(seed)
    q = wl.random_sequential_addition(nb, grid, 1.0, 3.0, seed)
    u = 0.05 * rng.standard_normal((nb, 3))
    me = me_scale * rng.uniform(-0.5, 2.0, size=nb)
    F = force * rng.standard_normal((nb, 3))
    v = wl.random_fluid(grid, vamp, seed + 1)
    return icm.State(v, q, u, me, F)


@pytest.mark.parametrize("slip", ["visc", "full", "zero"])
def test_momentum_conserved_without_force(slip):
    grid = (12, 10, 14)
    prm = _prm(grid, kT=1e-3, dt=0.1, kernel=4, seed=9, slip=slip)
    st = _state(grid, 6, 21)
    p0 = icm.total_momentum(st, prm)
    assert np.abs(p0).max() > 1e-3      # a non-trivial momentum to conserve
    for _ in range(4):
        st = icm.icm_step(st, prm)
        np.testing.assert_allclose(icm.total_momentum(st, prm), p0, rtol=0, atol=1e-13 * np.abs(p0).max() * 50)


def test_momentum_change_equals_impulse_of_force():
    grid = (10, 12, 10)
    prm = _prm(grid, kT=0.0, dt=0.07, kernel=3)
    st = _state(grid, 5, 31, force=0.3)
    for _ in range(3):
        p0 = icm.total_momentum(st, prm)
        st2 = icm.icm_step(st, prm)
        np.testing.assert_allclose(icm.total_momentum(st2, prm) - p0, prm.dt * st.force.sum(axis=0), atol=1e-13)
        st = st2


def test_no_slip_exact_for_neutral_blobs():
    grid = (10, 10, 12)
    prm = _prm(grid, kT=1e-3, dt=0.05, kernel=4)
    st = _state(grid, 4, 41, me_scale=0.0, force=0.1)
    trace = {}
    st2 = icm.icm_step(st, prm, trace)
    np.testing.assert_allclose(st2.u, icm.interpolate(st2.v, trace["q_half"], 4, 1.0), atol=1e-15)


def test_fluid_divergence_free_after_step():
    grid = (9, 12, 8)
    prm = _prm(grid, kT=1e-2, dt=0.05, kernel=3)
    st = _state(grid, 3, 51)
    st2 = icm.icm_step(st, prm)
    assert np.abs(icm.divergence(st2.v, 1.0)).max() < 1e-13 * np.abs(st2.v).max()


def _run_to(T, dt, st, prm_kw, grid):
    prm = _prm(grid, dt=dt, **prm_kw)
    n = int(round(T / dt))
    st = st.copy()
    for _ in range(n):
        st = icm.icm_step(st, prm)
    return st


def test_second_order_in_time_for_neutral_blob():
    """Deterministic, m_e = 0: a pulled blob's position error shrinks ~4x per halving of dt."""
    grid = (16, 16, 16)
    st = icm.State(np.zeros((3, 16, 16, 16)), [[5.3, 7.1, 8.9]], [[0, 0, 0]], [0.0], [[0.02, 0.01, -0.015]])
    kw = dict(kT=0.0, kernel=4, advection=True)
    T = 2.0
    q = [_run_to(T, dt, st, kw, grid).q[0] for dt in (0.5, 0.25, 0.125)]
    e1 = np.linalg.norm(q[0] - q[1])
    e2 = np.linalg.norm(q[1] - q[2])
    assert e1 > 0
    assert 3.0 < e1 / e2 < 5.0


def _final_slip(me, dt, T=1.6):
    grid = (16, 16, 16)
    st = icm.State(np.zeros((3, 16, 16, 16)), [[5.3, 7.1, 8.9]], [[0, 0, 0]], [me], [[0.02, 0.01, -0.015]])
    prm = _prm(grid, kT=0.0, dt=dt, kernel=4, slip="visc")
    for _ in range(int(round(T / dt))):
        tr = {}
        st = icm.icm_step(st, prm, tr)
    return np.linalg.norm(st.u - icm.interpolate(st.v, tr["q_half"], 4, 1.0))


def test_slip_is_order_me_dt2_for_inertial_blob():
    """Appendix C: the no-slip violation u^{n+1} - J^{n+1/2} v^{n+1} (viscous slip option)
    is O(m_e dt^2): zero for m_e = 0, linear in m_e, and at least second order in dt
    (it falls ~dt^3 here because dv itself shrinks with dt on this smooth problem)."""
    assert _final_slip(0.0, 0.2) == 0.0
    s1, s2 = _final_slip(0.3, 0.2), _final_slip(0.6, 0.2)
    assert s1 > 0 and s2 / s1 == pytest.approx(2.0, rel=0.05)
    a, b, c = (_final_slip(0.6, dt) for dt in (0.2, 0.1, 0.05))
    assert a / b > 4.0 and b / c > 4.0


@pytest.mark.slow
def test_fluid_equilibrium_variance_exact_for_any_dt():
    """Linear fluctuating Stokes (no advection, no blobs): every transverse mode has
    variance kT/(rho dV_f) for any dt, so a face carries (2/3)(1 - N^-3) kT/(rho dV_f)."""
    grid = (8, 8, 8)
    kT = 1e-3
    for dt in (0.5, 5.0):
        prm = _prm(grid, kT=kT, dt=dt, kernel=4, seed=123, advection=False)
        st = icm.State(np.zeros((3, 8, 8, 8)), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3)))
        acc, cnt = 0.0, 0
        for n in range(260):
            st = icm.icm_step(st, prm)
            if n >= 20:
                acc += np.mean(st.v ** 2)
                cnt += 1
        want = (2.0 / 3.0) * (1.0 - 8.0 ** -3) * kT
        assert acc / cnt == pytest.approx(want, rel=0.03)


@pytest.mark.slow
def test_passive_blob_velocity_variance_is_kT_JPS():
    """m_e = 0, F = 0: blobs are tracers, u = J v, so <u u^T> = (kT/rho) J P' S with P'
    the projection without the (unforced, zero) mean mode."""
    grid = (10, 10, 10)
    kT = 1e-3
    prm = _prm(grid, kT=kT, dt=1.0, kernel=3, seed=7, advection=False)
    rng = np.random.default_rng(8)
    nb = 12
    q0 = rng.uniform(0, 10, size=(nb, 3))
    st = icm.State(np.zeros((3, 10, 10, 10)), q0, np.zeros((nb, 3)), np.zeros(nb), np.zeros((nb, 3)))
    acc, cnt = 0.0, 0
    for n in range(420):
        st = icm.icm_step(st, prm)
        if n >= 20:
            acc += np.mean(st.u ** 2)
            cnt += 1
    # exact JPS trace at the (slowly drifting) positions, minus the mean-mode term
    tr = 0.0
    for q in st.q:
        for c in range(3):
            F = np.zeros((1, 3))
            F[0, c] = 1.0
            tr += icm.interpolate(icm.spectral_solve(icm.spread(F, q[None], 3, 1.0, (10, 10, 10)), 1.0, 0.0, 1.0),
                                  q[None], 3, 1.0)[0, c]
    jps = tr / (3 * nb) - 1.0 / 1000.0
    assert acc / cnt == pytest.approx(kT * jps, rel=0.06)


@pytest.mark.parametrize("kernel", [3, 4])
def test_JPS_close_to_two_thirds_inverse_volume(kernel):
    """Sec. III.A.2: for N = 32 the diagonal of dV~ J P S - I is within ~5% and the
    off-diagonal is ~0.1%, where dV~ = 3 dV / 2."""
    n = 32
    shape = (n, n, n)
    dvt = 1.5 * icm.blob_volume(kernel, 1.0)
    rng = np.random.default_rng(kernel)
    for q in rng.uniform(0, n, size=(4, 3)):
        m = np.zeros((3, 3))
        for c in range(3):
            F = np.zeros((1, 3))
            F[0, c] = 1.0
            m[:, c] = icm.interpolate(icm.spectral_solve(icm.spread(F, q[None], kernel, 1.0, shape), 1.0, 0.0, 1.0),
                                      q[None], kernel, 1.0)[0]
        dI = dvt * m - np.eye(3)
        assert np.abs(np.diag(dI)).max() < 0.05
        assert np.abs(dI - np.diag(np.diag(dI))).max() < 0.005


def test_trap_force_hand_values_at_the_midpoint():
    """F^{n+1/2} = F - k (q^{n+1/2} - c) to the nearest image; with v = 0, q^{n+1/2} = q."""
    grid = (16, 16, 16)
    prm = _prm(grid, kT=0.0, dt=0.5, trap_k=0.25, trap_center=(0.0, 0.0, 0.0))
    q = [[10.0, 1.0, 15.5], [3.0, 8.5, 0.25]]
    st = icm.State(np.zeros((3, 16, 16, 16)), q, np.zeros((2, 3)), [0.0, 0.0], [[0.1, 0.0, 0.0], [0.0, 0.0, 0.0]])
    tr = {}
    icm.icm_step(st, prm, tr)
    # nearest-image displacements by hand: (-6, 1, -0.5) and (3, -7.5, 0.25)
    want = np.array([[0.1 + 1.5, -0.25, 0.125], [-0.75, 1.875, -0.0625]])
    np.testing.assert_allclose(tr["force_half"], want, rtol=0, atol=1e-15)


def test_trap_impulse_changes_momentum():
    """Appendix C: P^{n+1} - P^n = dt sum_i F_i^{n+1/2}, with the trap force at q^{n+1/2}."""
    grid = (12, 12, 12)
    st = _state(grid, 5, 77, me_scale=1.0, vamp=0.02, force=0.01)
    prm = _prm(grid, kT=1e-3, dt=0.1, trap_k=0.05, trap_center=(6.0, 5.0, 7.0))
    p0 = icm.total_momentum(st, prm)
    tr = {}
    st1 = icm.icm_step(st, prm, tr)
    dP = icm.total_momentum(st1, prm) - p0
    impulse = prm.dt * tr["force_half"].sum(axis=0)
    assert np.abs(impulse).max() > 1e-3
    np.testing.assert_allclose(dP, impulse, rtol=1e-11, atol=1e-15)


def trap_trajectory(dt, T, me=0.0, k=0.01, slip="visc"):
    """Positions after each step of a blob released from rest 10 cells from the trap
    centre on a 16^3 grid (the setup of Sec. III.D, kT = 0)."""
    grid = (16, 16, 16)
    prm = _prm(grid, kT=0.0, dt=dt, kernel=4, slip=slip, trap_k=k, trap_center=(0.0, 0.0, 0.0))
    st = icm.State(np.zeros((3, 16, 16, 16)), [[10.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]], [me], [[0.0, 0.0, 0.0]])
    out = []
    for _ in range(int(round(T / dt))):
        st = icm.icm_step(st, prm)
        out.append(st.q[0].copy())
    return np.array(out)


def e_dt(qa, qb, box=16.0):
    """Eq. E_dt_definition: mean distance between the dt run at step n and the dt/2 run at
    step 2n (nearest image)."""
    d = qa - qb[1::2]
    d -= box * np.round(d / box)
    return np.linalg.norm(d, axis=1).mean()


def test_trap_error_decays_second_order_for_neutral_blob():
    """Sec. III.D, Fig. convergenceShort (left): second order for m_e = 0."""
    T = 16.0
    q = {dt: trap_trajectory(dt, T) for dt in (1.0, 0.5, 0.25)}
    assert np.linalg.norm(q[0.25][-1] - [10.0, 0.0, 0.0]) > 1e-3     # the blob moved
    e1, e2 = e_dt(q[1.0], q[0.5]), e_dt(q[0.5], q[0.25])
    assert 3.2 < e1 / e2 < 4.8
