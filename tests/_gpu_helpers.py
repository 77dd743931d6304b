"""Helpers shared by the GPU parity tests: move a state between the oracle and the
CUDA library through the C ABI, and norm-wise relative errors."""
import numpy as np

from oracle import icm as oracle

# Norm-wise relative tolerances per output (the FP64 GPU path must agree with the
# FP64 oracle to 1e-12; the FP32 path to 2e-5).
TOL = {64: 1e-12, 32: 2e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def min_image(d, box):
    return d - box * np.round(d / box)


def flags_of(prm):
    f = 0 if prm.advection else 0x1
    f |= {"visc": 0x0, "zero": 0x2, "full": 0x4}[prm.slip]
    if prm.thermal_drift:
        f |= 0x8
    return f


def make_sim(prm, state, precision):
    import paper_1212_6427_gb300 as icm
    sim = icm.Simulation(prm.grid, prm.h, prm.rho, prm.eta, prm.kT, prm.dt, prm.kernel, prm.seed, precision,
                         flags_of(prm))
    if state.q.shape[0]:
        sim.add_blobs(state.q, state.u, state.me)
        sim.set_forces(state.force)
    if prm.trap_k != 0.0:
        sim.set_trap(prm.trap_k, prm.trap_center)
    if prm.wca_epsilon != 0.0:
        sim.set_wca(prm.wca_epsilon, prm.wca_sigma)
    sim.write(state.q, state.u, state.v.ravel(), None if state.adv_prev is None else state.adv_prev.ravel(),
              state.slip_g, state.step)
    return sim


def read_oracle_state(sim, prm, me, force):
    r = sim.read(fluid=True)
    adv, g, hist = sim.read_aux()
    shape = (3,) + prm.shape
    return oracle.State(r["fluid"].reshape(shape), r["pos"], r["vel"], me, force,
                        adv.reshape(shape) if hist else None, g, r["step"]), r["momentum"]


def compare_states(got, want, prm, q_prev):
    """Errors of v, u and the blob displacement q^{n+1} - q^n.  The displacement error is
    taken beyond the floor that FP64 positions in [0, L) set (two ulps of L per
    component): both sides round q^{n+1} = q^n + dt/2 J(...) to such positions, so a
    displacement can never be compared more finely than that."""
    box = prm.box
    err = dict(v=rel(got.v, want.v))
    if want.q.shape[0]:
        err["u"] = rel(got.u, want.u)
        dq_got, dq_want = min_image(got.q - q_prev, box), min_image(want.q - q_prev, box)
        floor = 2.0 * np.finfo(np.float64).eps * float(np.max(box)) * np.sqrt(want.q.size)
        err["dq"] = float(max(0.0, np.linalg.norm(dq_got - dq_want) - floor) / np.linalg.norm(dq_want))
        err["q"] = float(np.linalg.norm(min_image(got.q - want.q, box)) / np.linalg.norm(want.q))
    return err
