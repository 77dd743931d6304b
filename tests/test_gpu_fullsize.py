"""The full-size workloads (256^3 grid with 20000 blobs, 4-point kernel; 128^3 with 2000
blobs, 3-point) in the launch configuration bench.py times: whole steps of the 256^3
configuration against the oracle at sampled time levels (an oracle step takes tens of
seconds there), one FP32 step against the FP64 GPU step from the same state, the
conservation laws of the step, and the operators of the step against the oracle at
full size."""
import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm as oracle

from _gpu_helpers import TOL, compare_states, make_sim, read_oracle_state, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icm():
    import paper_1212_6427_gb300 as m
    from paper_1212_6427_gb300 import build
    build.build_library()
    return m


@pytest.fixture(scope="module")
def large():
    w = wl.workload("large")
    w["v0"] = wl.random_fluid(w["grid"], 0.05, 7)
    return w


def _large_prm(w):
    return oracle.Params(w["grid"], h=w["h"], rho=w["rho"], eta=w["eta"], kT=w["kT"], dt=w["dt"], kernel=w["kernel"],
                         seed=w["seed"])


@pytest.fixture(scope="module")
def large_samples(icm, large):
    """Two sampled time levels of the 256^3 configuration with the oracle's next step:
    level 0 (the synthetic state, no history) and level 5 (read back from five FP64 GPU
    steps, so the Adams-Bashforth history and the lagged slip term are in play)."""
    w = large
    prm = _large_prm(w)
    st0 = oracle.State(w["v0"], w["q"], w["u"], w["me"], w["force"])
    sim = make_sim(prm, st0, 64)
    sim.step(5)
    st5, _ = read_oracle_state(sim, prm, w["me"], w["force"])
    sim.close()
    assert st5.step == 5 and st5.adv_prev is not None
    return prm, [(st0, oracle.icm_step(st0, prm)), (st5, oracle.icm_step(st5, prm))]


@pytest.mark.parametrize("precision", [32, 64])
def test_large_config_steps_match_oracle(icm, large_samples, precision):
    """The 256^3 / 20000-blob / 4-point configuration bench.py times (FP32 in the plan the
    autotuner picks there, FP64 in the default plan, as bench.py's FP64 leg): at each
    sampled level the state is written into the simulation, one GPU step is taken, and
    v, u, the blob displacement and the total momentum are compared with the oracle's
    step from the same state (FP32 at 2e-5, FP64 at 1e-12, norm-wise)."""
    prm, samples = large_samples
    st0 = samples[0][0]
    sim = make_sim(prm, st0, precision)
    if precision == 32:
        icm.icm_autotune(sim.handle, 2)      # state restored; the plan bench.py uses
    worst = {}
    for cur, want in samples:
        sim.write(cur.q, cur.u, cur.v.ravel(), None if cur.adv_prev is None else cur.adv_prev.ravel(), cur.slip_g,
                  cur.step)
        sim.step(1)
        got, mom = read_oracle_state(sim, prm, cur.me, cur.force)
        assert got.step == cur.step + 1
        err = compare_states(got, want, prm, cur.q)
        scale = prm.rho * prm.h ** 3 * np.abs(want.v).sum() + np.abs(want.me[:, None] * want.u).sum()
        err["P"] = float(np.abs(mom - oracle.total_momentum(want, prm)).max() / scale)
        for k, e in err.items():
            worst[k] = max(worst.get(k, 0.0), e)
    sim.close()
    print("256^3 step vs oracle, FP%d: %s" % (precision, {k: "%.2e" % e for k, e in worst.items()}))
    for k, e in worst.items():
        assert e < TOL[precision], (k, e, worst)


def _sim(icm, w, precision):
    s = icm.Simulation(w["grid"], w["h"], w["rho"], w["eta"], w["kT"], w["dt"], w["kernel"], w["seed"], precision)
    s.add_blobs(w["q"], w["u"], w["me"])
    s.set_forces(w["force"])
    s.write(w["q"], w["u"], w["v0"].ravel(), None, None, 0)
    return s


def test_large_fp32_step_matches_fp64_step(icm, large):
    """Two steps of the tuned FP32 step (the plan bench.py times) against the FP64 path."""
    s32 = _sim(icm, large, 32)
    icm.icm_autotune(s32.handle, 2)        # state restored; the plan bench.py uses
    s64 = _sim(icm, large, 64)
    s32.step(2)
    s64.step(2)
    a, b = s32.read(fluid=True), s64.read(fluid=True)
    assert a["step"] == b["step"] == 2
    assert rel(a["fluid"], b["fluid"]) < TOL[32]
    assert rel(a["vel"], b["vel"]) < TOL[32]
    L = np.array(large["grid"], dtype=float) * large["h"]
    dq = a["pos"] - b["pos"]
    dq -= L * np.round(dq / L)
    disp = b["pos"] - large["q"]
    disp -= L * np.round(disp / L)
    assert np.linalg.norm(dq) < TOL[32] * np.linalg.norm(disp)
    s32.close()
    s64.close()


def test_large_step_momentum_and_divergence(icm, large):
    """P^{n+1} - P^n = dt sum F (FP64 bookkeeping) and D v^{n+1} = 0 to FP32 roundoff."""
    s = _sim(icm, large, 32)
    p0 = s.read()["momentum"]
    s.step(1)
    r = s.read(fluid=True)
    dP = r["momentum"] - p0
    want = large["dt"] * np.asarray(large["force"]).sum(axis=0)
    np.testing.assert_allclose(dP, want, rtol=1e-9, atol=1e-12 * np.abs(p0).max())
    nx, ny, nz = large["grid"]
    v = r["fluid"].reshape(3, nz, ny, nx)
    div = oracle.divergence(v, large["h"])
    assert np.abs(div).max() < 1e-4 * np.abs(v).max() / large["h"]
    s.close()


def test_large_operators_match_oracle(icm, large):
    """Solve, interpolation and spreading at 256^3 with 20000 blobs (FP32 bar)."""
    w = large
    s = icm.Simulation(w["grid"], w["h"], w["rho"], w["eta"], w["kT"], w["dt"], w["kernel"], w["seed"], 32)
    v = w["v0"]
    got = icm.icm_op_spectral_solve(s.handle, w["rho"] / w["dt"], 0.5 * w["eta"], v.ravel())
    assert rel(got, oracle.spectral_solve(v, w["rho"] / w["dt"], 0.5 * w["eta"], w["h"])) < TOL[32] / 2
    assert rel(icm.icm_op_interpolate(s.handle, w["q"], v.ravel()), oracle.interpolate(v, w["q"], 4, w["h"])) \
        < TOL[32] / 2
    shape = (w["grid"][2], w["grid"][1], w["grid"][0])
    F = np.random.default_rng(3).standard_normal((len(w["q"]), 3))
    assert rel(icm.icm_op_spread(s.handle, s.ncell, w["q"], F), oracle.spread(F, w["q"], 4, w["h"], shape)) \
        < TOL[32] / 2
    s.close()


def test_bulk_rhs_matches_oracle(icm):
    """The explicit right-hand side at 128^3 (stress normals, advection, AB2) against the oracle."""
    w = wl.workload("bulk")
    s = icm.Simulation(w["grid"], w["h"], w["rho"], w["eta"], w["kT"], w["dt"], w["kernel"], w["seed"], 32)
    v = wl.random_fluid(w["grid"], 0.05, 8)
    a_prev = wl.random_fluid(w["grid"], 0.01, 9)
    r, a = icm.icm_op_explicit_rhs(s.handle, v.ravel(), a_prev.ravel(), 5)
    prm = oracle.Params(w["grid"], h=w["h"], rho=w["rho"], eta=w["eta"], kT=w["kT"], dt=w["dt"], kernel=w["kernel"],
                        seed=w["seed"])
    rw, aw = oracle.explicit_rhs(v, a_prev, 5, prm)
    assert rel(r, rw) < TOL[32] / 2
    assert rel(a, aw) < TOL[32] / 2
    s.close()


@pytest.fixture(scope="module")
def widest():
    # the largest register sides along x and y (512, 384) with a 256 z side: 50M cells
    cfg = dict(grid=(512, 384, 256), h=1.0, rho=1.0, eta=1.0, kT=1e-3, dt=0.01, kernel=4, seed=41, precision=32,
               steps=1, nblobs=20000, me_range=(-0.5, 2.0), force=(1e-4, 0.0, -5e-5), place_seed=42,
               min_spacing=2.0)
    w = wl._materialise(cfg)
    w["v0"] = wl.random_fluid(w["grid"], 0.05, 43)
    return w


def test_widest_sides_step(icm, widest):
    """One tuned FP32 step on a 512 x 384 x 256 grid against the FP64 step, with the
    conservation laws of the step."""
    w = widest
    s32 = _sim(icm, w, 32)
    icm.icm_autotune(s32.handle, 1)
    p0 = s32.read()["momentum"]
    s64 = _sim(icm, w, 64)
    s32.step(1)
    s64.step(1)
    a, b = s32.read(fluid=True), s64.read(fluid=True)
    s32.close()
    s64.close()
    assert rel(a["fluid"], b["fluid"]) < TOL[32]
    assert rel(a["vel"], b["vel"]) < TOL[32]
    dP = a["momentum"] - p0
    want = w["dt"] * np.asarray(w["force"]).sum(axis=0)
    np.testing.assert_allclose(dP, want, rtol=1e-9, atol=1e-12 * np.abs(p0).max())
    nx, ny, nz = w["grid"]
    v = a["fluid"].reshape(3, nz, ny, nx)
    div = oracle.divergence(v, w["h"])
    assert np.abs(div).max() < 1e-4 * np.abs(v).max() / w["h"]
