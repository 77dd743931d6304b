"""GPU parity of the Stokes limit of the solve and of the blob-grid coupling matrices
of Sec. III.A.2 (icm_op_coupling) against the oracle, and the paper's hydrodynamic
radius of the three-point kernel measured on the GPU."""
import numpy as np
import pytest

from oracle import icm as oracle

from _gpu_helpers import TOL, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icm():
    import paper_1212_6427_gb300 as m
    from paper_1212_6427_gb300 import build
    build.build_library()
    return m


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("grid", [(16, 16, 16), (32, 12, 24), (9, 18, 8), (64, 32, 48)])
def test_stokes_solve_matches_oracle(icm, precision, grid):
    sim = icm.Simulation(grid, 0.8, 1.0, 1.3, 0.0, 0.05, 4, 1, precision, 0)
    nx, ny, nz = grid
    r = np.random.default_rng(5).standard_normal((3, nz, ny, nx))
    got = icm.icm_op_spectral_solve(sim.handle, 0.0, 1.3, r.ravel())
    want = oracle.spectral_solve(r, 0.0, 1.3, 0.8)
    assert rel(got, want) < TOL[precision] / 2
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("kernel", [3, 4])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (0.0, 1.3), (2.0, 0.5)])
def test_coupling_matrices_match_oracle(icm, precision, kernel, ab):
    grid = (16, 24, 12)
    sim = icm.Simulation(grid, 1.0, 1.0, 1.0, 0.0, 0.05, kernel, 1, precision, 0)
    rng = np.random.default_rng(kernel * 10 + int(ab[1] * 10))
    qj = rng.uniform(0, 1, size=(4, 3)) * grid
    qi = qj + rng.uniform(-3, 3, size=(4, 3))
    qi[0] = qj[0]
    got = icm.icm_op_coupling(sim.handle, qi, qj, ab[0], ab[1])
    want = np.array([oracle.coupling_matrix(qi[p], qj[p], grid, kernel, 1.0, ab[0], ab[1]) for p in range(4)])
    assert rel(got, want) < TOL[precision]
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_three_point_hydrodynamic_radius_on_gpu(precision):
    """Sec. III.A.2: R_H ~ 0.91 dx for the three-point kernel."""
    from paper_1212_6427_gb300 import experiments
    r = experiments.hydrodynamic_radius((32, 32, 32), 3, npos=8, precision=precision)
    assert r["R_H"] == pytest.approx(0.91, rel=0.02)
    assert r["mu_rel_spread"] < 0.02


def test_translational_invariance_statistics_match_oracle():
    from paper_1212_6427_gb300 import experiments
    got = experiments.jps_translational((16, 16, 16), 4, npos=5, seed=3, precision=64)
    rng = np.random.default_rng(3)
    q = rng.uniform(0.0, 1.0, size=(5, 3)) * 16.0
    di = np.array([oracle.jps_deviation(q[p], (16, 16, 16), 4, 1.0) for p in range(5)])
    diag = np.diagonal(di, axis1=1, axis2=2)
    assert got["mean_diag"] == pytest.approx(diag.mean(), rel=1e-9, abs=1e-12)
    assert got["max_abs_diag"] == pytest.approx(np.abs(diag).max(), rel=1e-9)


def test_coupling_input_errors(icm):
    sim = icm.Simulation((16, 16, 16), kT=0.0, kernel=4, precision=64)
    with pytest.raises(icm.IcmError):
        icm.icm_op_coupling(sim.handle, [[1.0, 2.0, 3.0]], [[1.0, 2.0, np.nan]], 1.0, 0.0)
    with pytest.raises(icm.IcmError):
        icm.icm_op_coupling(sim.handle, [[1.0, 2.0, 3.0]], [[1.0, 2.0, 3.0]], 0.0, 0.0)
    with pytest.raises(icm.IcmError):
        icm.icm_op_spectral_solve(sim.handle, -1.0, 1.0, np.zeros(3 * 16 ** 3))
    sim.close()
