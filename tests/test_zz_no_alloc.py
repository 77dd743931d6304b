"""icm_fluid_momentum_static: the fluid momentum of a device face field, computed
without allocating any device memory (for callers that cannot call cudaMalloc,
e.g. while a stream capture is open or when a framework already owns the GPU's
memory).  Its result must equal the momentum icm_read_state reports for the same
field (the library's allocating reduction), within the FP64 parity tolerance,
on two calls in a row that reuse the shared static scratch array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def icm():
    from paper_1212_6427_gb300 import build
    build.build_library()
    import paper_1212_6427_gb300 as m
    return m


def _reference_momentum(icm, grid, fluid, precision, rho, h):
    """Momentum through the existing entry points: icm_write_state + icm_read_state."""
    sim = icm.Simulation(grid, h=h, rho=rho, eta=1.0, kT=0.0, dt=0.05, kernel=4, seed=1, precision=precision)
    sim.write(np.zeros((0, 3)), np.zeros((0, 3)), fluid)
    p = sim.read()["momentum"]
    sim.close()
    return p


@pytest.mark.parametrize("precision", [64, 32])
def test_static_momentum_matches_read_state_twice(icm, precision):
    import torch
    dtype = torch.float64 if precision == 64 else torch.float32
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(precision)
    cases = [((48, 36, 32), 1.3, 0.7), ((16, 16, 12), 0.9, 1.1)]    # the second call is smaller
    for grid, rho, h in cases:
        n = int(np.prod(grid))
        fluid = 0.2 * rng.standard_normal(3 * n) + 0.01
        want = _reference_momentum(icm, grid, fluid, precision, rho, h)
        dev = torch.tensor(fluid, dtype=dtype, device="cuda")
        torch.cuda.synchronize()
        got = icm.icm_fluid_momentum_static(dev.data_ptr(), precision, n, rho, h, stream.cuda_stream)
        assert np.abs(want).max() > 0
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL, (grid, got, want)


def test_static_momentum_rejects_bad_sizes(icm):
    import torch
    dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    for ncell in (0, 134217728 + 1):
        with pytest.raises(icm.IcmError) as ei:
            icm.icm_fluid_momentum_static(dev.data_ptr(), 64, ncell, 1.0, 1.0)
        assert ei.value.status == icm.ICM_EINVAL
    with pytest.raises(icm.IcmError):
        icm.icm_fluid_momentum_static(dev.data_ptr(), 16, 1, 1.0, 1.0)
