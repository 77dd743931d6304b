"""icm_fluid_momentum_static: the fluid momentum of a device face field, computed
without allocating any device memory (for callers that cannot call cudaMalloc,
e.g. while a stream capture is open or when a framework already owns the GPU's
memory).  Its result must equal, within the FP64 parity tolerance, on two calls in
a row that reuse the shared static scratch array:
  * the momentum icm_read_state reports for the same field (the library's
    allocating reduction), and
  * rho h^3 sum v summed by numpy in FP64 over the same (device-rounded) values,
    which shares nothing with the library.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import icm_workloads as wl

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


def _numpy_momentum(dev, rho, h):
    """rho h^3 sum_k v_k per component, numpy FP64 over the values as stored on the device."""
    vals = dev.cpu().numpy().astype(np.float64).reshape(3, -1)
    return rho * h ** 3 * vals.sum(axis=1)


def _relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [64, 32])
def test_static_momentum_matches_read_state_twice(icm, precision):
    import torch
    dtype = torch.float64 if precision == 64 else torch.float32
    stream = torch.cuda.Stream()
    cases = [((48, 36, 32), 1.3, 0.7, 11), ((16, 16, 12), 0.9, 1.1, 12)]    # the second call is smaller
    for grid, rho, h, seed in cases:
        n = int(np.prod(grid))
        fluid = (wl.random_fluid(grid, 0.2, seed) + 0.01).ravel()
        want = _reference_momentum(icm, grid, fluid, precision, rho, h)
        dev = torch.tensor(fluid, dtype=dtype, device="cuda")
        torch.cuda.synchronize()
        got = icm.icm_fluid_momentum_static(dev.data_ptr(), precision, n, rho, h, stream.cuda_stream)
        assert np.abs(want).max() > 0
        assert _relerr(got, want) < TOL, (grid, got, want)
        assert _relerr(got, _numpy_momentum(dev, rho, h)) < TOL, (grid, got)


def test_static_momentum_many_partials_256cubed(icm):
    """256^3 FP32 cells: 2048 partial sums per component, so every thread of the final
    reduction folds eight of them; twice in a row against numpy's FP64 sum."""
    import torch
    grid = (256, 256, 256)
    n = int(np.prod(grid))
    stream = torch.cuda.Stream()
    for seed, rho, h in ((21, 1.0, 1.0), (22, 1.3, 0.8)):
        fluid = wl.random_fluid(grid, 0.05, seed).ravel() + 1e-3
        dev = torch.tensor(fluid, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        got = icm.icm_fluid_momentum_static(dev.data_ptr(), 32, n, rho, h, stream.cuda_stream)
        assert _relerr(got, _numpy_momentum(dev, rho, h)) < TOL, (seed, got)
        del dev


def test_static_momentum_beside_an_open_capture(icm):
    """A capture is open on one stream: the call on another non-blocking stream works and
    the capture still ends cleanly; the capturing stream itself is refused (ICM_EINVAL)
    without disturbing the capture."""
    import torch
    grid = (32, 24, 16)
    n = int(np.prod(grid))
    fluid = (wl.random_fluid(grid, 0.1, 31) + 0.02).ravel()
    dev = torch.tensor(fluid, dtype=torch.float64, device="cuda")
    x = torch.ones(1024, device="cuda")
    other = torch.cuda.Stream()
    cap = torch.cuda.Stream()
    want = _numpy_momentum(dev, 1.2, 0.9)
    # the first call on a device looks up the scratch address: make it before the capture
    icm.icm_fluid_momentum_static(dev.data_ptr(), 64, n, 1.2, 0.9, other.cuda_stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
        y = x * 2.0
        got = icm.icm_fluid_momentum_static(dev.data_ptr(), 64, n, 1.2, 0.9, other.cuda_stream)
        with pytest.raises(icm.IcmError) as ei:
            icm.icm_fluid_momentum_static(dev.data_ptr(), 64, n, 1.2, 0.9, cap.cuda_stream)
        refused = ei.value.status
    g.replay()
    torch.cuda.synchronize()
    assert refused == icm.ICM_EINVAL
    assert float(y.sum()) == 2048.0
    assert _relerr(got, want) < TOL


def test_static_momentum_rejects_bad_sizes(icm):
    import torch
    dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    for ncell in (0, 134217728 + 1):
        with pytest.raises(icm.IcmError) as ei:
            icm.icm_fluid_momentum_static(dev.data_ptr(), 64, ncell, 1.0, 1.0)
        assert ei.value.status == icm.ICM_EINVAL
    with pytest.raises(icm.IcmError):
        icm.icm_fluid_momentum_static(dev.data_ptr(), 16, 1, 1.0, 1.0)
