"""Accumulations by atomics, checked without a race detector.

The spreads add every blob's contribution to the grid with atomics (FP32 or FP64, in
global memory for the operator, in shared memory inside the x passes) and the gathers add
each row block's part of J to FP64 accumulators, so the order of the additions changes
from run to run.  A lost or doubled update would show as the error of a whole term.
These tests hold the GPU spread, cell by cell, to an FP64 sum in a fixed order within the
rounding bound of a sum of n terms (n the terms of that cell), two runs to twice that,
and a step without blobs (no atomics anywhere) to bit-for-bit repeatability."""
import numpy as np
import pytest

import icm_workloads as wl
from oracle import icm as oracle

from _gpu_helpers import make_sim, rel

pytestmark = pytest.mark.gpu

EPS = {32: 2.0 ** -24, 64: 2.0 ** -53}


@pytest.fixture(scope="module")
def icm():
    import paper_1212_6427_gb300 as m
    from paper_1212_6427_gb300 import build
    build.build_library()
    return m


def _cell_terms(q, F, kernel, h, shape):
    """Per cell and component: the number of blob terms added there, the sum of their
    magnitudes and the largest magnitude (FP64, fixed order)."""
    count = np.zeros((3,) + tuple(shape))
    absum = np.zeros_like(count)
    big = np.zeros_like(count)
    for comp in range(3):
        (ix, iy, iz), (wx, wy, wz) = oracle._blob_stencil(q, comp, kernel, h, shape)
        w = ix.shape[1]
        t = np.abs(wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
                   * (F[:, comp] / h ** 3)[:, None, None, None])
        at = (np.broadcast_to(iz[:, :, None, None], t.shape).ravel(),
              np.broadcast_to(iy[:, None, :, None], t.shape).ravel(),
              np.broadcast_to(ix[:, None, None, :], t.shape).ravel())
        np.add.at(count[comp], at, 1.0)
        np.add.at(absum[comp], at, t.ravel())
        np.maximum.at(big[comp], at, t.ravel())
    return count, absum, big


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("kernel", [3, 4])
def test_atomic_spread_is_a_sum_of_every_term(icm, precision, kernel):
    """4000 blobs on 8 x 12 x 9 cells: every cell takes 70 to 320 terms per component,
    added by concurrent atomics.  |GPU - fixed-order FP64 sum| <= (n + 8) eps sum |t| in
    every cell (n terms, a few roundings per term), and two runs differ by at most twice
    that.  The bound is below 5% of every cell's largest term, so that term lost or added
    twice would break it."""
    grid = (8, 12, 9)
    h = 0.9
    sim = icm.Simulation(grid, h, 1.3, 0.7, 0.0, 0.05, kernel, 3, precision)
    shape = (grid[2], grid[1], grid[0])
    rng = np.random.default_rng(41)
    q = rng.uniform(0, 1, size=(4000, 3)) * np.array(grid) * h
    F = rng.standard_normal((4000, 3))
    want = oracle.spread(F, q, kernel, h, shape)
    count, absum, big = _cell_terms(q, F, kernel, h, shape)
    assert count.min() >= 50
    bound = (count + 8.0) * EPS[precision] * absum
    assert np.all(bound < 0.05 * big)   # losing any cell's largest term would show
    runs = [icm.icm_op_spread(sim.handle, sim.ncell, q, F).reshape(want.shape) for _ in range(2)]
    for got in runs:
        assert np.all(np.abs(got - want) <= bound)
    assert np.all(np.abs(runs[0] - runs[1]) <= 2.0 * bound)
    sim.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_step_without_blobs_repeats_bit_for_bit(icm, precision):
    """No blobs: no atomics in the step (the noise, stencils, FFT passes and the FP64
    momentum sums are fixed-order), so the same state stepped twice gives the same bits."""
    prm = oracle.Params((48, 32, 64), kT=1e-3, dt=0.05, kernel=4, seed=17)
    st = oracle.State(wl.random_fluid(prm.grid, 0.05, 5), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0),
                      np.zeros((0, 3)))
    out = []
    for _ in range(2):
        sim = make_sim(prm, st, precision)
        sim.step(3)
        out.append(sim.read(fluid=True))
        sim.close()
    np.testing.assert_array_equal(out[0]["fluid"], out[1]["fluid"])
    np.testing.assert_array_equal(out[0]["momentum"], out[1]["momentum"])


@pytest.mark.parametrize("precision", [32, 64])
def test_step_with_blobs_repeats_to_rounding(icm, precision):
    """With blobs the spreads (shared-memory atomics in the x passes) and the gathers
    (FP64 atomics over row blocks) add in a varying order: two runs of three steps from
    one state agree to rounding, not necessarily bit for bit."""
    grid = (64, 32, 48)
    prm = oracle.Params(grid, kT=1e-3, dt=0.05, kernel=4, seed=19)
    nb = 40
    rng = np.random.default_rng(6)
    q = wl.random_sequential_addition(nb, grid, 1.0, 2.0, 6)
    st = oracle.State(wl.random_fluid(grid, 0.05, 7), q, 0.05 * rng.standard_normal((nb, 3)),
                      rng.uniform(-0.5, 2.0, size=nb), 0.01 * rng.standard_normal((nb, 3)))
    out = []
    for _ in range(2):
        sim = make_sim(prm, st, precision)
        sim.step(3)
        out.append(sim.read(fluid=True))
        sim.close()
    tol = 1e-5 if precision == 32 else 1e-13
    for k in ("fluid", "vel", "pos"):
        assert rel(out[1][k], out[0][k]) < tol, k
