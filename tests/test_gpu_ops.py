"""GPU parity of each operator of the step against the FP64 oracle, through the C ABI.

Sizes span several shared-memory tiles and ragged tails (odd and radix-3 sides,
non-cubic boxes, blobs on the periodic seam)."""
import os

import numpy as np
import pytest

import icm_workloads as wl

from oracle import icm as oracle
from oracle import philox

from _gpu_helpers import TOL, rel

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GRIDS = [(16, 16, 16), (32, 12, 24), (9, 18, 8), (48, 32, 27), (96, 8, 16), (64, 128, 96), (256, 24, 192),
         (128, 64, 48), (384, 8, 12)]


@pytest.fixture(scope="module")
def icm():
    import paper_1212_6427_gb300 as m
    from paper_1212_6427_gb300 import build
    build.build_library()
    return m


def _sim(icm, grid, precision, kernel=4, kT=1e-3, dt=0.05, h=1.0, seed=7, flags=0):
    return icm.Simulation(grid, h, 1.3, 0.7, kT, dt, kernel, seed, precision, flags)


def test_philox_bitwise_against_oracle_and_known_answers(icm):
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        rows = [[int(x, 16) for x in ln.split()] for ln in fh if ln.strip() and not ln.startswith("#")]
    for r in rows:
        got = icm.icm_op_philox(1, r[0:4], r[4:6])
        assert [int(x) for x in got[0]] == r[6:10]
    n = 100_000
    got = icm.icm_op_philox(n, (5, 77, 1, 0), (0xDEADBEEF, 0x12345678))
    want = philox.philox4x32((np.arange(5, 5 + n), 77, 1, 0), (0xDEADBEEF, 0x12345678))
    for w in range(4):
        assert np.array_equal(got[:, w], want[w])


@pytest.mark.parametrize("precision", [64, 32])
def test_stress_normals(icm, precision):
    grid = (16, 12, 9)
    sim = _sim(icm, grid, precision, seed=(1 << 40) + 3)
    n = int(np.prod(grid))
    got = icm.icm_op_stress_normals(sim.handle, n, 11)
    want = philox.stress_normals((1 << 40) + 3, 11, n, grid[0] * grid[1])
    tol = 1e-14 if precision == 64 else 2e-6
    assert rel(got, want) < tol
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("ab", [(26.0, 0.35), (1.0, 0.0), (1.3, 0.0175)])
def test_spectral_solve(icm, precision, grid, ab):
    sim = _sim(icm, grid, precision, h=0.8)
    nx, ny, nz = grid
    rng = np.random.default_rng(1)
    r = rng.standard_normal((3, nz, ny, nx))
    got = icm.icm_op_spectral_solve(sim.handle, ab[0], ab[1], r.ravel())
    want = oracle.spectral_solve(r, ab[0], ab[1], 0.8)
    assert rel(got, want) < TOL[precision] / 2
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("grid,kernel", [((8, 8, 8), 4), ((6, 6, 6), 3), ((12, 12, 12), 3), ((12, 8, 6), 3)])
def test_spectral_solve_against_naive_dft(icm, precision, grid, kernel):
    """The GPU solve against the solve whose transforms are the plain O(N^2) DFT sums
    (no FFT on either side of the comparison), on 8^3, 6^3, 12^3 and a mixed grid."""
    sim = _sim(icm, grid, precision, kernel=kernel, h=0.9)
    nx, ny, nz = grid
    r = np.random.default_rng(6).standard_normal((3, nz, ny, nx))
    for a, b in ((20.0, 0.5), (1.0, 0.0), (1.3, 0.0175)):
        got = icm.icm_op_spectral_solve(sim.handle, a, b, r.ravel())
        assert rel(got, oracle.spectral_solve_dft(r, a, b, 0.9)) < TOL[precision] / 2, (a, b)
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("kernel", [3, 4])
@pytest.mark.parametrize("grid", [(16, 16, 16), (9, 18, 8), (48, 32, 27)])
def test_interpolate_spread_and_laplacian_gather(icm, precision, kernel, grid):
    h = 0.9
    sim = _sim(icm, grid, precision, kernel=kernel, h=h)
    nx, ny, nz = grid
    box = np.array(grid) * h
    rng = np.random.default_rng(2)
    q = rng.uniform(0, 1, size=(300, 3)) * box
    q[:4] = [[0.0, 0.0, 0.0], [box[0] - 1e-12, 0.5 * h, 0.25 * h], [0.5 * h, box[1] - 0.5 * h, 1e-9],
             [h * 3.5, h * 4.5, h * 2.0]]
    v = rng.standard_normal((3, nz, ny, nx))
    F = rng.standard_normal((300, 3))
    tol = TOL[precision] / 2
    assert rel(icm.icm_op_interpolate(sim.handle, q, v.ravel()), oracle.interpolate(v, q, kernel, h)) < tol
    want_l = oracle.interpolate(oracle.vector_laplacian(v, h), q, kernel, h)
    assert rel(icm.icm_op_interpolate_laplacian(sim.handle, q, v.ravel()), want_l) < tol
    got_s = icm.icm_op_spread(sim.handle, sim.ncell, q, F)
    assert rel(got_s, oracle.spread(F, q, kernel, h, (nz, ny, nx))) < tol
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("grid", [(16, 16, 16), (48, 24, 36), (9, 18, 8), (6, 8, 12), (96, 36, 12), (24, 12, 9),
                                  (72, 16, 27)])
@pytest.mark.parametrize("kT,hist,adv", [(1e-3, True, True), (0.0, False, True), (2e-3, True, False)])
def test_explicit_rhs(icm, precision, grid, kT, hist, adv):
    """The right-hand side against the oracle with fixed z marches (4 and 16 planes per
    block) and persistent blocks (rhs_kz = 0); the three launch shapes run the same
    arithmetic, so their results agree bit for bit.  Tiles of 32 x 16 cells are wider
    than the short sides here (several periodic wraps per tile) and ragged on the others.
    Odd Nz: the last plane's off-diagonal normals come from an unpaired Philox call and
    the march wraps from it to plane 0; marches start on odd planes (whose call is the
    one of the plane below)."""
    sim = _sim(icm, grid, precision, kernel=3, kT=kT, flags=0 if adv else 0x1, seed=99)
    nx, ny, nz = grid
    rng = np.random.default_rng(3)
    v = 0.3 * rng.standard_normal((3, nz, ny, nx))
    a_prev = rng.standard_normal((3, nz, ny, nx)) if hist else None
    step = 17
    prm = oracle.Params(grid, h=1.0, rho=1.3, eta=0.7, kT=kT, dt=0.05, kernel=3, seed=99, advection=adv)
    rw, aw = oracle.explicit_rhs(v, a_prev, step, prm)
    first = None
    for kz in (16, 0, 4):
        icm.icm_set_plan(sim.handle, rhs_kz=kz)
        r, a = icm.icm_op_explicit_rhs(sim.handle, v.ravel(), None if a_prev is None else a_prev.ravel(), step)
        assert rel(r, rw) < TOL[precision] / 2, kz
        if adv:
            assert rel(a, aw) < TOL[precision] / 2, kz
        if first is None:
            first = (r, a)
        else:
            assert np.array_equal(r, first[0]) and np.array_equal(a, first[1]), kz
    sim.close()


def test_host_io_buffers_are_the_callers(icm):
    """icm_set_blob_forces has copied the caller's (page-locked) buffer when it returns,
    and icm_read_state's total momentum (the device sum of m_e u plus the FP64 fluid
    bookkeeping) equals the same sum formed on the host from what it returned."""
    import torch
    import icm_workloads as wl
    grid, nb = (32, 32, 16), 40
    q = wl.random_sequential_addition(nb, grid, 1.0, 2.0, 5)
    rng = np.random.default_rng(5)
    u = 0.02 * rng.standard_normal((nb, 3))
    me = rng.uniform(-0.5, 2.0, size=nb)
    f = 1e-3 * rng.standard_normal((nb, 3))
    out = []
    for overwrite in (False, True):
        sim = icm.Simulation(grid, 1.0, 1.0, 1.0, 1e-3, 0.05, 4, 11, 32)
        sim.add_blobs(q, u, me)
        pinned = torch.empty((nb, 3), dtype=torch.float64, pin_memory=True).numpy()
        for step in range(3):
            pinned[:] = f * (step + 1)
            sim.set_forces(pinned)
            if overwrite:   # the library's copy is already taken: this must not reach the step
                pinned[:] = np.nan
            sim.step(1)
        r = sim.read(fluid=True)
        fv = r["fluid"].reshape(3, -1)
        fluid_p = fv.sum(axis=1)   # rho dV_f = 1
        blob_p = (me[:, None] * r["vel"]).sum(axis=0)
        # the FP64 bookkeeping and the FP32 field's own sum differ by the field's rounding
        scale = np.abs(fv).sum() + np.abs(me[:, None] * r["vel"]).sum()
        assert np.abs(r["momentum"] - (fluid_p + blob_p)).max() < 1e-6 * scale
        out.append(r)
        sim.close()
    for k in ("pos", "vel", "momentum"):
        np.testing.assert_array_equal(out[0][k], out[1][k])


def test_queued_reads_match_synchronous_reads(icm):
    """icm_read_begin / icm_read_finish: a read queued behind a step returns that step's
    state even when the next step is queued before the host collects it (two slots in
    turn), the same values a synchronous read gives; the pending count is enforced."""
    grid = (32, 16, 24)
    nb = 12
    q = wl.random_sequential_addition(nb, grid, 1.0, 2.0, 5)
    rng = np.random.default_rng(5)
    u0, me = 0.02 * rng.standard_normal((nb, 3)), rng.uniform(-0.5, 2.0, size=nb)
    sims = []
    for _ in range(2):
        s = _sim(icm, grid, 64)
        s.add_blobs(q, u0, me)
        sims.append(s)
    queued, direct = sims
    f = 1e-3 * rng.standard_normal((nb, 3))
    want = []
    for _ in range(5):
        direct.set_forces(f)
        direct.step(1)
        want.append(direct.read())
    got = []
    queued.set_forces(f)
    queued.step(1)
    queued.read_begin()
    for _ in range(4):
        queued.set_forces(f)
        queued.step(1)
        queued.read_begin()
        got.append(queued.read_finish())   # the step before the one just queued
    got.append(queued.read_finish())
    for g, w in zip(got, want):
        assert g["step"] == w["step"]
        for k in ("pos", "vel", "momentum"):
            np.testing.assert_allclose(g[k], w[k], rtol=1e-12, atol=1e-15)
    # a read queued with nothing after it equals a synchronous read bit for bit
    queued.read_begin()
    now = queued.read()
    late = queued.read_finish()
    for k in ("pos", "vel", "momentum", "step"):
        np.testing.assert_array_equal(np.asarray(late[k]), np.asarray(now[k]))
    with pytest.raises(icm.IcmError):
        queued.read_finish()
    queued.read_begin()
    queued.read_begin()
    with pytest.raises(icm.IcmError) as ei:
        queued.read_begin()
    assert ei.value.status == icm.ICM_EBUSY
    queued.read_finish()
    queued.read_finish()
    # no blobs are added while a read is pending (it returns the blobs it was queued with)
    queued.read_begin()
    extra = wl.random_sequential_addition(200, grid, 1.0, 0.5, 9)
    with pytest.raises(icm.IcmError) as ei:
        queued.add_blobs(extra, np.zeros((200, 3)), np.zeros(200))
    assert ei.value.status == icm.ICM_EBUSY
    assert queued.read_finish()["pos"].shape == (nb, 3)
    queued.add_blobs(extra, np.zeros((200, 3)), np.zeros(200))   # staging grows at the next read
    queued.read_begin()
    assert queued.read_finish()["pos"].shape == (nb + 200, 3)
    for s in sims:
        s.close()
