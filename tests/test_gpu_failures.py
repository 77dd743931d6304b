"""Failure detection in forms that fault, trap or hang no GPU.

* A bounded device-side wait that runs out: a one-thread kernel arms an mbarrier for a
  transaction that is never issued and waits with the bounded wait of the TMA z pass
  (1 ms here); the host sees ICM_ETIMEOUT at its next icm_sync and the context keeps
  working.
* Device allocations refused by the caller's allocator (a host-side allocator that
  returns NULL on its k-th call): icm_create, icm_add_blobs and icm_autotune report
  ICM_ENOMEM and leave nothing allocated behind; the server keeps a job it cannot place
  waiting and places it at a later pump.
* Jobs withdrawn from the server between pumps (icm_server_cancel): the other jobs'
  results are those they have alone."""
import time

import numpy as np
import pytest

import icm_workloads as wl

from _gpu_helpers import TOL, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icm():
    from paper_1212_6427_gb300 import build
    build.build_library()
    import paper_1212_6427_gb300 as m
    m.use_torch_allocator()
    yield m
    m.use_torch_allocator()


class RefusingAllocator:
    """Device memory from torch's caching allocator, counting every request and refusing
    (returning NULL for) the fail_at-th one; `live` holds what is allocated now."""

    def __init__(self, icm):
        import torch
        self.icm = icm
        self.calls = 0
        self.fail_at = None
        self.live = {}

        def _alloc(ctx, nbytes, stream):
            self.calls += 1
            if self.fail_at is not None and self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            self.live[p] = int(nbytes)
            return p

        def _free(ctx, ptr, stream):
            self.live.pop(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.fa = icm.binding._ALLOC_T(_alloc)
        self.ff = icm.binding._FREE_T(_free)

    def install(self):
        self.icm.binding._check(self.icm.lib().icm_set_default_allocator(self.fa, self.ff, None))

    def arm(self, k):
        self.calls = 0
        self.fail_at = k

    def bytes(self):
        return sum(self.live.values())


_KEEP = []   # simulations keep the allocator's function pointers: they outlive every test


@pytest.fixture()
def refusing(icm):
    a = RefusingAllocator(icm)
    _KEEP.append(a)
    a.install()
    yield a
    icm.use_torch_allocator()


GRID = (32, 16, 12)   # x side 32: blob work inside the x passes, so add_blobs allocates bins too


def _create(icm, precision=64, grid=GRID):
    return icm.icm_create(grid, 1.0, 1.0, 1.0, 1e-3, 0.05, 4, 5, precision, 0, None)


def _blobs(n=6, seed=3, grid=GRID):
    q = wl.random_sequential_addition(n, grid, 1.0, 2.0, seed)
    rng = np.random.default_rng(seed)
    return q, 0.01 * rng.standard_normal((n, 3)), rng.uniform(-0.5, 2.0, size=n)


def test_bounded_wait_timeout_is_reported_and_the_context_stays_usable(icm):
    sim = icm.Simulation(GRID, 1.0, 1.0, 1.0, 1e-3, 0.05, 4, 5, 32)
    q, u, me = _blobs()
    sim.add_blobs(q, u, me)
    sim.step(2)
    sim.sync()
    t0 = time.perf_counter()
    icm.icm_debug_wait_timeout(sim.handle, 1_000_000)        # 1 ms
    with pytest.raises(icm.IcmError) as ei:
        sim.sync()
    assert ei.value.status == icm.ICM_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    sim.sync()                                                 # the report cleared the bit
    sim.close()                                                # destroyed cleanly
    fresh = icm.Simulation(GRID, 1.0, 1.0, 1.0, 1e-3, 0.05, 4, 5, 32)
    fresh.add_blobs(q, u, me)
    fresh.step(3)
    r = fresh.read(fluid=True)
    assert r["step"] == 3 and np.isfinite(r["fluid"]).all() and np.isfinite(r["vel"]).all()
    fresh.close()
    with pytest.raises(icm.IcmError):
        icm.icm_debug_wait_timeout(None, 1000)


def test_create_reports_enomem_and_leaks_nothing(icm, refusing):
    h = _create(icm)
    n_alloc = refusing.calls
    assert n_alloc >= 9
    assert refusing.bytes() == icm.icm_device_bytes(h)
    icm.icm_destroy(h)
    assert refusing.live == {}
    for k in sorted({1, 2, 4, n_alloc // 2, n_alloc - 1, n_alloc}):
        refusing.arm(k)
        with pytest.raises(icm.IcmError) as ei:
            _create(icm)
        assert ei.value.status == icm.ICM_ENOMEM, k
        assert refusing.live == {}, k


def test_add_blobs_and_autotune_report_enomem_and_keep_the_simulation(icm, refusing):
    h = _create(icm)
    q, u, me = _blobs()
    before = icm.icm_device_bytes(h)
    for k in (1, 2):                      # the blob arrays, then the fused-pass bins
        refusing.arm(k)
        with pytest.raises(icm.IcmError) as ei:
            icm.icm_add_blobs(h, q, u, me)
        assert ei.value.status == icm.ICM_ENOMEM
        assert icm.icm_device_bytes(h) == before == refusing.bytes()
        assert icm.icm_num_blobs(h) == 0
    refusing.arm(None)
    icm.icm_add_blobs(h, q, u, me)
    icm.icm_step(h, 2)
    ref = icm.icm_read_state(h, int(np.prod(GRID)))
    with_blobs = icm.icm_device_bytes(h)
    for k in (1, 2, 3, 4):                # the autotuner's four state-copy buffers
        refusing.arm(k)
        with pytest.raises(icm.IcmError) as ei:
            icm.icm_autotune(h, 1)
        assert ei.value.status == icm.ICM_ENOMEM
        assert icm.icm_device_bytes(h) == with_blobs == refusing.bytes()
        again = icm.icm_read_state(h, int(np.prod(GRID)))
        assert again[4] == ref[4] == 2                     # no step was taken
        assert np.array_equal(again[0], ref[0]) and np.array_equal(again[1], ref[1])
    refusing.arm(None)
    icm.icm_step(h, 1)
    assert icm.icm_read_state(h, int(np.prod(GRID)))[4] == 3
    icm.icm_destroy(h)
    assert refusing.live == {}


def _job(precision, side, kernel, nb, seed, steps):
    cfg = dict(grid=(side, side, side), h=1.0, rho=1.0, eta=1.0, kT=2e-3, dt=0.05, kernel=kernel, seed=seed,
               precision=precision, steps=steps, nblobs=nb, me_range=(-0.5, 2.0), force=(1e-3, 0.0, -2e-3),
               place_seed=seed + 100, min_spacing=2.0)
    return wl._materialise(cfg)


def _submit(icm, sv, j):
    return icm.icm_server_submit(sv, j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"], j["kernel"], j["seed"],
                                 j["precision"], 0, j["q"], j["u"], j["me"], j["force"], j["steps"])


def _alone(icm, j):
    sim = icm.Simulation(j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"], j["kernel"], j["seed"],
                         j["precision"])
    sim.add_blobs(j["q"], j["u"], j["me"])
    sim.set_forces(j["force"])
    sim.step(j["steps"])
    r = sim.read()
    sim.close()
    return r


def _drain(icm, sv, njobs, k=2):
    done, pumps = 0, 0
    while done < njobs:
        _, _, f = icm.icm_server_pump(sv, k)
        done += f
        pumps += 1
        time.sleep(0.0002)
        assert pumps < 100000


def test_server_keeps_a_job_it_cannot_place_waiting(icm, refusing):
    jobs = [_job(64, 16, 4, 5, 61, 6), _job(64, 24, 3, 9, 62, 5)]
    sv = icm.icm_server_create(10 ** 10, 4)
    ids = [_submit(icm, sv, j) for j in jobs]
    refusing.arm(3)                                   # the first job's third allocation
    a, w, f = icm.icm_server_pump(sv, 2)
    assert (a, w, f) == (0, 2, 0)
    assert icm.icm_server_bytes_in_use(sv) == 0 and refusing.live == {}
    assert icm.icm_server_result(sv, ids[0], len(jobs[0]["q"]))["state"] == 0
    refusing.arm(None)
    _drain(icm, sv, len(jobs))
    assert icm.icm_server_bytes_in_use(sv) == 0
    results = [icm.icm_server_result(sv, i, len(j["q"])) for i, j in zip(ids, jobs)]
    icm.icm_server_destroy(sv)
    assert refusing.live == {}
    icm.use_torch_allocator()
    for r, j in zip(results, jobs):
        assert r["state"] == 2
        want = _alone(icm, j)
        assert rel(r["vel"], want["vel"]) < TOL[64]
        np.testing.assert_allclose(r["momentum"], want["momentum"], rtol=1e-12, atol=1e-14)


def test_server_cancel_leaves_the_other_jobs_unchanged(icm):
    jobs = [_job(64, 16, 4, 5, 71, 30), _job(64, 24, 3, 9, 72, 30), _job(64, 16, 3, 4, 73, 12),
            _job(64, 12, 4, 3, 74, 10)]
    sv = icm.icm_server_create(10 ** 10, 2)
    ids = [_submit(icm, sv, j) for j in jobs]
    a, w, f = icm.icm_server_pump(sv, 2)
    assert (a, w) == (2, 2)
    icm.icm_server_cancel(sv, ids[1])                 # active
    icm.icm_server_cancel(sv, ids[2])                 # waiting
    with pytest.raises(icm.IcmError):
        icm.icm_server_cancel(sv, 12345)
    _drain(icm, sv, 2)
    assert icm.icm_server_bytes_in_use(sv) == 0
    states = [icm.icm_server_result(sv, i, len(j["q"]))["state"] for i, j in zip(ids, jobs)]
    assert states == [2, 4, 4, 2]
    icm.icm_server_cancel(sv, ids[0])                 # finished: left as it is
    for i in (0, 3):
        r = icm.icm_server_result(sv, ids[i], len(jobs[i]["q"]))
        assert r["state"] == 2
        want = _alone(icm, jobs[i])
        assert rel(r["vel"], want["vel"]) < TOL[64]
        assert rel(r["pos"], want["pos"]) < TOL[64]
    icm.icm_server_destroy(sv)
