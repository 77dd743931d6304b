"""Batched replicas and the serving loop: every simulation gives the same result
whether it runs alone or together with others (one graph launch advancing many),
within the parity tolerance, and the server never holds more device memory than
its budget."""
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
    return m


def _jobs(precision, count=5, seed0=40):
    out = []
    for r, (side, kernel, nb) in enumerate([(32, 4, 7), (48, 3, 12), (24, 4, 1), (32, 3, 20), (16, 4, 3)][:count]):
        cfg = dict(grid=(side, side, side), h=1.0, rho=1.0, eta=1.0, kT=2e-3, dt=0.05, kernel=kernel,
                   seed=seed0 + r, precision=precision, steps=4 + r, nblobs=nb, me_range=(-0.5, 2.0),
                   force=(1e-3, 0.0, -2e-3), place_seed=seed0 + 100 + r, min_spacing=2.0)
        out.append(wl._materialise(cfg))
    return out


def _alone(icm, j):
    sim = icm.Simulation(j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"], j["kernel"], j["seed"],
                         j["precision"])
    sim.add_blobs(j["q"], j["u"], j["me"])
    sim.set_forces(j["force"])
    sim.step(j["steps"])
    r = sim.read()
    sim.close()
    return r


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("tune", [False, True])
def test_batch_matches_individual_runs(icm, precision, tune):
    jobs = _jobs(precision, 4)
    sims = []
    for j in jobs:
        s = icm.Simulation(j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"], j["kernel"], j["seed"], precision)
        s.add_blobs(j["q"], j["u"], j["me"])
        s.set_forces(j["force"])
        sims.append(s)
    b = icm.icm_batch_create()
    icm.icm_batch_set(b, [s.handle for s in sims])
    if tune:   # the batch autotuner runs trial steps and restores every member's state
        icm.icm_batch_autotune(b, 2)
        assert all(s.read()["step"] == 0 for s in sims)
    icm.icm_batch_step(b, 5)
    icm.icm_batch_sync(b)
    for j, s in zip(jobs, sims):
        got = s.read()
        assert got["step"] == 5
        j5 = dict(j, steps=5)
        want = _alone(icm, j5)
        assert rel(got["vel"], want["vel"]) < TOL[precision]
        assert rel(got["pos"], want["pos"]) < TOL[precision] * 1e-2
    icm.icm_batch_destroy(b)
    for s in sims:
        s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_server_results_same_alone_and_in_the_mix(icm, precision):
    jobs = _jobs(precision)
    est = [icm.icm_estimate_device_bytes(j["grid"], precision, len(j["q"])) for j in jobs]
    budget = int(sum(sorted(est)[-2:]) * 1.05)           # about two jobs at a time
    sv = icm.icm_server_create(budget, 8)
    ids = []
    peak = 0
    pending = list(jobs)
    done = 0
    pumps = 0
    while done < len(jobs):
        if pending and pumps % 2 == 0:                     # staggered arrivals
            j = pending.pop(0)
            ids.append(icm.icm_server_submit(sv, j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"],
                                             j["kernel"], j["seed"], precision, 0, j["q"], j["u"], j["me"],
                                             j["force"], j["steps"]))
        a, w, f = icm.icm_server_pump(sv, 2)
        peak = max(peak, icm.icm_server_bytes_in_use(sv))
        done += f
        pumps += 1
        time.sleep(0.0002)                               # pumps do not wait for the GPU
        assert pumps < 100000
    assert peak <= budget
    for jid, j in zip(ids, jobs):
        r = icm.icm_server_result(sv, jid, len(j["q"]))
        assert r["state"] == 2 and r["latency_s"] > 0
        want = _alone(icm, j)
        assert rel(r["vel"], want["vel"]) < TOL[precision]
        assert rel(r["pos"], want["pos"]) < TOL[precision] * 1e-2
        np.testing.assert_allclose(r["momentum"], want["momentum"], rtol=1e-9, atol=1e-12)
    icm.icm_server_destroy(sv)


def test_server_rejects_job_larger_than_budget(icm):
    sv = icm.icm_server_create(1 << 20, 4)
    with pytest.raises(icm.IcmError) as ei:
        icm.icm_server_submit(sv, (64, 64, 64), 1.0, 1.0, 1.0, 0.0, 0.05, 4, 1, 32, 0, np.zeros((1, 3)), None,
                              np.zeros(1), None, 3)
    assert ei.value.status == icm.ICM_ENOMEM
    icm.icm_server_destroy(sv)


def _grouped_jobs(precision):
    # (side, h, kernel, blobs, excess mass): three 32^3 members of one group (one
    # neutrally buoyant, so it skips the second and third solves), a 32^3 member with
    # another cell width (a grid of its own: stepped ungrouped), two 48^3 members
    # (a second group), a 24^3 member (no register FFT passes: ungrouped) and two 64^3
    # members (a third group, one of them neutrally buoyant)
    spec = [(32, 1.0, 4, 7, (-0.5, 2.0)), (32, 1.0, 3, 12, None), (32, 1.0, 4, 5, (0.0, 1.0)),
            (32, 0.5, 4, 6, (-0.5, 2.0)), (48, 1.0, 3, 4, (-0.5, 2.0)), (48, 1.0, 4, 9, (-0.5, 2.0)),
            (24, 1.0, 4, 3, (-0.5, 2.0)), (64, 1.0, 4, 8, (-0.5, 2.0)), (64, 1.0, 3, 5, None)]
    out = []
    for r, (side, h, kernel, nb, me_range) in enumerate(spec):
        cfg = dict(grid=(side, side, side), h=h, rho=1.0, eta=1.0, kT=2e-3 * h ** 3, dt=0.05 * h * h, kernel=kernel,
                   seed=70 + r, precision=precision, steps=5, nblobs=nb, me_range=me_range,
                   force=(1e-3, 0.0, -2e-3), place_seed=170 + r, min_spacing=2.0)
        out.append(wl._materialise(cfg))
    return out


@pytest.mark.parametrize("precision", [64, 32])
def test_grouped_batch_matches_individual_runs(icm, precision):
    jobs = _grouped_jobs(precision)
    sims = []
    for j in jobs:
        s = icm.Simulation(j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"], j["kernel"], j["seed"], precision)
        s.add_blobs(j["q"], j["u"], j["me"])
        s.set_forces(j["force"])
        sims.append(s)
    b = icm.icm_batch_create()
    icm.icm_batch_set(b, [s.handle for s in sims])
    assert icm.icm_batch_get_grouped(b) == 0
    icm.icm_batch_set_grouped(b, 1)
    assert icm.icm_batch_get_grouped(b) == 1
    icm.icm_batch_step(b, 2)
    icm.icm_batch_step(b, 3)   # replays the same graph
    icm.icm_batch_sync(b)
    for j, s in zip(jobs, sims):
        got = s.read()
        assert got["step"] == 5
        want = _alone(icm, j)
        assert rel(got["vel"], want["vel"]) < TOL[precision]
        assert rel(got["pos"], want["pos"]) < TOL[precision] * 1e-2
        np.testing.assert_allclose(got["momentum"], want["momentum"], rtol=1e-9, atol=1e-12)
    with pytest.raises(icm.IcmError):
        icm.icm_batch_set_grouped(b, 4)
    icm.icm_batch_destroy(b)
    for s in sims:
        s.close()


def _stage_jobs(precision):
    # (side, h, kernel, blobs, excess mass, kT, trap): register sides only.  Two groups of
    # 32^3 members (one neutrally buoyant, one without blobs), a group of two 48^3
    # members (one without noise), a 64^3 member and a 32^3 member with another cell
    # width (groups of one), one member in a harmonic trap; kernels 3 and 4 mixed.
    spec = [(32, 1.0, 4, 7, (-0.5, 2.0), 2e-3, None), (32, 1.0, 3, 12, None, 2e-3, None),
            (32, 1.0, 4, 0, None, 2e-3, None), (48, 1.0, 3, 4, (-0.5, 2.0), 0.0, None),
            (48, 1.0, 4, 9, (-0.5, 2.0), 2e-3, (0.02, (20.0, 24.0, 30.0))), (64, 1.0, 4, 8, (-0.5, 2.0), 2e-3, None),
            (32, 0.5, 3, 5, (0.0, 1.0), 2.5e-4, None)]
    out = []
    for r, (side, h, kernel, nb, me_range, kT, trap) in enumerate(spec):
        cfg = dict(grid=(side, side, side), h=h, rho=1.0, eta=1.0, kT=kT, dt=0.05 * h * h, kernel=kernel,
                   seed=80 + r, precision=precision, steps=5, nblobs=nb, me_range=me_range,
                   force=(1e-3, 0.0, -2e-3), place_seed=180 + r, min_spacing=2.0)
        j = wl._materialise(cfg)
        j["trap"] = trap
        out.append(j)
    return out


def _make(icm, j, precision):
    s = icm.Simulation(j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"], j["kernel"], j["seed"], precision)
    if len(j["q"]):
        s.add_blobs(j["q"], j["u"], j["me"])
        s.set_forces(j["force"])
    if j.get("trap"):
        s.set_trap(j["trap"][0], j["trap"][1])
    return s


@pytest.mark.parametrize("grouped", [2, 3])
@pytest.mark.parametrize("precision", [64, 32])
def test_batched_stages_match_individual_runs(icm, precision, grouped):
    """Batched stages (grouped = 2): every per-member stage is one launch over all members
    of mixed grids, kernels and blob counts; each member's result equals its run alone.
    With grouped = 3 the same (one member has no blobs: the blob work stays in separate
    launches)."""
    jobs = _stage_jobs(precision)
    sims = [_make(icm, j, precision) for j in jobs]
    b = icm.icm_batch_create()
    icm.icm_batch_set(b, [s.handle for s in sims])
    icm.icm_batch_set_grouped(b, grouped)
    assert icm.icm_batch_get_grouped(b) == grouped
    icm.icm_batch_step(b, 2)
    icm.icm_batch_step(b, 3)   # replays the same graph
    icm.icm_batch_sync(b)
    # 13 stage launches at most (two RHS launches: members with and without noise) and
    # five FFT launches per group and solve (four groups, all with excess mass)
    assert 0 < icm.icm_batch_kernels_per_step(b) <= 13 + 5 * 3 * 4
    for j, s in zip(jobs, sims):
        got = s.read()
        assert got["step"] == 5
        alone = _make(icm, j, precision)
        alone.step(5)
        want = alone.read()
        alone.close()
        if len(j["q"]):
            assert rel(got["vel"], want["vel"]) < TOL[precision]
            assert rel(got["pos"], want["pos"]) < TOL[precision] * 1e-2
        np.testing.assert_allclose(got["momentum"], want["momentum"], rtol=1e-9, atol=1e-12)
    icm.icm_batch_destroy(b)
    for s in sims:
        s.close()


def _blob_stage_jobs(precision):
    # every member with blobs: the blob work runs inside the group x passes.  A neutrally
    # buoyant 32^3 member beside an inertial one, a 48^3 pair (one without noise, one in
    # a harmonic trap), a 64^3 member without forces, a 32^3 member with another cell width.
    spec = [(32, 1.0, 4, 7, (-0.5, 2.0), 2e-3, None, (1e-3, 0.0, -2e-3)),
            (32, 1.0, 3, 12, None, 2e-3, None, (0.0, 2e-3, 0.0)),
            (48, 1.0, 3, 4, (-0.5, 2.0), 0.0, None, (1e-3, 0.0, -2e-3)),
            (48, 1.0, 4, 9, (-0.5, 2.0), 2e-3, (0.02, (20.0, 24.0, 30.0)), (1e-3, 0.0, -2e-3)),
            (64, 1.0, 4, 8, (-0.5, 2.0), 2e-3, None, (0.0, 0.0, 0.0)),
            (32, 0.5, 3, 5, (0.0, 1.0), 2.5e-4, None, (1e-3, 0.0, -2e-3))]
    out = []
    for r, (side, h, kernel, nb, me_range, kT, trap, force) in enumerate(spec):
        cfg = dict(grid=(side, side, side), h=h, rho=1.0, eta=1.0, kT=kT, dt=0.05 * h * h, kernel=kernel,
                   seed=90 + r, precision=precision, steps=5, nblobs=nb, me_range=me_range, force=force,
                   place_seed=190 + r, min_spacing=2.0)
        j = wl._materialise(cfg)
        j["trap"] = trap
        out.append(j)
    return out


@pytest.mark.parametrize("precision", [64, 32])
def test_batched_stages_with_blob_passes_match_individual_runs(icm, precision):
    """Batched stages (grouped = 3) whose members all have blobs on register x sides: the
    spreads and gathers run inside the group x passes (row bins of every member in three
    launches, no separate spread, zeroing or gather launch); each member's result equals
    its run alone."""
    jobs = _blob_stage_jobs(precision)
    sims = [_make(icm, j, precision) for j in jobs]
    b = icm.icm_batch_create()
    icm.icm_batch_set(b, [s.handle for s in sims])
    icm.icm_batch_set_grouped(b, 3)
    icm.icm_batch_step(b, 2)
    icm.icm_batch_step(b, 3)
    icm.icm_batch_sync(b)
    # scalars (2), predictor, bins (3), RHS with and without noise (2), steps 4 and 6-8
    # from the accumulators (2), finish; five FFT launches for each of four groups in
    # each of the three solves
    assert icm.icm_batch_kernels_per_step(b) == 11 + 5 * 4 * 3
    for j, s in zip(jobs, sims):
        got = s.read()
        assert got["step"] == 5
        alone = _make(icm, j, precision)
        alone.step(5)
        want = alone.read()
        alone.close()
        assert rel(got["vel"], want["vel"]) < TOL[precision]
        assert rel(got["pos"], want["pos"]) < TOL[precision] * 1e-2
        np.testing.assert_allclose(got["momentum"], want["momentum"], rtol=1e-9, atol=1e-12)
    icm.icm_batch_destroy(b)
    for s in sims:
        s.close()


def test_batched_stages_fall_back_without_register_sides(icm):
    """A member whose grid has no register FFT passes (24^3): grouped = 2 steps the batch
    as grouped = 1 would, with the same results as the members alone."""
    jobs = _grouped_jobs(64)[5:8]
    sims = [_make(icm, j, 64) for j in jobs]
    b = icm.icm_batch_create()
    icm.icm_batch_set(b, [s.handle for s in sims])
    icm.icm_batch_set_grouped(b, 2)
    icm.icm_batch_step(b, 5)
    icm.icm_batch_sync(b)
    for j, s in zip(jobs, sims):
        want = _alone(icm, j)
        assert rel(s.read()["vel"], want["vel"]) < TOL[64]
    icm.icm_batch_destroy(b)
    for s in sims:
        s.close()


@pytest.mark.parametrize("z_split", [0, 1])
def test_batched_stages_tensor_map_group_matches_individual_runs(icm, z_split):
    """Batched stages with a group on z side 96 (its members' spectra in one buffer, the
    tensor-map z pass over all of them) beside a side-64 group, with either z split: each
    member's result equals its run alone with the same plan."""
    spec = [(96, 4, 9, 201), (96, 3, 5, 202), (64, 4, 7, 203), (64, 3, 4, 204)]
    jobs = []
    for side, kernel, nb, seed in spec:
        cfg = dict(grid=(side, side, side), h=1.0, rho=1.0, eta=1.0, kT=1e-3, dt=0.05, kernel=kernel, seed=seed,
                   precision=32, steps=4, nblobs=nb, me_range=(-0.5, 2.0), force=(1e-3, 0.0, -2e-3),
                   place_seed=seed + 100, min_spacing=2.0)
        j = wl._materialise(cfg)
        j["trap"] = None
        jobs.append(j)
    plan = dict(fused_blobs=1, tma_z=1, rhs_kz=0, fork=1, fused_xy=0, z_split=z_split)
    sims = [_make(icm, j, 32) for j in jobs]
    for s in sims:
        icm.icm_set_plan(s.handle, **plan)
    b = icm.icm_batch_create()
    icm.icm_batch_set(b, [s.handle for s in sims])
    icm.icm_batch_set_grouped(b, 2)
    icm.icm_batch_step(b, 4)
    icm.icm_batch_sync(b)
    for j, s in zip(jobs, sims):
        got = s.read()
        alone = _make(icm, j, 32)
        icm.icm_set_plan(alone.handle, **plan)
        alone.step(4)
        want = alone.read()
        alone.close()
        assert got["step"] == 4
        assert rel(got["vel"], want["vel"]) < TOL[32]
        assert rel(got["pos"], want["pos"]) < TOL[32] * 1e-2
        np.testing.assert_allclose(got["momentum"], want["momentum"], rtol=1e-9, atol=1e-12)
    icm.icm_batch_destroy(b)
    for s in sims:
        s.close()
