"""Thin ctypes binding of libicm (include/icm.h): same names, argument marshalling only.

Every step of the method runs in the CUDA library.  There is no CPU fallback:
if libicm.so is missing or cannot be loaded, every call raises.

PyTorch provides the device memory (its caching allocator, installed as the
library's allocator by `use_torch_allocator`) and the CUDA stream of each
simulation (`Simulation` creates a torch.cuda.Stream unless given one).
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# ICM_CHECKED=1 in the environment loads the checked build (device-side index checks,
# paper_1212_6427_gb300.build.build_library(checked=True)) instead of the ordinary one.
LIB_PATH = os.path.join(_PKG, "libicm_checked.so" if os.environ.get("ICM_CHECKED") == "1" else "libicm.so")

ICM_OK, ICM_EINVAL, ICM_ENOMEM, ICM_ECUDA, ICM_ECFL, ICM_ENONFINITE, ICM_ETIMEOUT, ICM_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
ICM_EINDEX = -8
STATUS_NAMES = {0: "ICM_OK", -1: "ICM_EINVAL", -2: "ICM_ENOMEM", -3: "ICM_ECUDA", -4: "ICM_ECFL",
                -5: "ICM_ENONFINITE", -6: "ICM_ETIMEOUT", -7: "ICM_EBUSY", -8: "ICM_EINDEX"}
FLAG_NO_ADVECTION, FLAG_SLIP_VISC, FLAG_SLIP_ZERO, FLAG_SLIP_FULL = 0x1, 0x0, 0x2, 0x4
FLAG_THERMAL_DRIFT = 0x8

# name -> (restype, argtypes)
_c_d = ctypes.c_double
_c_i32 = ctypes.c_int32
_c_i64 = ctypes.c_int64
_c_u32 = ctypes.c_uint32
_c_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

class Plan(ctypes.Structure):
    """icm_plan of include/icm.h."""
    _fields_ = [("fused_blobs", _c_i32), ("tma_z", _c_i32), ("rhs_kz", _c_i32), ("fork", _c_i32),
                ("fused_xy", _c_i32), ("z_split", _c_i32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class JobDesc(ctypes.Structure):
    """icm_job_desc of include/icm.h."""
    _fields_ = [("grid", _c_i32 * 3), ("h", _c_d), ("rho", _c_d), ("eta", _c_d), ("kT", _c_d), ("dt", _c_d),
                ("kernel", _c_i32), ("seed", _c_u64), ("precision", _c_i32), ("flags", _c_i32),
                ("nblobs", _c_i64), ("pos", _dp), ("vel", _dp), ("excess_mass", _dp), ("force", _dp),
                ("nsteps", _c_i64)]


SIGNATURES = {
    "icm_set_default_allocator": (_c_i32, [_ALLOC_T, _FREE_T, _vp]),
    "icm_create": (_c_i32, [ctypes.POINTER(_c_i32), _c_d, _c_d, _c_d, _c_d, _c_d, _c_i32, _c_u64, _c_i32, _c_i32,
                            _vp, ctypes.POINTER(_vp)]),
    "icm_destroy": (None, [_vp]),
    "icm_last_error": (ctypes.c_char_p, []),
    "icm_add_blobs": (_c_i32, [_vp, _c_i64, _dp, _dp, _dp]),
    "icm_set_blob_forces": (_c_i32, [_vp, _dp]),
    "icm_set_blob_trap": (_c_i32, [_vp, ctypes.c_double, _dp]),
    "icm_get_plan": (_c_i32, [_vp, ctypes.c_void_p]),
    "icm_set_plan": (_c_i32, [_vp, ctypes.c_void_p]),
    "icm_autotune": (_c_i32, [_vp, _c_i32, ctypes.c_void_p, _dp]),
    "icm_batch_autotune": (_c_i32, [_vp, _c_i32]),
    "icm_batch_set_grouped": (_c_i32, [_vp, _c_i32]),
    "icm_batch_get_grouped": (_c_i32, [_vp]),
    "icm_batch_kernels_per_step": (_c_i64, [_vp]),
    "icm_set_blob_wca": (_c_i32, [_vp, ctypes.c_double, ctypes.c_double]),
    "icm_step": (_c_i32, [_vp, _c_i64]),
    "icm_sync": (_c_i32, [_vp]),
    "icm_read_state": (_c_i32, [_vp, _dp, _dp, _dp, _dp, ctypes.POINTER(_c_i64)]),
    "icm_read_begin": (_c_i32, [_vp]),
    "icm_read_finish": (_c_i32, [_vp, _dp, _dp, _dp, ctypes.POINTER(_c_i64)]),
    "icm_write_state": (_c_i32, [_vp, _dp, _dp, _dp, _dp, _dp, _c_i64]),
    "icm_read_aux": (_c_i32, [_vp, _dp, _dp, ctypes.POINTER(_c_i32)]),
    "icm_profile_steps": (_c_i32, [_vp, _c_i64, _c_i32, ctypes.POINTER(_c_i32), ctypes.c_char_p, _dp, _dp]),
    "icm_fluid_momentum_static": (_c_i32, [_vp, _c_i32, _c_i64, _c_d, _c_d, _vp, _dp]),
    "icm_num_blobs": (_c_i64, [_vp]),
    "icm_kernel_volume": (_c_i32, [_c_i32, _c_d, _dp]),
    "icm_peak_fma": (_c_i32, [_c_i32, _vp, _dp]),
    "icm_batch_create": (_c_i32, [_vp, ctypes.POINTER(_vp)]),
    "icm_batch_set": (_c_i32, [_vp, _c_i32, ctypes.POINTER(_vp)]),
    "icm_batch_step": (_c_i32, [_vp, _c_i64]),
    "icm_batch_sync": (_c_i32, [_vp]),
    "icm_batch_destroy": (None, [_vp]),
    "icm_estimate_device_bytes": (_c_i64, [ctypes.POINTER(_c_i32), _c_i32, _c_i64]),
    "icm_server_create": (_c_i32, [_c_i64, _c_i32, ctypes.POINTER(_vp)]),
    "icm_server_submit": (_c_i32, [_vp, ctypes.POINTER(JobDesc), ctypes.POINTER(_c_i64)]),
    "icm_server_pump": (_c_i32, [_vp, _c_i32, ctypes.POINTER(_c_i32), ctypes.POINTER(_c_i32), ctypes.POINTER(_c_i32)]),
    "icm_server_result": (_c_i32, [_vp, _c_i64, ctypes.POINTER(_c_i32), _dp, _dp, _dp, _dp]),
    "icm_server_bytes_in_use": (_c_i64, [_vp]),
    "icm_server_cancel": (_c_i32, [_vp, _c_i64]),
    "icm_debug_wait_timeout": (_c_i32, [_vp, _c_i64]),
    "icm_server_destroy": (None, [_vp]),
    "icm_device_bytes": (_c_i64, [_vp]),
    "icm_op_interpolate": (_c_i32, [_vp, _c_i64, _dp, _dp, _dp]),
    "icm_op_interpolate_laplacian": (_c_i32, [_vp, _c_i64, _dp, _dp, _dp]),
    "icm_op_spread": (_c_i32, [_vp, _c_i64, _dp, _dp, _dp]),
    "icm_op_spectral_solve": (_c_i32, [_vp, _c_d, _c_d, _dp, _dp]),
    "icm_op_coupling": (_c_i32, [_vp, _c_i64, _dp, _dp, _c_d, _c_d, _dp]),
    "icm_op_explicit_rhs": (_c_i32, [_vp, _dp, _dp, _c_i64, _dp, _dp]),
    "icm_op_stress_normals": (_c_i32, [_vp, _c_i64, _dp]),
    "icm_op_philox": (_c_i32, [_c_i64, _c_u32, _c_u32, _c_u32, _c_u32, _c_u32, _c_u32, ctypes.POINTER(_c_u32)]),
}

_lib = None
_keep = []


class IcmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


def lib():
    """Load libicm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built; run paper_1212_6427_gb300.build.build_library()"
                               % os.path.basename(LIB_PATH))
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != ICM_OK:
        raise IcmError(status, lib().icm_last_error().decode())


def _f64(a, n=None):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and arr.size != n:
        raise ValueError("expected %d values, got %d" % (n, arr.size))
    return arr, arr.ctypes.data_as(_dp)


def _out(n):
    arr = np.empty(n, dtype=np.float64)
    return arr, arr.ctypes.data_as(_dp)


# ---------------------------------------------------------------------------
# Allocator: torch's caching allocator provides the library's device memory.
# ---------------------------------------------------------------------------
def use_torch_allocator():
    """Install torch's caching allocator as the library's allocator, once per process.

    Simulations keep the function pointers they were created with, so the ctypes
    thunks must live as long as the process: they are created once and never replaced."""
    if _keep:
        _check(lib().icm_set_default_allocator(_keep[0], _keep[1], None))
        return
    import torch

    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory -> the library reports ICM_ENOMEM
            return None

    def _free(ctx, ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = _ALLOC_T(_alloc), _FREE_T(_free)
    _keep[:] = [fa, ff]
    _check(lib().icm_set_default_allocator(fa, ff, None))


def use_cuda_malloc():
    """Simulations created afterwards use cudaMalloc/cudaFree (existing ones keep theirs)."""
    _check(lib().icm_set_default_allocator(_ALLOC_T(), _FREE_T(), None))


# ---------------------------------------------------------------------------
# C-ABI functions, same names
# ---------------------------------------------------------------------------
def icm_create(grid, h, rho, eta, kT, dt, kernel, seed, precision=32, flags=0, cuda_stream=None):
    g = (_c_i32 * 3)(*[int(x) for x in grid])
    out = _vp()
    _check(lib().icm_create(g, h, rho, eta, kT, dt, int(kernel), int(seed) & 0xFFFFFFFFFFFFFFFF, int(precision),
                            int(flags), cuda_stream, ctypes.byref(out)))
    return out


def icm_destroy(sim):
    lib().icm_destroy(sim)


def icm_last_error():
    return lib().icm_last_error().decode()


def icm_add_blobs(sim, pos, vel, excess_mass):
    p, pp = _f64(pos)
    n = p.size // 3
    _, vp = _f64(vel, 3 * n)
    _, mp = _f64(excess_mass, n)
    _check(lib().icm_add_blobs(sim, n, pp, vp, mp))


def icm_set_blob_forces(sim, force):
    f, fp = _f64(force)
    _check(lib().icm_set_blob_forces(sim, fp))


def icm_set_blob_trap(sim, k, center):
    c = np.ascontiguousarray(center, dtype=np.float64).reshape(3)
    _check(lib().icm_set_blob_trap(sim, float(k), c.ctypes.data_as(_dp)))


def icm_set_blob_wca(sim, epsilon, sigma):
    _check(lib().icm_set_blob_wca(sim, float(epsilon), float(sigma)))


def icm_get_plan(sim):
    p = Plan()
    _check(lib().icm_get_plan(sim, ctypes.byref(p)))
    return p.as_dict()


def icm_set_plan(sim, fused_blobs=1, tma_z=1, rhs_kz=16, fork=1, fused_xy=0, z_split=0):
    p = Plan(int(fused_blobs), int(tma_z), int(rhs_kz), int(fork), int(fused_xy), int(z_split))
    _check(lib().icm_set_plan(sim, ctypes.byref(p)))


def icm_autotune(sim, nsteps=3):
    """Tune the plan; returns (plan dict, ms per step of the chosen plan)."""
    p = Plan()
    ms = ctypes.c_double(0.0)
    _check(lib().icm_autotune(sim, int(nsteps), ctypes.byref(p), ctypes.byref(ms)))
    return p.as_dict(), ms.value


def icm_batch_autotune(batch, nsteps=3):
    _check(lib().icm_batch_autotune(batch, int(nsteps)))


def icm_batch_set_grouped(batch, grouped):
    _check(lib().icm_batch_set_grouped(batch, int(grouped)))


def icm_batch_get_grouped(batch):
    return int(lib().icm_batch_get_grouped(batch))


def icm_batch_kernels_per_step(batch):
    return int(lib().icm_batch_kernels_per_step(batch))


def icm_step(sim, nsteps=1):
    _check(lib().icm_step(sim, int(nsteps)))


def icm_sync(sim):
    _check(lib().icm_sync(sim))


def icm_debug_wait_timeout(sim, limit_ns):
    _check(lib().icm_debug_wait_timeout(sim, int(limit_ns)))


def icm_profile_steps(sim, nsteps, max_stages=128):
    """[(stage name, total ms over nsteps, algorithmic bytes per launch)] of one step's launches."""
    n = _c_i32()
    names = ctypes.create_string_buffer(32 * max_stages)
    ms, mp = _out(max_stages)
    by, bp = _out(max_stages)
    _check(lib().icm_profile_steps(sim, int(nsteps), max_stages, ctypes.byref(n), names, mp, bp))
    raw = names.raw
    out = []
    for i in range(n.value):
        nm = raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out.append((nm, float(ms[i]), float(by[i])))
    return out


def icm_fluid_momentum_static(fluid_v_dev_ptr, precision, ncell, rho, h, cuda_stream=None):
    """rho h^3 sum v of a device face field, computed without any device allocation."""
    out, op = _out(3)
    _check(lib().icm_fluid_momentum_static(ctypes.c_void_p(int(fluid_v_dev_ptr)), int(precision), int(ncell),
                                           float(rho), float(h), cuda_stream, op))
    return out


def icm_peak_fma(precision=64, cuda_stream=None):
    """Measured FMA throughput of the current device in flop/s (FP32 or FP64)."""
    out, op = _out(1)
    _check(lib().icm_peak_fma(int(precision), cuda_stream, op))
    return float(out[0])


def icm_kernel_volume(kernel, h=1.0):
    """dV = h^3 / (sum phi^2)^3 of the Peskin kernel, as the library computes it."""
    out, op = _out(1)
    _check(lib().icm_kernel_volume(int(kernel), float(h), op))
    return float(out[0])


def icm_num_blobs(sim):
    return int(lib().icm_num_blobs(sim))


def icm_device_bytes(sim):
    return int(lib().icm_device_bytes(sim))


def icm_read_state(sim, ncell, fluid=False, check=True):
    """Returns (pos (n,3), vel (n,3), fluid_v (3N,) or None, momentum (3,), step, status)."""
    nb = icm_num_blobs(sim)
    pos, pp = _out(3 * nb)
    vel, vp = _out(3 * nb)
    mom, mp = _out(3)
    if fluid:
        fv, fp = _out(3 * ncell)
    else:
        fv, fp = None, None
    step = _c_i64()
    st = lib().icm_read_state(sim, pp, vp, fp, mp, ctypes.byref(step))
    if check:
        _check(st)
    return pos.reshape(nb, 3), vel.reshape(nb, 3), fv, mom, int(step.value), st


def icm_read_begin(sim):
    _check(lib().icm_read_begin(sim))


def icm_read_finish(sim, check=True):
    """The oldest queued read: (pos (n,3), vel (n,3), momentum (3,), step, status)."""
    nb = icm_num_blobs(sim)
    pos, pp = _out(3 * nb)
    vel, vp = _out(3 * nb)
    mom, mp = _out(3)
    step = _c_i64()
    st = lib().icm_read_finish(sim, pp, vp, mp, ctypes.byref(step))
    if check:
        _check(st)
    return pos.reshape(nb, 3), vel.reshape(nb, 3), mom, int(step.value), st


def icm_write_state(sim, pos, vel, fluid_v, adv_prev=None, slip_g=None, step=0):
    nb = icm_num_blobs(sim)
    _, pp = _f64(pos, 3 * nb)
    _, vp = _f64(vel, 3 * nb)
    fv, fp = _f64(fluid_v)
    _, ap = _f64(adv_prev, fv.size)
    _, gp = _f64(slip_g, 3 * nb)
    _check(lib().icm_write_state(sim, pp, vp, fp, ap, gp, int(step)))


def icm_read_aux(sim, ncell):
    nb = icm_num_blobs(sim)
    adv, ap = _out(3 * ncell)
    g, gp = _out(3 * nb)
    hist = _c_i32()
    _check(lib().icm_read_aux(sim, ap, gp, ctypes.byref(hist)))
    return adv, g.reshape(nb, 3), int(hist.value)


def icm_op_interpolate(sim, pos, fluid_v):
    p, pp = _f64(pos)
    n = p.size // 3
    _, fp = _f64(fluid_v)
    out, op = _out(3 * n)
    _check(lib().icm_op_interpolate(sim, n, pp, fp, op))
    return out.reshape(n, 3)


def icm_op_interpolate_laplacian(sim, pos, fluid_v):
    p, pp = _f64(pos)
    n = p.size // 3
    _, fp = _f64(fluid_v)
    out, op = _out(3 * n)
    _check(lib().icm_op_interpolate_laplacian(sim, n, pp, fp, op))
    return out.reshape(n, 3)


def icm_op_spread(sim, ncell, pos, force):
    p, pp = _f64(pos)
    n = p.size // 3
    _, fp = _f64(force, 3 * n)
    out, op = _out(3 * ncell)
    _check(lib().icm_op_spread(sim, n, pp, fp, op))
    return out


def icm_op_spectral_solve(sim, a, b, rhs):
    r, rp = _f64(rhs)
    out, op = _out(r.size)
    _check(lib().icm_op_spectral_solve(sim, float(a), float(b), rp, op))
    return out


def icm_op_coupling(sim, qi, qj, a, b):
    """(n, 3, 3) matrices J(qi) (a - b L)^-1 P S(qj) of each pair of positions."""
    qi = np.ascontiguousarray(qi, dtype=np.float64).reshape(-1, 3)
    qj = np.ascontiguousarray(qj, dtype=np.float64).reshape(-1, 3)
    n = qi.shape[0]
    if qj.shape[0] != n:
        raise ValueError("qi and qj must have the same number of positions")
    out, op = _out(9 * n)
    _check(lib().icm_op_coupling(sim, n, qi.ctypes.data_as(_dp), qj.ctypes.data_as(_dp), float(a), float(b), op))
    return out.reshape(n, 3, 3)


def icm_op_explicit_rhs(sim, fluid_v, adv_prev, step):
    fv, fp = _f64(fluid_v)
    _, ap = _f64(adv_prev, fv.size)
    r, rp = _out(fv.size)
    a, aq = _out(fv.size)
    _check(lib().icm_op_explicit_rhs(sim, fp, ap, int(step), rp, aq))
    return r, a


def icm_op_stress_normals(sim, ncell, step):
    out, op = _out(6 * ncell)
    _check(lib().icm_op_stress_normals(sim, int(step), op))
    return out.reshape(6, ncell)


def icm_op_philox(n, ctr, key):
    out = np.empty(4 * max(int(n), 0), dtype=np.uint32)
    _check(lib().icm_op_philox(int(n), *[int(c) & 0xFFFFFFFF for c in ctr], *[int(k) & 0xFFFFFFFF for k in key],
                               out.ctypes.data_as(ctypes.POINTER(_c_u32))))
    return out.reshape(-1, 4)


def icm_batch_create(cuda_stream=None):
    out = _vp()
    _check(lib().icm_batch_create(cuda_stream, ctypes.byref(out)))
    return out


def icm_batch_set(batch, sims):
    arr = (_vp * max(1, len(sims)))(*[s.value if isinstance(s, _vp) else s for s in sims])
    _check(lib().icm_batch_set(batch, len(sims), arr))


def icm_batch_step(batch, nsteps=1):
    _check(lib().icm_batch_step(batch, int(nsteps)))


def icm_batch_sync(batch):
    _check(lib().icm_batch_sync(batch))


def icm_batch_destroy(batch):
    lib().icm_batch_destroy(batch)


def icm_estimate_device_bytes(grid, precision, nblobs):
    g = (_c_i32 * 3)(*[int(x) for x in grid])
    return int(lib().icm_estimate_device_bytes(g, int(precision), int(nblobs)))


def icm_server_create(hbm_budget_bytes, max_active):
    out = _vp()
    _check(lib().icm_server_create(int(hbm_budget_bytes), int(max_active), ctypes.byref(out)))
    return out


def icm_server_submit(server, grid, h, rho, eta, kT, dt, kernel, seed, precision, flags, pos, vel, excess_mass,
                      force, nsteps):
    p, pp = _f64(pos)
    n = p.size // 3
    _, vp = _f64(vel, 3 * n)
    m, mp = _f64(excess_mass, n)
    _, fp = _f64(force, 3 * n)
    d = JobDesc((_c_i32 * 3)(*[int(x) for x in grid]), h, rho, eta, kT, dt, int(kernel),
                int(seed) & 0xFFFFFFFFFFFFFFFF, int(precision), int(flags), n, pp, vp, mp, fp, int(nsteps))
    jid = _c_i64()
    _check(lib().icm_server_submit(server, ctypes.byref(d), ctypes.byref(jid)))
    return int(jid.value)


def icm_server_pump(server, steps_per_pump=1):
    a, w, f = _c_i32(), _c_i32(), _c_i32()
    _check(lib().icm_server_pump(server, int(steps_per_pump), ctypes.byref(a), ctypes.byref(w), ctypes.byref(f)))
    return int(a.value), int(w.value), int(f.value)


def icm_server_result(server, job_id, nblobs):
    st = _c_i32()
    pos, pp = _out(3 * nblobs)
    vel, vp = _out(3 * nblobs)
    mom, mp = _out(3)
    lat, lp = _out(1)
    _check(lib().icm_server_result(server, int(job_id), ctypes.byref(st), pp, vp, mp, lp))
    return dict(state=int(st.value), pos=pos.reshape(nblobs, 3), vel=vel.reshape(nblobs, 3), momentum=mom,
                latency_s=float(lat[0]))


def icm_server_bytes_in_use(server):
    return int(lib().icm_server_bytes_in_use(server))


def icm_server_cancel(server, job_id):
    _check(lib().icm_server_cancel(server, int(job_id)))


def icm_server_destroy(server):
    lib().icm_server_destroy(server)


# ---------------------------------------------------------------------------
# Convenience owner of one simulation (still only marshalling)
# ---------------------------------------------------------------------------
class Simulation:
    """One ICM simulation on the GPU: device memory from torch's caching allocator,
    work on a dedicated torch.cuda.Stream."""

    def __init__(self, grid, h=1.0, rho=1.0, eta=1.0, kT=0.0, dt=0.05, kernel=4, seed=1, precision=32, flags=0,
                 stream=None):
        import torch
        use_torch_allocator()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.grid = tuple(int(x) for x in grid)
        self.ncell = int(np.prod(self.grid))
        self.precision = precision
        self.handle = icm_create(self.grid, h, rho, eta, kT, dt, kernel, seed, precision, flags,
                                 ctypes.c_void_p(self.stream.cuda_stream))

    def close(self):
        if self.handle is not None:
            icm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_blobs(self, pos, vel=None, excess_mass=None):
        n = np.asarray(pos).size // 3
        icm_add_blobs(self.handle, pos, vel, np.zeros(n) if excess_mass is None else excess_mass)

    def set_forces(self, force):
        icm_set_blob_forces(self.handle, force)

    def set_trap(self, k, center):
        icm_set_blob_trap(self.handle, k, center)

    def set_wca(self, epsilon, sigma):
        icm_set_blob_wca(self.handle, epsilon, sigma)

    def step(self, n=1):
        icm_step(self.handle, n)

    def sync(self):
        icm_sync(self.handle)

    def read(self, fluid=False):
        pos, vel, fv, mom, step, _ = icm_read_state(self.handle, self.ncell, fluid)
        return dict(pos=pos, vel=vel, fluid=fv, momentum=mom, step=step)

    def read_begin(self):
        icm_read_begin(self.handle)

    def read_finish(self):
        pos, vel, mom, step, _ = icm_read_finish(self.handle)
        return dict(pos=pos, vel=vel, momentum=mom, step=step)

    def write(self, pos, vel, fluid_v, adv_prev=None, slip_g=None, step=0):
        icm_write_state(self.handle, pos, vel, fluid_v, adv_prev, slip_g, step)

    def read_aux(self):
        return icm_read_aux(self.handle, self.ncell)

    def profile(self, nsteps):
        return icm_profile_steps(self.handle, nsteps)
