"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module holds only input recipes (grid sizes, physical parameters, blob
placement, masses, initial velocities): none of the method's arithmetic.  Both
the oracle and the CUDA library are fed from it; neither is imported here.

The paper's runs use no dataset; every workload below is synthetic, with the
sizes and distributions of the five configurations the library is measured on:
  plain  : 32^3, FP64, one neutrally buoyant blob, 4-point kernel, kT = 1e-3, dt = 0.05
  bulk   : 128^3, FP32, 2000 blobs (min spacing 2h), 3-point, m_e ~ U[-0.5, 2] rho h^3
  large  : 256^3, FP32, 20000 blobs (min spacing 2h), 4-point, F = (1e-4, 0, 0), dt = 0.01
  batch  : replicas of side {32, 48, 64, 96}, 1..500 blobs, kernel 3 or 4
  served : Poisson arrivals (mean 50/s), sides 32..128, 1..2000 blobs, kT ~ U[1e-4, 1e-2]
"""
import numpy as np

# The incompressible dragged fluid mass m~_f of a blob in units of rho h^3, a plain
# number per kernel, used only to size the initial velocity spread of the recipes:
# 12 for the 3-point kernel (3/2 of the blob volume 8 h^3 the paper gives) and
# 768/27 for the 4-point kernel (3/2 of its volume (8/3)^3 h^3).
DRAGGED_MASS_PER_RHO_H3 = {3: 12.0, 4: 768.0 / 27.0}


def random_sequential_addition(n, grid, h, min_spacing, seed, max_tries=200):
    """n points uniform in the periodic box, no two closer than min_spacing.

    Uses a cell hash of side >= min_spacing; raises if the box is too full.
    """
    rng = np.random.default_rng(seed)
    box = np.asarray(grid, dtype=np.float64) * h
    if n == 0:
        return np.zeros((0, 3))
    ncell = np.maximum((box // min_spacing).astype(int), 1)
    csize = box / ncell
    buckets = {}
    pts = np.zeros((n, 3))
    placed = 0
    tries = 0
    while placed < n:
        tries += 1
        if tries > max_tries * n + 1000:
            raise RuntimeError("random sequential addition: box too dense")
        p = rng.uniform(0.0, 1.0, size=3) * box
        c = (p // csize).astype(int) % ncell
        ok = True
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    key = tuple((c + (dx, dy, dz)) % ncell)
                    for idx in buckets.get(key, ()):
                        d = pts[idx] - p
                        d -= box * np.round(d / box)
                        if d @ d < min_spacing ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts[placed] = p
            buckets.setdefault(tuple(c), []).append(placed)
            placed += 1
    return pts


def workload(name, **over):
    """Parameters and blob arrays of a named workload.

    Returns a dict with keys: grid (Nx,Ny,Nz), h, rho, eta, kT, dt, kernel, seed,
    precision, steps, q (Nb,3), u (Nb,3), me (Nb,), force (Nb,3).
    """
    if name == "plain":
        cfg = dict(grid=(32, 32, 32), h=1.0, rho=1.0, eta=1.0, kT=1e-3, dt=0.05, kernel=4, seed=1,
                   precision=64, steps=100, nblobs=1, me_range=None, force=(0.0, 0.0, 0.0), place_seed=1,
                   min_spacing=0.0)
    elif name == "bulk":
        cfg = dict(grid=(128, 128, 128), h=1.0, rho=1.0, eta=1.0, kT=1e-3, dt=0.02, kernel=3, seed=2,
                   precision=32, steps=1000, nblobs=2000, me_range=(-0.5, 2.0), force=(0.0, 0.0, 0.0),
                   place_seed=2, min_spacing=2.0)
    elif name == "large":
        cfg = dict(grid=(256, 256, 256), h=1.0, rho=1.0, eta=1.0, kT=1e-3, dt=0.01, kernel=4, seed=3,
                   precision=32, steps=500, nblobs=20000, me_range=(-0.5, 2.0), force=(1e-4, 0.0, 0.0),
                   place_seed=3, min_spacing=2.0)
    else:
        raise KeyError(name)
    cfg.update(over)
    return _materialise(cfg)


def _materialise(cfg):
    h, rho = cfg["h"], cfg["rho"]
    nb = int(cfg["nblobs"])
    if cfg.get("min_spacing", 0.0) > 0.0:
        q = random_sequential_addition(nb, cfg["grid"], h, cfg["min_spacing"] * h, cfg["place_seed"])
    else:
        rng = np.random.default_rng(cfg["place_seed"])
        q = rng.uniform(0.0, 1.0, size=(nb, 3)) * np.asarray(cfg["grid"]) * h
    rng = np.random.default_rng(cfg["place_seed"] + 1000)
    if cfg["me_range"] is None:
        me = np.zeros(nb)
    else:
        lo, hi = cfg["me_range"]
        me = rng.uniform(lo, hi, size=nb) * rho * h ** 3
    # equilibrium blob velocity variance kT / m~ with m~ = m_e + m~_f
    mt = me + DRAGGED_MASS_PER_RHO_H3[cfg["kernel"]] * rho * h ** 3
    if cfg["kT"] > 0.0 and cfg["me_range"] is not None:
        u = rng.standard_normal((nb, 3)) * np.sqrt(cfg["kT"] / mt)[:, None]
    else:
        u = np.zeros((nb, 3))
    force = np.tile(np.asarray(cfg["force"], dtype=np.float64), (nb, 1))
    out = dict(cfg)
    out.update(q=q, u=u, me=me, force=force)
    return out


def random_fluid(grid, amplitude, seed):
    """A random (not divergence-free) face velocity field, shape (3, Nz, Ny, Nx)."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    return amplitude * rng.standard_normal((3, nz, ny, nx))


def batch_replicas(count=64, seed0=1):
    """Replica recipes: side ~ U{32,48,64,96}, N_b ~ U[1,500], kernel ~ U{3,4}, seeds 1..count."""
    out = []
    for r in range(count):
        seed = seed0 + r
        rng = np.random.default_rng(10_000 + seed)
        side = int(rng.choice([32, 48, 64, 96]))
        nb = int(rng.integers(1, 501))
        kernel = int(rng.choice([3, 4]))
        cfg = dict(grid=(side, side, side), h=1.0, rho=1.0, eta=1.0, kT=1e-3, dt=0.05, kernel=kernel,
                   seed=seed, precision=32, steps=200, nblobs=nb, me_range=(-0.5, 2.0),
                   force=(0.0, 0.0, 0.0), place_seed=20_000 + seed, min_spacing=2.0)
        out.append(_materialise(cfg))
    return out


def served_jobs(count, rate=50.0, seed=5):
    """Poisson arrivals (mean `rate`/s) of jobs: side ~ U{32,48,64,96,128}, N_b ~ U[1,2000],
    kT ~ U[1e-4, 1e-2], steps ~ U[50, 500]; other parameters as the batch replicas."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    jobs = []
    for n in range(count):
        side = int(rng.choice([32, 48, 64, 96, 128]))
        nb = int(rng.integers(1, 2001))
        kernel = int(rng.choice([3, 4]))
        cfg = dict(grid=(side, side, side), h=1.0, rho=1.0, eta=1.0, kT=float(rng.uniform(1e-4, 1e-2)),
                   dt=0.05, kernel=kernel, seed=1000 + n, precision=32, steps=int(rng.integers(50, 501)),
                   nblobs=nb, me_range=(-0.5, 2.0), force=(0.0, 0.0, 0.0), place_seed=30_000 + n,
                   min_spacing=2.0)
        job = _materialise(cfg)
        job["arrival"] = float(t[n])
        jobs.append(job)
    return jobs
