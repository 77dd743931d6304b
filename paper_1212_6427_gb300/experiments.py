"""Numerical experiments of arXiv:1212.6427 run through the library's C ABI on the GPU.

* Temporal accuracy (Sec. III.D, Eq. E_dt_definition): a blob released from rest in the
  harmonic potential V = k r^2 / 2; E(dt) is the mean distance between the trajectories
  with steps dt and dt/2, and the observed order is log2 E(dt) / E(dt/2).
* Translational invariance of J P S (Sec. III.A.2, Fig. JPS left): statistics of
  dI(q) = (3/2) dV (J P S)(q) - I over random positions q.
* Pair coupling (Fig. JPS right): (3/2) dV J_i P S_j for two blobs a distance l apart.
* Thermal drift bias (Appendix B.2, Fig. DriftBias): freely diffusing, neutrally buoyant,
  non-interacting blobs at equilibrium should fill a grid cell uniformly; without the
  thermal drift forcing they favour the cell corners.  Reported: the ratio of the
  occupation of the corner and centre octants of the cell (each 1/8 of its volume).
* Equilibrium radial distribution function (Sec. IV.A, Fig. RDF): blobs with WCA pair
  forces in the fluctuating solvent; g(r) of the sampled configurations, to be compared
  with Monte Carlo sampling of exp(-U/kT).
* Single-blob mobility mu = -J L^-1 S of the steady Stokes problem and the effective
  hydrodynamic radius, from 6 pi eta mu = 1/R_H - 2.8373/L (the first-order lattice
  correction of a cubic array of spheres, Hasimoto 1959).

    python -m paper_1212_6427_gb300.experiments trap --precision 64
    python -m paper_1212_6427_gb300.experiments jps --grid 32 --kernel 3
    python -m paper_1212_6427_gb300.experiments pair --grid 32 --kernel 3
    python -m paper_1212_6427_gb300.experiments radius --grid 32 --kernel 3
    python -m paper_1212_6427_gb300.experiments drift --grid 16 --kernel 3
    python -m paper_1212_6427_gb300.experiments rdf --grid 32 --kernel 3
"""
import argparse
import json
import math

import numpy as np

from .binding import FLAG_THERMAL_DRIFT, Simulation, icm_kernel_volume, icm_op_coupling

HASIMOTO = 2.8373   # first-order coefficient of the periodic-lattice mobility correction


def kernel_volume(kernel, h=1.0):
    """The blob volume dV of the Peskin kernel, from the library (icm_kernel_volume)."""
    return icm_kernel_volume(kernel, h)


def trap_trajectory(dt, T, me=0.0, k=0.01, precision=64, slip_flags=0, grid=(16, 16, 16), r0=10.0):
    """Positions after each step of a blob released from rest at (r0, 0, 0), trap centre at
    the origin, kT = 0, h = rho = eta = 1, four-point kernel."""
    sim = Simulation(grid, 1.0, 1.0, 1.0, 0.0, dt, 4, 1, precision, slip_flags)
    try:
        sim.add_blobs([[r0, 0.0, 0.0]], [[0.0, 0.0, 0.0]], [me])
        sim.set_forces([[0.0, 0.0, 0.0]])
        sim.set_trap(k, (0.0, 0.0, 0.0))
        out = []
        for _ in range(int(round(T / dt))):
            sim.step(1)
            out.append(sim.read()["pos"][0].copy())
        return np.array(out)
    finally:
        sim.close()


def trap_error(dts=(1.0, 0.5, 0.25, 0.125), T=16.0, me=0.0, k=0.01, precision=64, slip_flags=0):
    """E(dt) of Eq. E_dt_definition for each consecutive pair of dts, and the observed
    orders log2(E(dt) / E(dt/2))."""
    q = {dt: trap_trajectory(dt, T, me, k, precision, slip_flags) for dt in dts}
    errs = []
    for a, b in zip(dts[:-1], dts[1:]):
        d = q[a] - q[b][1::2]
        d -= 16.0 * np.round(d / 16.0)
        errs.append(float(np.linalg.norm(d, axis=1).mean()))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    return {"dt": list(dts[:-1]), "E": errs, "order": orders, "me": me, "k": k, "T": T, "precision": precision}


def _sim(grid, kernel, precision, eta=1.0):
    return Simulation(grid, 1.0, 1.0, eta, 0.0, 0.05, kernel, 1, precision, 0)


def jps_translational(grid=(32, 32, 32), kernel=3, npos=100, seed=1, precision=64):
    """Mean diagonal, max |diagonal| and max |off-diagonal| of dI(q) over random q."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.0, 1.0, size=(npos, 3)) * np.asarray(grid, dtype=float)
    sim = _sim(grid, kernel, precision)
    try:
        m = icm_op_coupling(sim.handle, q, q, 1.0, 0.0)
    finally:
        sim.close()
    di = 1.5 * kernel_volume(kernel) * m - np.eye(3)
    diag = np.diagonal(di, axis1=1, axis2=2)
    off = di - np.einsum("nij,ij->nij", di, np.eye(3))
    return {"grid": list(grid), "kernel": kernel, "positions": npos, "mean_diag": float(diag.mean()),
            "max_abs_diag": float(np.abs(diag).max()), "max_abs_offdiag": float(np.abs(off).max())}


def pair_coupling(grid=(32, 32, 32), kernel=3, ls=(0, 1, 2, 3, 4, 5, 6, 8, 10), direction=(1.0, 0.0, 0.0),
                  q0=(9.3, 10.6, 12.1), precision=64):
    """Max |diagonal| and max |off-diagonal| of (3/2) dV J_i P S_j at distances l."""
    u = np.asarray(direction, dtype=float)
    u /= np.linalg.norm(u)
    qj = np.tile(np.asarray(q0, dtype=float), (len(ls), 1))
    qi = qj + np.asarray(ls, dtype=float)[:, None] * u
    sim = _sim(grid, kernel, precision)
    try:
        m = 1.5 * kernel_volume(kernel) * icm_op_coupling(sim.handle, qi, qj, 1.0, 0.0)
    finally:
        sim.close()
    diag = np.abs(np.diagonal(m, axis1=1, axis2=2)).max(axis=1)
    off = np.abs(m - np.einsum("nij,ij->nij", m, np.eye(3))).max(axis=(1, 2))
    return {"grid": list(grid), "kernel": kernel, "direction": list(u), "l": list(ls),
            "max_diag": diag.tolist(), "max_offdiag": off.tolist()}


def hydrodynamic_radius(grid=(32, 32, 32), kernel=3, npos=16, seed=2, eta=1.0, precision=64):
    """Mean single-blob Stokes mobility over random positions, its spread, and R_H."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.0, 1.0, size=(npos, 3)) * np.asarray(grid, dtype=float)
    sim = _sim(grid, kernel, precision, eta)
    try:
        m = icm_op_coupling(sim.handle, q, q, 0.0, eta)
    finally:
        sim.close()
    mus = np.trace(m, axis1=1, axis2=2) / 3.0
    mu = float(mus.mean())
    L = float(grid[0])
    return {"grid": list(grid), "kernel": kernel, "positions": npos, "mu": mu,
            "mu_rel_spread": float(mus.std() / mu), "R_H": 1.0 / (6.0 * math.pi * eta * mu + HASIMOTO / L)}


def drift_bias(grid=(16, 16, 16), kernel=3, nblobs=100, kT=1.0, dt=0.05, steps=100000, sample_every=10,
               drift=True, seed=3, precision=32):
    """Occupation of the corner and centre octants of the grid cell by the fractional
    positions q/h - floor(q/h) of neutrally buoyant, non-interacting blobs (h = rho =
    eta = 1, so the viscous CFL number is dt), sampled every `sample_every` steps after
    a tenth of the run.  Returns the ratio corner/centre and its binomial error."""
    rng = np.random.default_rng(seed)
    q0 = rng.uniform(0.0, 1.0, size=(nblobs, 3)) * np.asarray(grid, dtype=float)
    sim = Simulation(grid, 1.0, 1.0, 1.0, kT, dt, kernel, seed, precision, FLAG_THERMAL_DRIFT if drift else 0)
    corner = centre = samples = 0
    try:
        sim.add_blobs(q0, None, np.zeros(nblobs))
        burn = steps // 10
        sim.step(burn)
        for _ in range((steps - burn) // sample_every):
            sim.step(sample_every)
            f = sim.read()["pos"]
            f = f - np.floor(f)
            d_node = np.abs(f - np.round(f))
            corner += int(np.all(d_node < 0.25, axis=1).sum())
            centre += int(np.all(np.abs(f - 0.5) < 0.25, axis=1).sum())
            samples += nblobs
    finally:
        sim.close()
    ratio = corner / max(centre, 1)
    err = ratio * math.sqrt(1.0 / max(corner, 1) + 1.0 / max(centre, 1))
    return {"grid": list(grid), "kernel": kernel, "blobs": nblobs, "kT": kT, "dt": dt, "steps": steps,
            "thermal_drift": drift, "samples": samples, "corner_fraction": corner / samples,
            "centre_fraction": centre / samples, "corner_over_centre": ratio, "ratio_error_uncorrelated": err}


def pair_rdf(samples, box, dr=0.1, rmax=8.0):
    """g(r) of a list of (n, 3) configurations in a periodic box (bin centres, g).  The
    pair distances of each configuration are histogrammed with torch (on the GPU when
    there is one): this is analysis of the sampled states, not part of the step."""
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    boxt = torch.tensor(np.asarray(box, dtype=float), dtype=torch.float64, device=dev)
    nbins = int(round(rmax / dr))
    hist = torch.zeros(nbins, dtype=torch.float64, device=dev)
    n = samples[0].shape[0]
    iu = torch.triu_indices(n, n, 1, device=dev)
    for q in samples:
        qt = torch.as_tensor(q, dtype=torch.float64, device=dev)
        d = qt[iu[0]] - qt[iu[1]]
        d -= boxt * torch.round(d / boxt)
        r = torch.sqrt((d * d).sum(dim=1))
        r = r[r < rmax]
        hist += 2.0 * torch.bincount((r / dr).long(), minlength=nbins)[:nbins].double()
    hist = hist.cpu().numpy()
    box = np.asarray(box, dtype=float)
    rho = n / box.prod()
    edges = np.arange(nbins + 1) * dr
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    return edges[:-1] + 0.5 * dr, hist / (len(samples) * n * rho * shell)


def rdf(grid=(32, 32, 32), kernel=3, n=1000, sigma=2.0, eps=1e-3, kT=1e-3, dt=1.0, me=0.0, burn=20000,
        steps=100000, sample_every=100, seed=5, precision=32):
    """g(r) of n blobs with WCA forces (Table tableRDF parameters by default: h = rho =
    eta = 1, so the viscous CFL number is dt), started on a simple cubic lattice."""
    side = int(math.ceil(n ** (1.0 / 3.0)))
    idx = np.arange(n)
    lattice = np.stack([idx % side, (idx // side) % side, idx // (side * side)], axis=1) + 0.5
    q0 = lattice * (np.asarray(grid, dtype=float) / side)
    import time
    sim = Simulation(grid, 1.0, 1.0, 1.0, kT, dt, kernel, seed, precision, 0)
    samples = []
    try:
        sim.add_blobs(q0, None, np.full(n, me))
        sim.set_wca(eps, sigma)
        sim.step(burn)
        sim.sync()
        t0 = time.perf_counter()
        for _ in range(steps // sample_every):
            sim.step(sample_every)
            samples.append(sim.read()["pos"].copy())
        t_steps = time.perf_counter() - t0
    finally:
        sim.close()
    r, g = pair_rdf(samples, grid)
    return {"grid": list(grid), "kernel": kernel, "n": n, "sigma": sigma, "eps": eps, "kT": kT, "dt": dt, "me": me,
            "burn": burn, "steps": steps, "samples": len(samples), "ms_per_step": 1e3 * t_steps / steps,
            "r": r.tolist(), "g": g.tolist()}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("experiment", choices=["trap", "jps", "pair", "radius", "drift", "rdf"])
    ap.add_argument("--steps", type=int, default=100000)
    ap.add_argument("--precision", type=int, default=64, choices=[32, 64])
    ap.add_argument("--grid", type=int, default=32)
    ap.add_argument("--kernel", type=int, default=3, choices=[3, 4])
    ap.add_argument("--positions", type=int, default=100)
    args = ap.parse_args(argv)
    g = (args.grid,) * 3
    if args.experiment == "trap":
        rows = [trap_error(me=me, precision=args.precision) for me in (0.0, 28.44, 284.4)]
    elif args.experiment == "jps":
        rows = [jps_translational(g, args.kernel, args.positions, precision=args.precision)]
    elif args.experiment == "pair":
        rows = [pair_coupling(g, args.kernel, direction=d, precision=args.precision)
                for d in ((1.0, 0.0, 0.0), (1.0, 1.0, 1.0))]
    elif args.experiment == "rdf":
        mf = kernel_volume(args.kernel)   # m_f = rho dV
        rows = [rdf(g, args.kernel, me=me, steps=args.steps, precision=args.precision) for me in (0.0, mf)]
    elif args.experiment == "drift":
        rows = [drift_bias(g, args.kernel, steps=args.steps, drift=d, precision=args.precision) for d in (False, True)]
    else:
        rows = [hydrodynamic_radius(g, args.kernel, min(args.positions, 32), precision=args.precision)]
    for r in rows:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
