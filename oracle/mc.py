"""Build and run the Monte Carlo reference sampler oracle/mc_wca.c (test
infrastructure; see that file).  Plain gcc, no GPU."""
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mc_wca.c")
BIN = os.path.join(HERE, "_build", "mc_wca")


def build(force=False):
    """Compile mc_wca.c into oracle/_build/mc_wca unless it is up to date."""
    if not force and os.path.exists(BIN) and os.path.getmtime(BIN) >= os.path.getmtime(SRC):
        return BIN
    os.makedirs(os.path.dirname(BIN), exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the Monte Carlo oracle")
    tmp = BIN + ".tmp"
    subprocess.run([cc, "-O2", "-o", tmp, SRC, "-lm"], check=True, capture_output=True, text=True)
    os.replace(tmp, BIN)
    return BIN


def wca_rdf(n, box, sigma, eps, kT, sweeps, burn, sample_every, seed, dr, rmax):
    """(r, g(r), acceptance) of Metropolis sampling of the WCA system."""
    args = [build(), str(n), *(repr(float(b)) for b in box), repr(float(sigma)), repr(float(eps)), repr(float(kT)),
            str(sweeps), str(burn), str(sample_every), str(seed), repr(float(dr)), repr(float(rmax))]
    out = subprocess.run(args, check=True, capture_output=True, text=True).stdout
    rows = [ln.split() for ln in out.splitlines() if ln and not ln.startswith("#")]
    acc = float([ln for ln in out.splitlines() if ln.startswith("# acceptance")][0].split()[2])
    r = np.array([float(a) for a, _ in rows])
    g = np.array([float(b) for _, b in rows])
    return r, g, acc
