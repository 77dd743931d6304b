"""Write tests/golden/wca_rdf_mc.txt: the equilibrium g(r) of the WCA suspension of
Sec. IV.A (Table tableRDF: N = 1000, 32^3 box of unit cells, sigma = 2, eps = kT = 0.001)
by Metropolis Monte Carlo (oracle/mc_wca.c), the reference the inertial coupling
dynamics is compared with.  Calls only oracle/.

    python tests/golden/make_wca_rdf.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mc  # noqa: E402

PARAMS = dict(n=1000, box=(32.0, 32.0, 32.0), sigma=2.0, eps=1e-3, kT=1e-3, sweeps=40000, burn=4000,
              sample_every=20, seed=2013, dr=0.1, rmax=8.0)


def main():
    r, g, acc = mc.wca_rdf(**PARAMS)
    path = os.path.join(HERE, "wca_rdf_mc.txt")
    with open(path, "w") as fh:
        fh.write("# g(r) of the WCA suspension of Sec. IV.A (Eq. WCA, Table tableRDF): N = 1000 particles,\n")
        fh.write("# 32^3 periodic box, sigma = 2, eps = kT = 0.001; Metropolis Monte Carlo, oracle/mc_wca.c,\n")
        fh.write("# %s; acceptance %.3f.  Written by tests/golden/make_wca_rdf.py.\n" % (PARAMS, acc))
        fh.write("# r g(r)\n")
        for a, b in zip(r, g):
            fh.write("%.4f %.6f\n" % (a, b))
    print(path)


if __name__ == "__main__":
    main()
