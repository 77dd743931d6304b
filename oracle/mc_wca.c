/* Metropolis Monte Carlo sampling of the Gibbs-Boltzmann distribution
 * P(Q) ~ exp(-U(Q)/kT) of N particles with the WCA pair potential
 *   V(r) = 4 eps ((s/r)^12 - (s/r)^6) + eps,  r < 2^(1/6) s;  0 beyond
 * in a periodic box (arXiv:1212.6427, Sec. IV.A, Eq. WCA and Eq. P_Q), and the radial
 * distribution function g(r) of the sampled configurations: the reference against
 * which the equilibrium g(r) of the inertial coupling dynamics is compared.
 *
 * Test infrastructure (oracle): plain, slow, obviously correct; shares nothing with
 * the GPU library.  Random numbers: splitmix64 (Steele, Lea, Flood, OOPSLA 2014).
 *
 * usage: mc_wca N Lx Ly Lz sigma eps kT sweeps burn sample_every seed dr rmax
 * prints "r g(r)" lines (bin centres) and a final "# acceptance" line.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

static uint64_t rng_state;

/* splitmix64: state += golden gamma; mix with two xor-shift-multiply rounds. */
static uint64_t splitmix64(void) {
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* uniform in [0, 1) with 53 random bits */
static double uniform(void) { return (double)(splitmix64() >> 11) * (1.0 / 9007199254740992.0); }

static int n;
static double L[3], sig, eps, kT, rc2;
static double *x;               /* n x 3 positions in [0, L) */
static int nc[3], ncells;       /* cell grid */
static int *cell_of, *cell_cnt, *cell_mem, cap;

static double wrap(double v, double len) {
  v -= len * floor(v / len);
  return v >= len ? v - len : v;
}

static double min_image(double d, double len) { return d - len * nearbyint(d / len); }

static double pair_energy(double r2) {
  if (r2 >= rc2) return 0.0;
  const double s6 = pow(sig * sig / r2, 3.0);
  return 4.0 * eps * (s6 * s6 - s6) + eps;
}

static int cell_index(const double* p) {
  int c[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = (int)(p[a] / L[a] * nc[a]);
    if (c[a] >= nc[a]) c[a] = nc[a] - 1;
  }
  return c[0] + nc[0] * (c[1] + nc[1] * c[2]);
}

static void cell_add(int i, int c) {
  if (cell_cnt[c] >= cap) {
    fprintf(stderr, "cell capacity exceeded\n");
    exit(2);
  }
  cell_mem[c * cap + cell_cnt[c]++] = i;
  cell_of[i] = c;
}

static void cell_remove(int i) {
  const int c = cell_of[i];
  for (int k = 0; k < cell_cnt[c]; ++k)
    if (cell_mem[c * cap + k] == i) {
      cell_mem[c * cap + k] = cell_mem[c * cap + --cell_cnt[c]];
      return;
    }
}

/* energy of particle i at position p with every other particle (cell list; cells are
 * at least the cut-off wide and at least 3 per axis, so the 27 neighbours are distinct) */
static double energy_of(int i, const double* p) {
  int c[3];
  const int ci = cell_index(p);
  c[0] = ci % nc[0];
  c[1] = (ci / nc[0]) % nc[1];
  c[2] = ci / (nc[0] * nc[1]);
  double u = 0.0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int cx = (c[0] + dx + nc[0]) % nc[0], cy = (c[1] + dy + nc[1]) % nc[1], cz = (c[2] + dz + nc[2]) % nc[2];
        const int cc = cx + nc[0] * (cy + nc[1] * cz);
        for (int k = 0; k < cell_cnt[cc]; ++k) {
          const int j = cell_mem[cc * cap + k];
          if (j == i) continue;
          double r2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double d = min_image(p[a] - x[3 * j + a], L[a]);
            r2 += d * d;
          }
          u += pair_energy(r2);
        }
      }
  return u;
}

int main(int argc, char** argv) {
  if (argc != 14) {
    fprintf(stderr, "usage: %s N Lx Ly Lz sigma eps kT sweeps burn sample_every seed dr rmax\n", argv[0]);
    return 1;
  }
  n = atoi(argv[1]);
  for (int a = 0; a < 3; ++a) L[a] = atof(argv[2 + a]);
  sig = atof(argv[5]);
  eps = atof(argv[6]);
  kT = atof(argv[7]);
  const long sweeps = atol(argv[8]), burn = atol(argv[9]), every = atol(argv[10]);
  rng_state = (uint64_t)strtoull(argv[11], NULL, 10);
  const double dr = atof(argv[12]), rmax = atof(argv[13]);
  const double rc = pow(2.0, 1.0 / 6.0) * sig;
  rc2 = rc * rc;
  for (int a = 0; a < 3; ++a) {
    nc[a] = (int)(L[a] / rc);
    if (nc[a] < 3 || rmax > 0.5 * L[a]) {
      fprintf(stderr, "box too small for the cell list or rmax\n");
      return 1;
    }
  }
  ncells = nc[0] * nc[1] * nc[2];
  cap = 64;
  x = malloc(sizeof(double) * 3 * n);
  cell_of = malloc(sizeof(int) * n);
  cell_cnt = calloc(ncells, sizeof(int));
  cell_mem = malloc(sizeof(int) * ncells * cap);
  /* start on a simple cubic lattice (no overlaps at the densities used) */
  int side = 1;
  while (side * side * side < n) ++side;
  for (int i = 0; i < n; ++i) {
    const int ix = i % side, iy = (i / side) % side, iz = i / (side * side);
    x[3 * i + 0] = (ix + 0.5) * L[0] / side;
    x[3 * i + 1] = (iy + 0.5) * L[1] / side;
    x[3 * i + 2] = (iz + 0.5) * L[2] / side;
    cell_add(i, cell_index(&x[3 * i]));
  }
  const int nbins = (int)(rmax / dr);
  double* hist = calloc(nbins, sizeof(double));
  double delta = 0.2 * sig;
  long accepted = 0, tried = 0, samples = 0;
  for (long sw = 0; sw < sweeps; ++sw) {
    long acc_sweep = 0;
    for (int m = 0; m < n; ++m) {
      const int i = (int)(uniform() * n);
      double p[3];
      for (int a = 0; a < 3; ++a) p[a] = wrap(x[3 * i + a] + delta * (2.0 * uniform() - 1.0), L[a]);
      const double du = energy_of(i, p) - energy_of(i, &x[3 * i]);
      if (du <= 0.0 || uniform() < exp(-du / kT)) {
        cell_remove(i);
        for (int a = 0; a < 3; ++a) x[3 * i + a] = p[a];
        cell_add(i, cell_index(p));
        ++acc_sweep;
      }
    }
    if (sw < burn) {   /* tune the step to ~40% acceptance while equilibrating */
      const double f = (double)acc_sweep / n;
      delta *= f > 0.4 ? 1.05 : 0.95;
      if (delta > 0.5 * rc) delta = 0.5 * rc;
      continue;
    }
    accepted += acc_sweep;
    tried += n;
    if ((sw - burn) % every == 0) {
      ++samples;
      for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
          double r2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double d = min_image(x[3 * i + a] - x[3 * j + a], L[a]);
            r2 += d * d;
          }
          const double r = sqrt(r2);
          if (r < rmax) hist[(int)(r / dr)] += 2.0;   /* counted once for i and once for j */
        }
    }
  }
  const double rho = n / (L[0] * L[1] * L[2]);
  for (int k = 0; k < nbins; ++k) {
    const double r0 = k * dr, r1 = r0 + dr;
    const double shell = 4.0 / 3.0 * M_PI * (r1 * r1 * r1 - r0 * r0 * r0);
    printf("%.4f %.6f\n", r0 + 0.5 * dr, hist[k] / ((double)samples * n * rho * shell));
  }
  printf("# acceptance %.4f samples %ld delta %.4f\n", (double)accepted / (double)tried, samples, delta);
  free(x);
  free(cell_of);
  free(cell_cnt);
  free(cell_mem);
  free(hist);
  return 0;
}
