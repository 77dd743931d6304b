"""FP64 CPU oracle of one step of the incompressible Inertial Coupling Method.

TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct statement
of what the CUDA library computes, used by the parity tests, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / reference legs of
``bench.py``.  Nothing in the library imports or calls it; it shares no code,
table or helper with the CUDA path.  It is written in numpy, float64
throughout; numpy's FFT serves as the library FFT primitive of the Helmholtz and
projection solves.

Paper: F. Balboa Usabiaga, R. Delgado-Buscalioni, B. E. Griffith, A. Donev,
"Inertial coupling method for particles in an incompressible fluctuating
fluid", arXiv:1212.6427.  Citations below are to its sections and equations.

Readings of points the paper leaves open:
  * MAC grid (Sec. III.A): cell (i,j,k) centred at ((i+1/2)h, (j+1/2)h, (k+1/2)h);
    v_x[i,j,k] sits on the low x face (ih, (j+1/2)h, (k+1/2)h), likewise v_y, v_z.
    Arrays have shape (Nz, Ny, Nx) so the flat index is i + Nx (j + Ny k).
  * Divergence (Dv)_c = sum_a (v_a[c+e_a] - v_a[c])/h, gradient
    (Gp)_a[c] = (p_c - p_{c-e_a})/h, Laplacian = 7-point stencil on each
    component's own grid.  The projection is the exact discrete staggered one,
    P = I - G (D G)^-1 D, with P = I on the k = 0 (mean) mode.
  * Peskin 3-point and 4-point kernels (Sec. III.A.1: the minimal-support
    functions with unit sum, zero first moment and constant sum of squares).
    3-point nodes: round-half-up(s) + {-1,0,1}; 4-point: floor(s) + {-1,0,1,2},
    s = q/h - offset of the component along that axis.
  * Stochastic stress (Sec. III.B.2): 6 normals per cell (see oracle.philox);
    Sigma_aa = 2 s Z_aa at cell centres, Sigma_ab = sqrt(2) s Z_ab on the
    edges, s = sqrt(kT eta / (dV_f dt)); that is W + W^T with 9 i.i.d. normals.
  * Advection (Sec. II.B, skew-adjoint, conservative): centred divergence form
    div(rho v v^T) with two-point averages; Adams-Bashforth start-up A^{-1} = A^0.
  * The blob volume dV = h^3 / (sum phi^2)^3 is the kernel's exact value
    (8 h^3 for 3-point, (8/3)^3 h^3 for 4-point), m~_f = 3 rho dV / 2.
  * Slip correction options: 'visc' (Eq. delta_u_nph_visc, the paper's default),
    'full' (Eq. delta_u_nph), 'zero'.
"""
import numpy as np

from .philox import stress_normals

DIM = 3
KERNEL_WIDTH = {3: 3, 4: 4}


# ---------------------------------------------------------------------------
# Peskin kernels (Sec. III.A.1, Eq. JS_invariance)
# ---------------------------------------------------------------------------
def phi3(r):
    """Peskin 3-point function of r in grid units."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    inner = r <= 0.5
    outer = (r > 0.5) & (r <= 1.5)
    out[inner] = (1.0 + np.sqrt(1.0 - 3.0 * r[inner] ** 2)) / 3.0
    ro = r[outer]
    out[outer] = (5.0 - 3.0 * ro - np.sqrt(np.maximum(1.0 - 3.0 * (1.0 - ro) ** 2, 0.0))) / 6.0
    return out


def phi4(r):
    """Peskin 4-point function of r in grid units."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    inner = r <= 1.0
    outer = (r > 1.0) & (r <= 2.0)
    ri = r[inner]
    out[inner] = (3.0 - 2.0 * ri + np.sqrt(1.0 + 4.0 * ri - 4.0 * ri ** 2)) / 8.0
    ro = r[outer]
    out[outer] = (5.0 - 2.0 * ro - np.sqrt(np.maximum(-7.0 + 12.0 * ro - 4.0 * ro ** 2, 0.0))) / 8.0
    return out


def phi(kernel, r):
    if kernel == 3:
        return phi3(r)
    if kernel == 4:
        return phi4(r)
    raise ValueError("kernel must be 3 or 4")


def dphi3(r):
    """Derivative of the Peskin 3-point function, from its closed form: -r/sqrt(1-3r^2)
    for |r| <= 1/2; sign(r) (-3 - 3t/sqrt(1-3t^2))/6, t = 1-|r|, for 1/2 <= |r| <= 3/2."""
    r = np.asarray(r, dtype=np.float64)
    a = np.abs(r)
    out = np.zeros_like(r)
    inner = a <= 0.5
    outer = (a > 0.5) & (a <= 1.5)
    out[inner] = -r[inner] / np.sqrt(1.0 - 3.0 * r[inner] ** 2)
    t = 1.0 - a[outer]
    out[outer] = np.sign(r[outer]) * (-3.0 - 3.0 * t / np.sqrt(1.0 - 3.0 * t ** 2)) / 6.0
    return out


def dphi4(r):
    """Derivative of the Peskin 4-point function, from its closed form:
    sign(r) (-2 + (2-4|r|)/sqrt(1+4|r|-4r^2))/8 for |r| <= 1;
    sign(r) (-2 - (6-4|r|)/sqrt(-7+12|r|-4r^2))/8 for 1 <= |r| <= 2."""
    r = np.asarray(r, dtype=np.float64)
    a = np.abs(r)
    out = np.zeros_like(r)
    inner = a <= 1.0
    outer = (a > 1.0) & (a <= 2.0)
    ai = a[inner]
    out[inner] = np.sign(r[inner]) * (-2.0 + (2.0 - 4.0 * ai) / np.sqrt(1.0 + 4.0 * ai - 4.0 * ai ** 2)) / 8.0
    ao = a[outer]
    out[outer] = np.sign(r[outer]) * (-2.0 - (6.0 - 4.0 * ao) / np.sqrt(-7.0 + 12.0 * ao - 4.0 * ao ** 2)) / 8.0
    return out


def dphi(kernel, r):
    if kernel == 3:
        return dphi3(r)
    if kernel == 4:
        return dphi4(r)
    raise ValueError("kernel must be 3 or 4")


def kernel_sum_sq(kernel):
    """sum_k phi^2 along one axis: 1/2 (3-point), 3/8 (4-point)."""
    return {3: 0.5, 4: 0.375}[kernel]


def blob_volume(kernel, h):
    """dV = (J S 1)^-1 = h^3 / (sum phi^2)^3  (Eq. dV_JS, Eq. JS_invariance)."""
    return h ** 3 / kernel_sum_sq(kernel) ** 3


def fluid_dragged_mass(kernel, h, rho):
    """m~_f = d rho dV / (d-1)  (Appendix A, after Eq. JPS)."""
    return DIM * rho * blob_volume(kernel, h) / (DIM - 1)


def stencil_1d(s, kernel):
    """Nodes and weights along one axis.  s = q/h - offset, shape (Nb,).

    Returns (nodes (Nb, w) int64, weights (Nb, w)).  Node indices are not wrapped.
    """
    s = np.asarray(s, dtype=np.float64)
    if kernel == 3:
        first = np.floor(s + 0.5).astype(np.int64) - 1
    elif kernel == 4:
        first = np.floor(s).astype(np.int64) - 1
    else:
        raise ValueError("kernel must be 3 or 4")
    w = KERNEL_WIDTH[kernel]
    nodes = first[:, None] + np.arange(w)[None, :]
    weights = phi(kernel, s[:, None] - nodes)
    return nodes, weights


def component_offsets(comp):
    """Offsets (in units of h) of velocity component `comp` along x, y, z."""
    return [0.0 if ax == comp else 0.5 for ax in range(DIM)]


def _blob_stencil(q, comp, kernel, h, shape):
    """Per-axis wrapped node indices and weights of all blobs for one component."""
    nz, ny, nx = shape
    sizes = (nx, ny, nz)
    offs = component_offsets(comp)
    idx, wts = [], []
    for ax in range(DIM):
        nodes, w = stencil_1d(q[:, ax] / h - offs[ax], kernel)
        idx.append(np.mod(nodes, sizes[ax]))
        wts.append(w)
    return idx, wts


# ---------------------------------------------------------------------------
# Interpolation J and spreading S (Sec. III.A.1)
# ---------------------------------------------------------------------------
def interpolate(field, q, kernel, h):
    """(J v)_i = sum_k phi(q_i - r_k) v_k for each component.  field: (3, Nz, Ny, Nx)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    out = np.zeros((q.shape[0], DIM))
    shape = field.shape[1:]
    for comp in range(DIM):
        (ix, iy, iz), (wx, wy, wz) = _blob_stencil(q, comp, kernel, h, shape)
        vals = field[comp][iz[:, :, None, None], iy[:, None, :, None], ix[:, None, None, :]]
        wgt = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
        out[:, comp] = np.sum(wgt * vals, axis=(1, 2, 3))
    return out


def spread(force, q, kernel, h, shape):
    """(S F)_k = dV_f^-1 sum_i phi(q_i - r_k) F_i for each component."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    force = np.atleast_2d(np.asarray(force, dtype=np.float64))
    out = np.zeros((DIM,) + tuple(shape))
    dvf = h ** 3
    for comp in range(DIM):
        (ix, iy, iz), (wx, wy, wz) = _blob_stencil(q, comp, kernel, h, shape)
        wgt = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
        contrib = wgt * (force[:, comp] / dvf)[:, None, None, None]
        zz = np.broadcast_to(iz[:, :, None, None], wgt.shape)
        yy = np.broadcast_to(iy[:, None, :, None], wgt.shape)
        xx = np.broadcast_to(ix[:, None, None, :], wgt.shape)
        np.add.at(out[comp], (zz.ravel(), yy.ravel(), xx.ravel()), contrib.ravel())
    return out


def spread_drift(coef, q, kernel, h, shape):
    """Thermal drift forcing of Appendix B.2 (Eq. thermal_drift, the kernel-derivative
    form): component a of the field is dV_f^-1 sum_i coef_i d/dq_a phi(q_i - r_k), i.e.
    (1/h) phi'(s_a) along the component's own axis times phi along the other two
    (= -coef_i times the gradient of the kernel with respect to r)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    coef = np.asarray(coef, dtype=np.float64).reshape(q.shape[0])
    out = np.zeros((DIM,) + tuple(shape))
    dvf = h ** 3
    for comp in range(DIM):
        (ix, iy, iz), wts = _blob_stencil(q, comp, kernel, h, shape)
        s = q[:, comp] / h                                    # the component's own axis: offset 0
        nodes, _ = stencil_1d(s, kernel)
        wts = list(wts)
        wts[comp] = dphi(kernel, s[:, None] - nodes) / h
        wx, wy, wz = wts
        wgt = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
        contrib = wgt * (coef / dvf)[:, None, None, None]
        zz = np.broadcast_to(iz[:, :, None, None], wgt.shape)
        yy = np.broadcast_to(iy[:, None, :, None], wgt.shape)
        xx = np.broadcast_to(ix[:, None, None, :], wgt.shape)
        np.add.at(out[comp], (zz.ravel(), yy.ravel(), xx.ravel()), contrib.ravel())
    return out


# ---------------------------------------------------------------------------
# Staggered finite differences (Sec. III.A; operators of the MAC scheme)
# ---------------------------------------------------------------------------
_NPAXIS = {0: 2, 1: 1, 2: 0}   # x, y, z -> numpy axis of an (Nz, Ny, Nx) array


def shift(f, axis, s):
    """g[c] = f[c + s e_axis] with periodic wrap."""
    return np.roll(f, -s, axis=_NPAXIS[axis])


def divergence(v, h):
    """Cell-centred (D v)_c = sum_a (v_a[c+e_a] - v_a[c]) / h."""
    return sum(shift(v[a], a, 1) - v[a] for a in range(DIM)) / h


def gradient(p, h):
    """Face-centred (G p)_a[c] = (p_c - p_{c-e_a}) / h."""
    return np.stack([(p - shift(p, a, -1)) / h for a in range(DIM)])


def laplacian(f, h):
    """7-point Laplacian of one scalar grid function."""
    return sum(shift(f, a, 1) - 2.0 * f + shift(f, a, -1) for a in range(DIM)) / h ** 2


def vector_laplacian(v, h):
    return np.stack([laplacian(v[a], h) for a in range(DIM)])


def advection(v, rho, h):
    """A = div(rho v v^T) on the faces, centred conservative form.

    Component a at face c:
      (rho/h) [ (ubar_a[c])^2 - (ubar_a[c-e_a])^2
                + sum_{b != a} ( (ut_a ut_b)|edge(c+e_b) - (ut_a ut_b)|edge(c) ) ]
    with ubar_a[c] = (v_a[c+e_a] + v_a[c])/2 at the cell centre and, on the
    (a,b) edge with index c, ut_a = (v_a[c] + v_a[c-e_b])/2 and
    ut_b = (v_b[c] + v_b[c-e_a])/2.
    """
    out = np.zeros_like(v)
    for a in range(DIM):
        ubar = 0.5 * (shift(v[a], a, 1) + v[a])
        acc = ubar ** 2 - shift(ubar ** 2, a, -1)
        for b in range(DIM):
            if b == a:
                continue
            ut_a = 0.5 * (v[a] + shift(v[a], b, -1))
            ut_b = 0.5 * (v[b] + shift(v[b], a, -1))
            flux = ut_a * ut_b
            acc = acc + shift(flux, b, 1) - flux
        out[a] = rho * acc / h
    return out


def stochastic_flux_divergence(z, s, h, shape):
    """div Sigma on the faces from the 6 per-cell normals (Sec. III.B.2).

    z: (6, ncell) ordered (xx, yy, zz, xy, xz, yz).  Sigma_aa = 2 s Z_aa at the
    cell centre c; Sigma_ab = sqrt(2) s Z_ab on the edge with index c
    (xy edge at (ih, jh, (k+1/2)h), xz at (ih, (j+1/2)h, kh), yz at ((i+1/2)h, jh, kh)).
    """
    zz = z.reshape((6,) + tuple(shape))
    diag = [2.0 * s * zz[0], 2.0 * s * zz[1], 2.0 * s * zz[2]]
    off = {(0, 1): np.sqrt(2.0) * s * zz[3], (0, 2): np.sqrt(2.0) * s * zz[4],
           (1, 2): np.sqrt(2.0) * s * zz[5]}
    out = np.zeros((DIM,) + tuple(shape))
    for a in range(DIM):
        acc = diag[a] - shift(diag[a], a, -1)
        for b in range(DIM):
            if b == a:
                continue
            sig = off[(min(a, b), max(a, b))]
            acc = acc + shift(sig, b, 1) - sig
        out[a] = acc / h
    return out


# ---------------------------------------------------------------------------
# FFT Helmholtz solve + projection (Sec. III.D, Appendix C)
# ---------------------------------------------------------------------------
def _symbols(shape, h):
    """d_a = (exp(i theta_a) - 1)/h on the full FFT grid, broadcast to `shape`."""
    nz, ny, nx = shape
    th = [2.0 * np.pi * np.fft.fftfreq(n) for n in (nx, ny, nz)]
    dx = (np.exp(1j * th[0]) - 1.0) / h
    dy = (np.exp(1j * th[1]) - 1.0) / h
    dz = (np.exp(1j * th[2]) - 1.0) / h
    return (dx[None, None, :], dy[None, :, None], dz[:, None, None])


def dft3(f):
    """The 3D discrete Fourier transform by its definition, an explicit O(N^2) sum:
    F[k] = sum_j f[j] exp(-2 pi i (kx jx / Nx + ky jy / Ny + kz jz / Nz)) over every
    pair (k, j) of grid points, as one dense matrix (small grids only)."""
    shape = f.shape
    idx = np.indices(shape).reshape(len(shape), -1)          # (3, N): (z, y, x) of every point
    phase = sum(np.outer(idx[a], idx[a]) / shape[a] for a in range(len(shape)))
    return (np.exp(-2j * np.pi * phase) @ f.reshape(-1)).reshape(shape)


def idft3(F):
    """Inverse of dft3 by its definition: f[j] = N^-1 sum_k F[k] exp(+2 pi i k.j/N)."""
    return np.conj(dft3(np.conj(F))) / F.size


def spectral_solve(rhs, a, b, h, fft=np.fft.fftn, ifft=np.fft.ifftn):
    """Solve (a I - b L) x + G pi = rhs, D x = 0 on the periodic MAC grid.

    In Fourier space x^ = P^ rhs^ / (a + b sum_a |d_a|^2), with
    (P^ w)_a = w_a - conj(d_a) (sum_b d_b w_b) / sum_b |d_b|^2 and P^ = I at k = 0.
    With (a, b) = (rho/dt, eta/2) this is the provisional solve (Eq.
    provisional_step-1); (1, 0) is the projection of step 5; (rho, dt eta/2) the
    viscous correction (Eq. dv_eq_modified-1).  (0, eta) is the steady Stokes solve
    of the mobility -J L^-1 S (Sec. III.A.2); there the k = 0 mode has no solution
    on the periodic grid and is set to zero (zero mean flow; a reading).
    The transform pair is numpy's FFT; spectral_solve_dft passes the plain DFT sums.
    """
    shape = rhs.shape[1:]
    d = _symbols(shape, h)
    rh = [fft(rhs[c]) for c in range(DIM)]
    dd = sum(np.abs(dc) ** 2 for dc in d)
    div = sum(d[c] * rh[c] for c in range(DIM))
    safe = np.where(dd == 0.0, 1.0, dd)
    ratio = np.where(dd == 0.0, 0.0, div / safe)
    denom = a + b * dd
    inv = np.where(denom == 0.0, 0.0, 1.0 / np.where(denom == 0.0, 1.0, denom))
    return np.stack([np.real(ifft((rh[c] - np.conj(d[c]) * ratio) * inv))
                     for c in range(DIM)])


def spectral_solve_dft(rhs, a, b, h):
    """spectral_solve with the transforms done by the plain O(N^2) DFT sums (dft3,
    idft3) instead of an FFT: the slow statement of the same solve, for small grids."""
    return spectral_solve(rhs, a, b, h, fft=dft3, ifft=idft3)


# ---------------------------------------------------------------------------
# Blob-grid operators of Sec. III.A.2 (translational invariance, mobility)
# ---------------------------------------------------------------------------
def coupling_matrix(qi, qj, grid, kernel, h, a=1.0, b=0.0):
    """3x3 matrix M_ab = e_a . J_i (a - b L)^-1 P S_j e_b: column b is the interpolation
    at qi of the solve of the spread of a unit force e_b at qj.  (a, b) = (1, 0) gives
    J_i P S_j; (0, eta) the Stokes mobility -J_i (eta L)^-1 P S_j."""
    shape = (grid[2], grid[1], grid[0])
    qi = np.atleast_2d(qi)
    qj = np.atleast_2d(qj)
    m = np.zeros((DIM, DIM))
    for col in range(DIM):
        F = np.zeros((1, DIM))
        F[0, col] = 1.0
        x = spectral_solve(spread(F, qj, kernel, h, shape), a, b, h)
        m[:, col] = interpolate(x, qi, kernel, h)[0]
    return m


def jps_deviation(q, grid, kernel, h):
    """dI(q) = (3/2) dV (J P S)(q) - I (Sec. III.A.2, Fig. JPS: d dV J P S / (d-1) ~ I)."""
    dv = blob_volume(kernel, h)
    return 1.5 * dv * coupling_matrix(q, q, grid, kernel, h) - np.eye(DIM)


def mobility(q, grid, kernel, h, eta):
    """Single-blob mobility mu(q) = -J L^-1 S of the steady Stokes problem eta L v - grad pi
    + S F = 0, div v = 0 (Sec. III.A.2), zero mean flow."""
    return coupling_matrix(q, q, grid, kernel, h, a=0.0, b=eta)


def hydrodynamic_radius(mu, eta, box_length):
    """R_H of an isolated sphere from the mobility mu of its periodic images on a cubic
    lattice of side L: 6 pi eta mu = 1/R_H - 2.8373/L (Hasimoto's first-order lattice
    correction, J. Fluid Mech. 5 (1959); the paper extrapolates R_H without saying how)."""
    return 1.0 / (6.0 * np.pi * eta * mu + 2.8373 / box_length)


# ---------------------------------------------------------------------------
# The time step (Sec. III.C "Summary of Algorithm"; Appendix C)
# ---------------------------------------------------------------------------
class Params:
    """Physical and numerical parameters of one simulation."""

    def __init__(self, grid, h=1.0, rho=1.0, eta=1.0, kT=0.0, dt=0.05, kernel=4,
                 seed=1, slip="visc", advection=True, trap_k=0.0, trap_center=(0.0, 0.0, 0.0),
                 thermal_drift=False, wca_epsilon=0.0, wca_sigma=1.0):
        self.grid = tuple(int(n) for n in grid)            # (Nx, Ny, Nz)
        self.h, self.rho, self.eta, self.kT, self.dt = float(h), float(rho), float(eta), float(kT), float(dt)
        self.kernel, self.seed, self.slip, self.advection = int(kernel), int(seed), slip, bool(advection)
        # harmonic trap V = k r^2 / 2 of the temporal accuracy test (Sec. III.D)
        self.trap_k = float(trap_k)
        self.trap_center = np.asarray(trap_center, dtype=np.float64).reshape(3)
        # thermal drift forcing kT m~_f/m~ d(delta_a)/dq (Appendix B.2, Eq. thermal_drift)
        self.thermal_drift = bool(thermal_drift)
        # purely repulsive truncated Lennard-Jones (WCA) pair potential (Sec. IV.A, Eq. WCA)
        self.wca_epsilon, self.wca_sigma = float(wca_epsilon), float(wca_sigma)

    @property
    def shape(self):
        nx, ny, nz = self.grid
        return (nz, ny, nx)

    @property
    def box(self):
        return np.array(self.grid, dtype=np.float64) * self.h


class State:
    """Fluid and blob state at time level n."""

    def __init__(self, v, q, u, me, force, adv_prev=None, slip_g=None, step=0):
        self.v = np.asarray(v, dtype=np.float64)                  # (3, Nz, Ny, Nx)
        self.q = np.atleast_2d(np.asarray(q, dtype=np.float64))   # (Nb, 3)
        nb = self.q.shape[0]
        self.u = np.asarray(u, dtype=np.float64).reshape(nb, 3)
        self.me = np.asarray(me, dtype=np.float64).reshape(nb)
        self.force = np.asarray(force, dtype=np.float64).reshape(nb, 3)
        self.adv_prev = None if adv_prev is None else np.asarray(adv_prev, dtype=np.float64)
        self.slip_g = np.zeros((nb, 3)) if slip_g is None else np.asarray(slip_g, dtype=np.float64).reshape(nb, 3)
        self.step = int(step)

    def copy(self):
        return State(self.v.copy(), self.q.copy(), self.u.copy(), self.me.copy(), self.force.copy(),
                     None if self.adv_prev is None else self.adv_prev.copy(), self.slip_g.copy(), self.step)


def wrap_positions(q, box):
    """Periodic images into [0, L) per axis."""
    out = np.mod(q, box)
    return np.where(out >= box, out - box, out)


def total_momentum(state, prm):
    """P = rho dV_f sum_k v_k + sum_i m_e,i u_i  (Sec. II, after Eq. no_slip)."""
    fluid = prm.rho * prm.h ** 3 * state.v.reshape(DIM, -1).sum(axis=1)
    return fluid + (state.me[:, None] * state.u).sum(axis=0)


def explicit_rhs(v, adv_prev, step, prm):
    """Dense part of the right-hand side of Eq. provisional_step-1.

    r = (rho/dt) v + (eta/2) L v + div Sigma^n - (3/2 A^n - 1/2 A^{n-1}).
    Returns (r, A^n).  A^{n-1} = None means no history: A^{-1} := A^n.
    """
    h = prm.h
    if prm.advection:
        adv_n = advection(v, prm.rho, h)
    else:
        adv_n = np.zeros_like(v)
    adv_old = adv_n if adv_prev is None else adv_prev
    ncell = int(np.prod(prm.shape))
    r = (prm.rho / prm.dt) * v + 0.5 * prm.eta * vector_laplacian(v, h)
    if prm.kT > 0.0:
        s = np.sqrt(prm.kT * prm.eta / (h ** 3 * prm.dt))
        nx, ny, _ = prm.grid
        z = stress_normals(prm.seed, step, ncell, nx * ny)
        r = r + stochastic_flux_divergence(z, s, h, prm.shape)
    r = r - (1.5 * adv_n - 0.5 * adv_old)
    return r, adv_n


def trap_force(q, prm):
    """Force of the harmonic potential V(r) = k r^2 / 2 of the temporal accuracy test
    (Sec. III.D, the experiment of Eq. E_dt_definition): F = -k (q - c).  Reading: in
    the periodic box, q - c is the displacement to the nearest image of the centre c."""
    q = np.atleast_2d(q)
    if prm.trap_k == 0.0:
        return np.zeros_like(q)
    d = q - prm.trap_center
    d = d - prm.box * np.round(d / prm.box)
    return -prm.trap_k * d


def wca_energy(q, prm):
    """U = sum over pairs i < j of V(r_ij), V(r) = 4 eps ((s/r)^12 - (s/r)^6) + eps for
    r < 2^(1/6) s, 0 beyond (Sec. IV.A, Eq. WCA); r_ij to the nearest image."""
    q = np.atleast_2d(q)
    eps, sig = prm.wca_epsilon, prm.wca_sigma
    u = 0.0
    for i in range(q.shape[0]):
        d = q[i] - q[i + 1:]
        d -= prm.box * np.round(d / prm.box)
        r = np.sqrt((d * d).sum(axis=1))
        r = r[r < 2.0 ** (1.0 / 6.0) * sig]
        u += np.sum(4.0 * eps * ((sig / r) ** 12 - (sig / r) ** 6) + eps)
    return u


def wca_force(q, prm):
    """F_i = -dU/dq_i of the WCA potential: sum_j 24 eps (2 s^12/r^14 - s^6/r^8) d_ij over
    the pairs within the cut-off, d_ij = q_i - q_j to the nearest image (all pairs)."""
    q = np.atleast_2d(q)
    nb = q.shape[0]
    if prm.wca_epsilon == 0.0 or nb < 2:
        return np.zeros_like(q)
    eps, sig = prm.wca_epsilon, prm.wca_sigma
    d = q[:, None, :] - q[None, :, :]
    d -= prm.box * np.round(d / prm.box)
    r2 = (d * d).sum(axis=2)
    np.fill_diagonal(r2, np.inf)
    inside = r2 < (2.0 ** (1.0 / 6.0) * sig) ** 2
    s6 = np.where(inside, sig ** 6 / r2 ** 3, 0.0)
    mag = np.where(inside, 24.0 * eps * (2.0 * s6 * s6 - s6) / r2, 0.0)
    return (mag[:, :, None] * d).sum(axis=1)


def icm_step(state, prm, trace=None):
    """Advance one ICM step, following the nine steps of Sec. III.C in order.

    `trace`, if a dict, receives the intermediate quantities by name.
    """
    h, rho, dt, kernel = prm.h, prm.rho, prm.dt, prm.kernel
    nu = prm.eta / rho
    shape = prm.shape
    box = prm.box
    v, q, me = state.v, state.q, state.me
    nb = q.shape[0]

    # Step 1, Eq. particle_pred: midpoint predictor; forces at q^{n+1/2} (the constant
    # external forces plus the harmonic trap and the WCA pair forces, if any).
    jv_n = interpolate(v, q, kernel, h)
    q_half = wrap_positions(q + 0.5 * dt * jv_n, box)
    force = state.force + trap_force(q_half, prm) + wca_force(q_half, prm)

    # Step 2, Eq. provisional_step-1: unperturbed fluid solve.
    r, adv_n = explicit_rhs(v, state.adv_prev, state.step, prm)
    r = r + spread(force, q_half, kernel, h, shape)
    if prm.thermal_drift and prm.kT > 0.0 and nb > 0:
        # Appendix B.2: the thermal drift, a forcing at q^{n+1/2} with weight kT m~_f / m~
        mtf = fluid_dragged_mass(kernel, h, rho)
        r = r + spread_drift(prm.kT * mtf / (mtf + me), q_half, kernel, h, shape)
    v_tilde = spectral_solve(r, rho / dt, 0.5 * prm.eta, h)

    if nb == 0 or np.all(me == 0.0):
        # Step 3: neutrally buoyant blobs; v^{n+1} = v~.
        v_new = v_tilde
        u_new = interpolate(v_new, q_half, kernel, h)
        g_new = np.zeros((nb, 3))
        extra = {}
    else:
        # Step 4, Eq. delta_u_nph / delta_u_nph_visc: slip correction, momentum change.
        j_vt = interpolate(v_tilde, q_half, kernel, h)
        if prm.slip == "visc":
            du = 0.5 * nu * dt * state.slip_g
        elif prm.slip == "full":
            du = interpolate(v, q_half, kernel, h) - jv_n + 0.5 * nu * dt * state.slip_g
        elif prm.slip == "zero":
            du = np.zeros((nb, 3))
        else:
            raise ValueError(prm.slip)
        dp = me[:, None] * (state.u - j_vt - du)

        # Step 5: inertial perturbation dv~ = m~_f / (rho (m~_f + m_e)) P S dp.
        mtf = fluid_dragged_mass(kernel, h, rho)
        coef = mtf / (rho * (mtf + me))
        dv_tilde = spectral_solve(spread(coef[:, None] * dp, q_half, kernel, h, shape), 1.0, 0.0, h)

        # Step 6, Eq. dv_eq_modified-1: viscous correction.
        j_dvt = interpolate(dv_tilde, q_half, kernel, h)
        src = spread(dp - me[:, None] * j_dvt, q_half, kernel, h, shape)
        dv = spectral_solve(src, rho, 0.5 * dt * prm.eta, h)

        # Step 7, Eq. update_v.
        v_new = v_tilde + dv
        # Step 8, Eq. update_u: momentum-conserving blob velocity.
        u_new = j_vt + j_dvt + du
        # Lagged viscous slip term J^{n+1/2} L dv^{n+1/2}, used by the next step.
        g_new = interpolate(vector_laplacian(dv, h), q_half, kernel, h)
        extra = dict(j_vt=j_vt, du=du, dp=dp, dv_tilde=dv_tilde, j_dvt=j_dvt, dv=dv)

    # Step 9, Eq. update_q: midpoint position update.
    q_new = wrap_positions(q + 0.5 * dt * interpolate(v_new + v, q_half, kernel, h), box)

    if trace is not None:
        trace.update(dict(jv_n=jv_n, q_half=q_half, force_half=force, rhs=r, adv_n=adv_n, v_tilde=v_tilde), **extra)
    return State(v_new, q_new, u_new, me, state.force, adv_n, g_new, state.step + 1)
