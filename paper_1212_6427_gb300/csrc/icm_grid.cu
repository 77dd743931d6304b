// Grid kernels of the ICM step (arXiv:1212.6427, Sec. III.B-C):
//   * the explicit right-hand side of Eq. provisional_step-1, one fused pass:
//       r = (rho/dt) v + (eta/2) L v + div Sigma^n - (3/2 A^n - 1/2 A^{n-1}),
//     with the stochastic stress Sigma^n = sqrt(kT eta/(dV_f dt)) (W + W^T) drawn
//     from Philox4x32-10 on the fly (never stored) and A = div(rho v v^T) in
//     centred conservative (skew-adjoint) form, Adams-Bashforth in time
//     (Eq. Adams_Bashforth).  A^n overwrites A^{n-1} in place.
//   * FP64 compensated sums of face fields (momentum bookkeeping, Sec. II).
#include "icm_internal.h"

namespace icm {
namespace {

constexpr int TX = 32, TY = 16;     // cells per block in x and y
constexpr int KZ = 16;              // z planes marched per block
constexpr int HX = TX + 2, HY = TY + 2;

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// One (TX+2) x (TY+2) plane of stress normals (halo of one cell) into ring slot s.
template <typename R>
__device__ __forceinline__ void gen_plane(R (*ring)[6][HY][HX], int slot, int i0, int j0, int k, const GridParams& g,
                                          uint32_t step, int tid, int nthr) {
  const int kk = wrapi(k, g.nz);
  for (int idx = tid; idx < HX * HY; idx += nthr) {
    const int hx = idx % HX, hy = idx / HX;
    const int gi = wrapi(i0 - 1 + hx, g.nx);
    const int gj = wrapi(j0 - 1 + hy, g.ny);
    const uint32_t cell = (uint32_t)(gi + g.nx * (gj + g.ny * kk));
    R z[6];
    cell_normals<R>(cell, step, g.key0, g.key1, z);
#pragma unroll
    for (int c = 0; c < 6; ++c) ring[slot][c][hy][hx] = z[c];
  }
}

template <typename R, bool NOISE>
__global__ void __launch_bounds__(TX* TY) k_rhs(const R* __restrict__ v, R* __restrict__ adv, R* __restrict__ rhs,
                                               GridParams g, const long long* __restrict__ step_dev,
                                               const int* __restrict__ hist_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R(*ring)[6][HY][HX] = reinterpret_cast<R(*)[6][HY][HX]>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty, nthr = TX * TY;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * KZ;
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < g.nx && j < g.ny;
  const uint32_t step = (uint32_t)(*step_dev);
  const bool hist = *hist_dev != 0;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long nc = g.ncell;
  const R rho = (R)g.rho, inv_h = (R)(1.0 / g.h), inv_h2 = (R)(1.0 / (g.h * g.h));
  const R rho_dt = (R)(g.rho / g.dt), half_eta = (R)(0.5 * g.eta);
  const R s_amp = (R)sqrt(g.kT * g.eta / (g.h * g.h * g.h * g.dt));
  const R sd = R(2) * s_amp, so = (R)(1.4142135623730951 * sqrt(g.kT * g.eta / (g.h * g.h * g.h * g.dt)));
  const R adv_on = g.advection ? R(1) : R(0);

  if (NOISE) {
    gen_plane<R>(ring, 0, i0, j0, k0 - 1, g, step, tid, nthr);
    gen_plane<R>(ring, 1, i0, j0, k0, g, step, tid, nthr);
  }
  const int kend = min(k0 + KZ, nz);
  for (int k = k0; k < kend; ++k) {
    const int kk = k - k0;
    const int sp = kk % 3, sc = (kk + 1) % 3, sn = (kk + 2) % 3;
    if (NOISE) gen_plane<R>(ring, sn, i0, j0, k + 1, g, step, tid, nthr);
    __syncthreads();
    if (active) {
      const int im = wrapi(i - 1, nx), ip = wrapi(i + 1, nx);
      const int jm = wrapi(j - 1, ny), jp = wrapi(j + 1, ny);
      const int km = wrapi(k - 1, nz), kp = wrapi(k + 1, nz);
      const long long rc = (long long)nx * (j + (long long)ny * k);
      const long long rym = (long long)nx * (jm + (long long)ny * k), ryp = (long long)nx * (jp + (long long)ny * k);
      const long long rzm = (long long)nx * (j + (long long)ny * km), rzp = (long long)nx * (j + (long long)ny * kp);
      const long long rypzm = (long long)nx * (jp + (long long)ny * km);
      const long long rymzp = (long long)nx * (jm + (long long)ny * kp);
      const R* vx = v;
      const R* vy = v + nc;
      const R* vz = v + 2 * nc;
      // component x
      const R x_c = vx[rc + i], x_xp = vx[rc + ip], x_xm = vx[rc + im];
      const R x_yp = vx[ryp + i], x_ym = vx[rym + i], x_zp = vx[rzp + i], x_zm = vx[rzm + i];
      const R x_xpym = vx[rym + ip], x_xpzm = vx[rzm + ip];
      // component y
      const R y_c = vy[rc + i], y_xp = vy[rc + ip], y_xm = vy[rc + im];
      const R y_yp = vy[ryp + i], y_ym = vy[rym + i], y_zp = vy[rzp + i], y_zm = vy[rzm + i];
      const R y_ypxm = vy[ryp + im], y_ypzm = vy[rypzm + i];
      // component z
      const R z_c = vz[rc + i], z_xp = vz[rc + ip], z_xm = vz[rc + im];
      const R z_yp = vz[ryp + i], z_ym = vz[rym + i], z_zp = vz[rzp + i], z_zm = vz[rzm + i];
      const R z_zpxm = vz[rzp + im], z_zpym = vz[rymzp + i];

      const R h2 = R(0.5);
      // edge products ut_a ut_b, edge index e: ut_a = (v_a[e] + v_a[e-e_b])/2, ut_b = (v_b[e] + v_b[e-e_a])/2
      const R exy_c = (x_c + x_ym) * h2 * ((y_c + y_xm) * h2);
      const R exy_yp = (x_yp + x_c) * h2 * ((y_yp + y_ypxm) * h2);
      const R exy_xp = (x_xp + x_xpym) * h2 * ((y_xp + y_c) * h2);
      const R exz_c = (x_c + x_zm) * h2 * ((z_c + z_xm) * h2);
      const R exz_zp = (x_zp + x_c) * h2 * ((z_zp + z_zpxm) * h2);
      const R exz_xp = (x_xp + x_xpzm) * h2 * ((z_xp + z_c) * h2);
      const R eyz_c = (y_c + y_zm) * h2 * ((z_c + z_ym) * h2);
      const R eyz_zp = (y_zp + y_c) * h2 * ((z_zp + z_zpym) * h2);
      const R eyz_yp = (y_yp + y_ypzm) * h2 * ((z_yp + z_c) * h2);

      const R ubx_c = (x_xp + x_c) * h2, ubx_m = (x_c + x_xm) * h2;
      const R uby_c = (y_yp + y_c) * h2, uby_m = (y_c + y_ym) * h2;
      const R ubz_c = (z_zp + z_c) * h2, ubz_m = (z_c + z_zm) * h2;
      const R ax = adv_on * rho * inv_h * (ubx_c * ubx_c - ubx_m * ubx_m + exy_yp - exy_c + exz_zp - exz_c);
      const R ay = adv_on * rho * inv_h * (uby_c * uby_c - uby_m * uby_m + exy_xp - exy_c + eyz_zp - eyz_c);
      const R az = adv_on * rho * inv_h * (ubz_c * ubz_c - ubz_m * ubz_m + exz_xp - exz_c + eyz_yp - eyz_c);

      const R lx = (x_xp + x_xm + x_yp + x_ym + x_zp + x_zm - R(6) * x_c) * inv_h2;
      const R ly = (y_xp + y_xm + y_yp + y_ym + y_zp + y_zm - R(6) * y_c) * inv_h2;
      const R lz = (z_xp + z_xm + z_yp + z_ym + z_zp + z_zm - R(6) * z_c) * inv_h2;

      R fx = R(0), fy = R(0), fz = R(0);
      if (NOISE) {
        const int lx_ = tx + 1, ly_ = ty + 1;
        auto cur = ring[sc];
        auto prv = ring[sp];
        auto nxt = ring[sn];
        fx = sd * (cur[0][ly_][lx_] - cur[0][ly_][lx_ - 1]) + so * (cur[3][ly_ + 1][lx_] - cur[3][ly_][lx_]) +
             so * (nxt[4][ly_][lx_] - cur[4][ly_][lx_]);
        fy = sd * (cur[1][ly_][lx_] - cur[1][ly_ - 1][lx_]) + so * (cur[3][ly_][lx_ + 1] - cur[3][ly_][lx_]) +
             so * (nxt[5][ly_][lx_] - cur[5][ly_][lx_]);
        fz = sd * (cur[2][ly_][lx_] - prv[2][ly_][lx_]) + so * (cur[4][ly_][lx_ + 1] - cur[4][ly_][lx_]) +
             so * (cur[5][ly_ + 1][lx_] - cur[5][ly_][lx_]);
        fx *= inv_h;
        fy *= inv_h;
        fz *= inv_h;
      }
      const long long o = rc + i;
      const R ox = hist ? adv[o] : ax;
      const R oy = hist ? adv[nc + o] : ay;
      const R oz = hist ? adv[2 * nc + o] : az;
      adv[o] = ax;
      adv[nc + o] = ay;
      adv[2 * nc + o] = az;
      rhs[o] = rho_dt * x_c + half_eta * lx + fx - (R(1.5) * ax - R(0.5) * ox);
      rhs[nc + o] = rho_dt * y_c + half_eta * ly + fy - (R(1.5) * ay - R(0.5) * oy);
      rhs[2 * nc + o] = rho_dt * z_c + half_eta * lz + fz - (R(1.5) * az - R(0.5) * oz);
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void k_normals(GridParams g, uint32_t step, R* __restrict__ out) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  R z[6];
  cell_normals<R>((uint32_t)c, step, g.key0, g.key1, z);
#pragma unroll
  for (int a = 0; a < 6; ++a) out[a * g.ncell + c] = z[a];
}

__global__ void k_philox(long long n, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         uint32_t* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32x4 r = philox4x32_10(u32x4{c0 + (uint32_t)i, c1, c2, c3}, k0, k1);
  out[4 * i + 0] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// Kahan-compensated per-thread sums, FP64 tree within the block -> partial[comp][block].
template <typename R>
__global__ void k_sum_partial(const R* __restrict__ v, long long n, double* __restrict__ partial) {
  const int comp = blockIdx.y;
  const R* p = v + comp * n;
  double s = 0.0, c = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double y = (double)p[i] - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[comp * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_sum_final(const double* __restrict__ partial, int np, double* __restrict__ out) {
  const int comp = blockIdx.x;
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const double y = partial[comp * np + i] - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[comp] = red[0];
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ src, B* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (B)src[i];
}

__global__ void k_scal_before(double* scal, double dt) {
  const int a = threadIdx.x;
  if (a < 3) {
    scal[SC_K0 + a] = scal[SC_PBAR + a] + dt * scal[SC_SUMF + a];
    scal[SC_SUMSRC + a] = 0.0;
  }
}

__global__ void k_scal_after(double* scal, int inertial, long long* step_dev, int* hist_dev) {
  const int a = threadIdx.x;
  if (a < 3) scal[SC_PBAR + a] = scal[SC_K0 + a] + (inertial ? scal[SC_SUMSRC + a] : 0.0);
  if (a == 0) {
    *step_dev += 1;
    *hist_dev = 1;
  }
}

template <typename R>
size_t rhs_smem() { return (size_t)3 * 6 * HY * HX * sizeof(R); }

}  // namespace

template <typename R>
void explicit_rhs(const GridParams& g, const R* v, R* adv, R* rhs, const long long* step_dev, const int* hist_dev,
                  cudaStream_t st) {
  const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + KZ - 1) / KZ);
  const dim3 block(TX, TY);
  if (g.kT > 0.0)
    k_rhs<R, true><<<grid, block, rhs_smem<R>(), st>>>(v, adv, rhs, g, step_dev, hist_dev);
  else
    k_rhs<R, false><<<grid, block, 0, st>>>(v, adv, rhs, g, step_dev, hist_dev);
}

template <typename R>
void stress_normals(const GridParams& g, long long step, R* out, cudaStream_t st) {
  const int bs = 256;
  k_normals<R><<<(unsigned)((g.ncell + bs - 1) / bs), bs, 0, st>>>(g, (uint32_t)step, out);
}

void philox_words(long long n, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                  uint32_t* out, cudaStream_t st) {
  if (n <= 0) return;
  const int bs = 256;
  k_philox<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(n, c0, c1, c2, c3, k0, k1, out);
}

template <typename R>
void field_sums(const R* v, long long ncell, double* out_dev, double* partial_dev, int npartial, cudaStream_t st) {
  k_sum_partial<R><<<dim3(npartial, 3), 256, 0, st>>>(v, ncell, partial_dev);
  k_sum_final<<<3, 256, 0, st>>>(partial_dev, npartial, out_dev);
}

template <typename R>
void convert_to_double(const R* src, double* dst, long long n, cudaStream_t st) {
  k_convert<R, double><<<1024, 256, 0, st>>>(src, dst, n);
}
template <typename R>
void convert_from_double(const double* src, R* dst, long long n, cudaStream_t st) {
  k_convert<double, R><<<1024, 256, 0, st>>>(src, dst, n);
}

void grid_prepare() {
  cudaFuncSetAttribute(k_rhs<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<float>());
  cudaFuncSetAttribute(k_rhs<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<double>());
}

void scalars_before_step(double* scal, double dt, double, double, cudaStream_t st) {
  k_scal_before<<<1, 32, 0, st>>>(scal, dt);
}
void scalars_after_step(double* scal, double, double, double, bool inertial, long long* step_dev, int* hist_dev,
                        cudaStream_t st) {
  k_scal_after<<<1, 32, 0, st>>>(scal, inertial ? 1 : 0, step_dev, hist_dev);
}

#define ICM_INST(R)                                                                                          \
  template void explicit_rhs<R>(const GridParams&, const R*, R*, R*, const long long*, const int*, cudaStream_t); \
  template void stress_normals<R>(const GridParams&, long long, R*, cudaStream_t);                           \
  template void field_sums<R>(const R*, long long, double*, double*, int, cudaStream_t);                      \
  template void convert_to_double<R>(const R*, double*, long long, cudaStream_t);                             \
  template void convert_from_double<R>(const double*, R*, long long, cudaStream_t);
ICM_INST(float)
ICM_INST(double)
#undef ICM_INST

}  // namespace icm
