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

constexpr int TX = 32, TY = 16;     // cells per block in x and y (one thread each)
constexpr int HX = TX + 2, HY = TY + 2;
constexpr int HALO = HX * HY;       // cells of one plane with a one-cell halo
constexpr int NT = TX * TY;         // threads per block
constexpr int PER = (HALO + NT - 1) / NT;   // halo cells loaded per thread

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Shared-memory rings of the marching block: velocity planes of the three components
// and planes of the six stress normals, each with a one-cell halo in x and y.  Plane k
// reads slots k-1, k, k+1 and writes k+2 (mod 4): with four slots the slot it writes
// was last read by plane k-2, which every thread has finished when it passes plane
// k's first barrier, so one barrier per plane suffices.
constexpr int kRing = 4;
template <typename R>
struct RhsSmem {
  R v[kRing][3][HY][HX];
  R z[kRing][6][HY][HX];
};

// One plane of stress normals (with halo) into ring slot `slot`.  Each thread first
// draws the normals of its own cell (no divergence), then the first HALO - NT threads
// draw the halo cells, computing only what their neighbours read: x-1 needs Z_xx,
// y-1 Z_yy, x+1 Z_xy and Z_xz, y+1 Z_xy and Z_yz; the corners nothing.
constexpr int NHALO = 2 * HX + 2 * TY;   // ring of halo cells around the TX x TY tile

template <typename R>
__device__ __forceinline__ void gen_plane(RhsSmem<R>& sm, int slot, int i0, int j0, int k, const GridParams& g,
                                          uint32_t step, int tid) {
  const int kk = wrapi(k, g.nz);
  {
    const int tx = tid % TX, ty = tid / TX;
    const int gi = wrapi(i0 + tx, g.nx), gj = wrapi(j0 + ty, g.ny);
    R z[6];
    cell_normals<R>((uint32_t)(gi + g.nx * (gj + g.ny * kk)), step, g.key0, g.key1, z);
#pragma unroll
    for (int c = 0; c < 6; ++c) sm.z[slot][c][ty + 1][tx + 1] = z[c];
  }
  for (int h = tid; h < NHALO; h += NT) {
    int hx, hy;
    if (h < HX) {                 // bottom row y = -1
      hx = h;
      hy = 0;
    } else if (h < 2 * HX) {      // top row y = TY
      hx = h - HX;
      hy = HY - 1;
    } else if (h < 2 * HX + TY) { // left column x = -1
      hx = 0;
      hy = 1 + (h - 2 * HX);
    } else {                      // right column x = TX
      hx = HX - 1;
      hy = 1 + (h - 2 * HX - TY);
    }
    const bool xl = hx == 0, xr = hx == HX - 1, yl = hy == 0, yr = hy == HY - 1;
    if ((xl || xr) && (yl || yr)) continue;
    const int gi = wrapi(i0 - 1 + hx, g.nx), gj = wrapi(j0 - 1 + hy, g.ny);
    R z[6];
    cell_normals_masked<R>((uint32_t)(gi + g.nx * (gj + g.ny * kk)), step, g.key0, g.key1, z, xl || yl, xr || yr,
                           xr || yr);
#pragma unroll
    for (int c = 0; c < 6; ++c) sm.z[slot][c][hy][hx] = z[c];
  }
}

// Plane offsets (x + Nx y, wrapped) of the halo cells thread tid loads: cells tid,
// tid + NT, ... of the (TX+2) x (TY+2) plane; -1 past the plane.
__device__ __forceinline__ void plane_offsets(int (&off)[PER], int i0, int j0, const GridParams& g, int tid) {
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int idx = tid + t * NT;
    const int hx = idx % HX, hy = idx / HX;
    off[t] = idx < HALO ? wrapi(i0 - 1 + hx, g.nx) + g.nx * wrapi(j0 - 1 + hy, g.ny) : -1;
  }
}

// Global loads of one velocity plane (with halo) into registers.
template <typename R>
__device__ __forceinline__ void load_plane(R (&r)[PER][3], const R* __restrict__ v, const int (&off)[PER], int k,
                                           const GridParams& g) {
  const long long zo = (long long)g.nx * g.ny * wrapi(k, g.nz);
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    if (off[t] >= 0) {
      const R* p = v + zo + off[t];
#pragma unroll
      for (int c = 0; c < 3; ++c) r[t][c] = p[c * g.ncell];
    }
  }
}

// The loaded plane into ring slot `slot` (the plane's cells are stored in load order).
template <typename R>
__device__ __forceinline__ void store_plane(RhsSmem<R>& sm, int slot, const R (&r)[PER][3], int tid) {
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int idx = tid + t * NT;
    if (idx < HALO) {
#pragma unroll
      for (int c = 0; c < 3; ++c) (&sm.v[slot][c][0][0])[idx] = r[t][c];
    }
  }
}

// Marching block: TX x TY cells per plane, g.kz planes (a plan choice).  Per plane: the loads of the
// plane after next are issued first, the stress normals of the next plane are
// generated while they are in flight, then the current plane is computed entirely
// from shared memory.
template <typename R, bool NOISE>
__global__ void __launch_bounds__(NT, 2) k_rhs(const R* __restrict__ v, R* __restrict__ adv, R* __restrict__ rhs,
                                            GridParams g, const long long* __restrict__ step_dev,
                                            const int* __restrict__ hist_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RhsSmem<R>& sm = *reinterpret_cast<RhsSmem<R>*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * g.kz;
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < g.nx && j < g.ny;
  const uint32_t step = (uint32_t)(*step_dev);
  const bool hist = *hist_dev != 0;
  const long long nc = g.ncell;
  const R rho = (R)g.rho, inv_h = (R)(1.0 / g.h), inv_h2 = (R)(1.0 / (g.h * g.h));
  const R rho_dt = (R)(g.rho / g.dt), half_eta = (R)(0.5 * g.eta);
  const double s_amp = sqrt(g.kT * g.eta / (g.h * g.h * g.h * g.dt));
  const R sd = (R)(2.0 * s_amp * (1.0 / g.h)), so = (R)(1.4142135623730951 * s_amp * (1.0 / g.h));
  const R adv_on = g.advection ? R(1) : R(0);
  const R h2 = R(0.5);
  const int lx = tx + 1, ly = ty + 1;

  R pre[PER][3];
  int off[PER];
  plane_offsets(off, i0, j0, g, tid);
  load_plane<R>(pre, v, off, k0 - 1, g);
  store_plane<R>(sm, 0, pre, tid);
  load_plane<R>(pre, v, off, k0, g);
  store_plane<R>(sm, 1, pre, tid);
  load_plane<R>(pre, v, off, k0 + 1, g);
  if (NOISE) {
    gen_plane<R>(sm, 0, i0, j0, k0 - 1, g, step, tid);
    gen_plane<R>(sm, 1, i0, j0, k0, g, step, tid);
  }
  const int kend = min(k0 + g.kz, g.nz);
  for (int k = k0; k < kend; ++k) {
    const int kk = k - k0;
    const int sp = kk % kRing, sc = (kk + 1) % kRing, sn = (kk + 2) % kRing;
    store_plane<R>(sm, sn, pre, tid);                       // plane k+1
    long long o = 0;
    R ao[3] = {R(0), R(0), R(0)};
    if (active) {
      o = i + (long long)g.nx * (j + (long long)g.ny * k);
      if (hist) {
        ao[0] = adv[o];
        ao[1] = adv[nc + o];
        ao[2] = adv[2 * nc + o];
      }
    }
    if (k + 1 < kend) load_plane<R>(pre, v, off, k + 2, g);   // in flight during the noise
    if (NOISE) gen_plane<R>(sm, sn, i0, j0, k + 1, g, step, tid);
    __syncthreads();
    if (active) {
      const auto P = sm.v[sp];
      const auto C = sm.v[sc];
      const auto N = sm.v[sn];
      // component x
      const R x_c = C[0][ly][lx], x_xp = C[0][ly][lx + 1], x_xm = C[0][ly][lx - 1];
      const R x_yp = C[0][ly + 1][lx], x_ym = C[0][ly - 1][lx], x_zp = N[0][ly][lx], x_zm = P[0][ly][lx];
      const R x_xpym = C[0][ly - 1][lx + 1], x_xpzm = P[0][ly][lx + 1];
      // component y
      const R y_c = C[1][ly][lx], y_xp = C[1][ly][lx + 1], y_xm = C[1][ly][lx - 1];
      const R y_yp = C[1][ly + 1][lx], y_ym = C[1][ly - 1][lx], y_zp = N[1][ly][lx], y_zm = P[1][ly][lx];
      const R y_ypxm = C[1][ly + 1][lx - 1], y_ypzm = P[1][ly + 1][lx];
      // component z
      const R z_c = C[2][ly][lx], z_xp = C[2][ly][lx + 1], z_xm = C[2][ly][lx - 1];
      const R z_yp = C[2][ly + 1][lx], z_ym = C[2][ly - 1][lx], z_zp = N[2][ly][lx], z_zm = P[2][ly][lx];
      const R z_zpxm = N[2][ly][lx - 1], z_zpym = N[2][ly - 1][lx];

      // edge products ut_a ut_b at edge index e: ut_a = (v_a[e] + v_a[e-e_b])/2, ut_b = (v_b[e] + v_b[e-e_a])/2
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
      const R lapx = (x_xp + x_xm + x_yp + x_ym + x_zp + x_zm - R(6) * x_c) * inv_h2;
      const R lapy = (y_xp + y_xm + y_yp + y_ym + y_zp + y_zm - R(6) * y_c) * inv_h2;
      const R lapz = (z_xp + z_xm + z_yp + z_ym + z_zp + z_zm - R(6) * z_c) * inv_h2;
      R fx = R(0), fy = R(0), fz = R(0);
      if (NOISE) {
        const auto ZC = sm.z[sc];
        const auto ZP = sm.z[sp];
        const auto ZN = sm.z[sn];
        // divergence of the stress at the faces: Sigma_aa at cells, Sigma_ab on edges
        fx = sd * (ZC[0][ly][lx] - ZC[0][ly][lx - 1]) + so * (ZC[3][ly + 1][lx] - ZC[3][ly][lx]) +
             so * (ZN[4][ly][lx] - ZC[4][ly][lx]);
        fy = sd * (ZC[1][ly][lx] - ZC[1][ly - 1][lx]) + so * (ZC[3][ly][lx + 1] - ZC[3][ly][lx]) +
             so * (ZN[5][ly][lx] - ZC[5][ly][lx]);
        fz = sd * (ZC[2][ly][lx] - ZP[2][ly][lx]) + so * (ZC[4][ly][lx + 1] - ZC[4][ly][lx]) +
             so * (ZC[5][ly + 1][lx] - ZC[5][ly][lx]);
      }
      if (!hist) {
        ao[0] = ax;
        ao[1] = ay;
        ao[2] = az;
      }
      adv[o] = ax;
      adv[nc + o] = ay;
      adv[2 * nc + o] = az;
      rhs[o] = rho_dt * x_c + half_eta * lapx + fx - (R(1.5) * ax - R(0.5) * ao[0]);
      rhs[nc + o] = rho_dt * y_c + half_eta * lapy + fy - (R(1.5) * ay - R(0.5) * ao[1]);
      rhs[2 * nc + o] = rho_dt * z_c + half_eta * lapz + fz - (R(1.5) * az - R(0.5) * ao[2]);
    }
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

// Peak FMA rate: kFmaChains independent dependent chains x = x * a + b per thread,
// `iters` rounds; a = 1 - 2^-20 and b = 2^-30 keep every value normal and bounded.
// The sum of the chains is stored only if it equals a value it cannot take, so the
// work is not removed.
constexpr int kFmaChains = 8;
template <typename R>
__global__ void __launch_bounds__(256) k_fma_chain(R* __restrict__ out, int iters, R a, R b) {
  R x[kFmaChains];
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) x[c] = R(1) + R(threadIdx.x + c) * R(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
  }
  R sum = R(0);
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) sum += x[c];
  if (out != nullptr && sum == R(-1)) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

template <typename R>
size_t rhs_smem() { return sizeof(RhsSmem<R>); }

}  // namespace

template <typename R>
void explicit_rhs(const GridParams& g, const R* v, R* adv, R* rhs, const long long* step_dev, const int* hist_dev,
                  cudaStream_t st) {
  const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + g.kz - 1) / g.kz);
  const dim3 block(TX, TY);
  if (g.kT > 0.0)
    k_rhs<R, true><<<grid, block, rhs_smem<R>(), st>>>(v, adv, rhs, g, step_dev, hist_dev);
  else
    k_rhs<R, false><<<grid, block, rhs_smem<R>(), st>>>(v, adv, rhs, g, step_dev, hist_dev);
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

double fma_rate(int precision, int iters, int blocks_per_sm, cudaStream_t st, double* seconds) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1.0;
  const int blocks = nsm * blocks_per_sm, threads = 256;
  void* out = nullptr;   // k_fma_chain stores nothing through a null pointer
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
  float ms = 0.0f;
  for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, st);
    if (precision == 64)
      k_fma_chain<double><<<blocks, threads, 0, st>>>((double*)out, iters, 1.0 - 0x1p-20, 0x1p-30);
    else
      k_fma_chain<float><<<blocks, threads, 0, st>>>((float*)out, iters, 1.0f - 0x1p-20f, 0x1p-30f);
    cudaEventRecord(e1, st);
  }
  const cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || ms <= 0.0f) return -1.0;
  if (seconds) *seconds = ms * 1e-3;
  return 2.0 * kFmaChains * (double)iters * blocks * threads / (ms * 1e-3);
}

void grid_prepare() {
  cudaFuncSetAttribute(k_rhs<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<float>());
  cudaFuncSetAttribute(k_rhs<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<double>());
  cudaFuncSetAttribute(k_rhs<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<float>());
  cudaFuncSetAttribute(k_rhs<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<double>());
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
