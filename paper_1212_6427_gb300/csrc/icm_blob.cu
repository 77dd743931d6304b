// Blob kernels of the ICM step (arXiv:1212.6427, Sec. III.A.1 and III.C).
//
// One warp per blob.  Lanes 0-8 build the 1-D Peskin stencils of the three
// staggered velocity components (first node and weights per axis, from the FP64
// position); the warp then walks the 3 x w^3 nodes with the x index fastest so
// that a group of lanes reads consecutive addresses, and reduces with shuffles.
//   interpolation (J v)_i = sum_k phi(q_i - r_k) v_k            (gather)
//   spreading     (S F)_k = dV_f^-1 sum_i phi(q_i - r_k) F_i    (atomicAdd scatter)
// Blob state (positions, velocities, masses, lagged slip terms) is FP64 in both
// precision modes; only the grid values are R.
#include <algorithm>

#include "icm_internal.h"
#include "icm_rows.cuh"

namespace icm {
namespace {

constexpr int kWarps = 8;

template <typename R, int K>
struct WarpStencil {
  int first[3][3];       // [component][axis] first node, wrapped into [0, n)
  R w[3][3][K + 2];      // weights; the Laplacian form uses indices 0..K+1 (zero padded)
  R d2[3][3][K + 2];     // second differences of the zero-padded weights
};

// Periodic image in [0, L), with 1/L precomputed (GB300 has little FP64 throughput,
// so the blob kernels keep their double-precision operations few).
__device__ __forceinline__ double wrap_pos(double x, double L, double inv_L) {
  double y = fma(-L, floor(x * inv_L), x);
  if (y >= L) y -= L;
  if (y < 0.0) y += L;
  return y;
}

// Lanes 0..8 fill the stencil of blob position q; `ext` adds the padded form.
template <typename R, int K>
__device__ __forceinline__ void build_stencil(WarpStencil<R, K>& S, const double q[3], const BlobParams& p, bool ext,
                                              int lane) {
  if (lane < 9) {
    const int comp = lane / 3, ax = lane % 3;
    const int n = ax == 0 ? p.nx : (ax == 1 ? p.ny : p.nz);
    const double off = (ax == comp) ? 0.0 : 0.5;
    const double s = fma(q[ax], p.inv_h, -off);
    // node 'first' + 1 is the anchor cell; offsets from it are exact small numbers in R
    const double anc = Peskin<R, K>::anchor(s);
    const long long f = (long long)anc - 1;
    const R frac = (R)(s - anc);
    R w[K];
#pragma unroll
    for (int a = 0; a < K; ++a) w[a] = Peskin<R, K>::phi(frac + R(1 - a));
    if (!ext) {
      long long fw = f % n;
      if (fw < 0) fw += n;
      S.first[comp][ax] = (int)fw;
#pragma unroll
      for (int a = 0; a < K; ++a) S.w[comp][ax][a] = w[a];
    } else {
      long long fw = (f - 1) % n;
      if (fw < 0) fw += n;
      S.first[comp][ax] = (int)fw;
      R we[K + 2];
      we[0] = R(0);
      we[K + 1] = R(0);
#pragma unroll
      for (int a = 0; a < K; ++a) we[a + 1] = w[a];
#pragma unroll
      for (int a = 0; a < K + 2; ++a) {
        const R lo = a > 0 ? we[a - 1] : R(0);
        const R hi = a < K + 1 ? we[a + 1] : R(0);
        S.w[comp][ax][a] = we[a];
        S.d2[comp][ax][a] = lo - R(2) * we[a] + hi;
      }
    }
  }
  __syncwarp();
}

__device__ __forceinline__ int wrap_add(int a, int b, int n) {
  const int t = a + b;
  return t >= n ? t - n : t;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// (J field) for the three components; result valid in every lane.  Each lane takes
// items lane, lane + 32, ... of the 3 w^3 nodes (x index fastest); the trip count is a
// compile-time constant so every load of a lane is issued before the first use.
template <typename R, int K>
__device__ __forceinline__ void gather(const WarpStencil<R, K>& S, const R* __restrict__ field, const BlobParams& p,
                                       int lane, double out[3]) {
  constexpr int W3 = K * K * K, ITEMS = 3 * W3, ROUNDS = (ITEMS + 31) / 32;
  R val[ROUNDS], wgt[ROUNDS];
#pragma unroll
  for (int j = 0; j < ROUNDS; ++j) {
    const int it = lane + 32 * j;
    val[j] = R(0);
    wgt[j] = R(0);
    if (it < ITEMS) {
      const int c = it / W3, r = it - c * W3;
      const int a = r % K, b = (r / K) % K, cz = r / (K * K);
      const int ix = wrap_add(S.first[c][0], a, p.nx);
      const int iy = wrap_add(S.first[c][1], b, p.ny);
      const int iz = wrap_add(S.first[c][2], cz, p.nz);
      wgt[j] = S.w[c][0][a] * S.w[c][1][b] * S.w[c][2][cz];
      const long long off = c * p.ncell + ix + (long long)p.nx * (iy + (long long)p.ny * iz);
      if (index_ok(off, 3 * p.ncell, p.err)) val[j] = __ldg(field + off);
    }
  }
  R acc[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int j = 0; j < ROUNDS; ++j) {
    const int it = lane + 32 * j;
    const int c = it / W3;
    const R t = wgt[j] * val[j];
    acc[0] += c == 0 ? t : R(0);
    acc[1] += c == 1 ? t : R(0);
    acc[2] += c == 2 ? t : R(0);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = (double)warp_sum(acc[c]);
}

// J (L field): gather with the discrete Laplacian of the weights (L is symmetric).
template <typename R, int K>
__device__ __forceinline__ void gather_lap(const WarpStencil<R, K>& S, const R* __restrict__ field,
                                           const BlobParams& p, int lane, double out[3]) {
  constexpr int E = K + 2, E3 = E * E * E, ITEMS = 3 * E3, ROUNDS = (ITEMS + 31) / 32;
  R acc[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int j = 0; j < ROUNDS; ++j) {
    const int it = lane + 32 * j;
    if (it < ITEMS) {
      const int c = it / E3, r = it - c * E3;
      const int a = r % E, b = (r / E) % E, cz = r / (E * E);
      const int ix = wrap_add(S.first[c][0], a, p.nx);
      const int iy = wrap_add(S.first[c][1], b, p.ny);
      const int iz = wrap_add(S.first[c][2], cz, p.nz);
      const R wx = S.w[c][0][a], wy = S.w[c][1][b], wz = S.w[c][2][cz];
      const R wgt = S.d2[c][0][a] * wy * wz + wx * S.d2[c][1][b] * wz + wx * wy * S.d2[c][2][cz];
      const long long off = c * p.ncell + ix + (long long)p.nx * (iy + (long long)p.ny * iz);
      const R t = index_ok(off, 3 * p.ncell, p.err) ? wgt * __ldg(field + off) : R(0);
      acc[0] += c == 0 ? t : R(0);
      acc[1] += c == 1 ? t : R(0);
      acc[2] += c == 2 ? t : R(0);
    }
  }
  const double inv_h2 = 1.0 / (p.h * p.h);
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = (double)warp_sum(acc[c]) * inv_h2;
}

template <typename R, int K>
__device__ __forceinline__ void scatter(const WarpStencil<R, K>& S, R* __restrict__ field, const BlobParams& p,
                                        int lane, const double vec[3]) {
  constexpr int W3 = K * K * K, ITEMS = 3 * W3, ROUNDS = (ITEMS + 31) / 32;
  const double inv_dvf = 1.0 / (p.h * p.h * p.h);
  const R amp[3] = {(R)(vec[0] * inv_dvf), (R)(vec[1] * inv_dvf), (R)(vec[2] * inv_dvf)};
#pragma unroll
  for (int j = 0; j < ROUNDS; ++j) {
    const int it = lane + 32 * j;
    if (it < ITEMS) {
      const int c = it / W3, r = it - c * W3;
      const int a = r % K, b = (r / K) % K, cz = r / (K * K);
      const int ix = wrap_add(S.first[c][0], a, p.nx);
      const int iy = wrap_add(S.first[c][1], b, p.ny);
      const int iz = wrap_add(S.first[c][2], cz, p.nz);
      const R wgt = S.w[c][0][a] * S.w[c][1][b] * S.w[c][2][cz];
      const long long off = c * p.ncell + ix + (long long)p.nx * (iy + (long long)p.ny * iz);
      if (index_ok(off, 3 * p.ncell, p.err)) atomicAdd(field + off, wgt * amp[c]);
    }
  }
}

__device__ __forceinline__ void load3(const double* a, long long b, double out[3]) {
  out[0] = a[3 * b];
  out[1] = a[3 * b + 1];
  out[2] = a[3 * b + 2];
}
__device__ __forceinline__ void store3(double* a, long long b, const double v[3]) {
  a[3 * b] = v[0];
  a[3 * b + 1] = v[1];
  a[3 * b + 2] = v[2];
}

// The per-component FP64 arithmetic of a blob runs on lanes 0-2 (one component each):
// on GB300 every FP64 warp instruction is expensive, so three lanes doing one
// component beat one lane doing three.
__device__ __forceinline__ double pick3(const double v[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }

#define ICM_WARP_SETUP                                                  \
  __shared__ WarpStencil<R, K> sten[kWarps];                            \
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;            \
  const long long b = (long long)blockIdx.x * kWarps + wid;             \
  if (b >= s.nb) return;                                                \
  WarpStencil<R, K>& S = sten[wid];

// Step 1 (Eq. particle_pred): w0 = J^n v^n, q^{n+1/2} = q^n + dt/2 w0; also
// w1 = J^{n+1/2} v^n, needed by the position update (Eq. update_q) and the full slip.
// With a harmonic trap (Sec. III.D), the force at q^{n+1/2}, F - k d (d to the nearest
// image of the centre), goes to fe and dt times its trap part to the prescribed grid
// sum K0 of the first solve (one atomic per block and component).
// Blob b of the predictor, by one warp; returns (in lanes 0-2) the trap force component.
template <typename R, int K>
__device__ __forceinline__ double predict_blob(const BlobParams& p, const BlobState& s, const R* __restrict__ v,
                                               long long b, int lane, WarpStencil<R, K>& S) {
  double q[3], w0[3], qh[3], w1[3];
  load3(s.q, b, q);
  build_stencil<R, K>(S, q, p, false, lane);
  gather<R, K>(S, v, p, lane, w0);
  // every lane needs q^{n+1/2} for the second stencil; lanes 0-2 compute one axis each
  const int ax = lane < 3 ? lane : 0;
  const double mine = wrap_pos(fma(0.5 * p.dt, pick3(w0, ax), pick3(q, ax)), p.box[ax], p.inv_box[ax]);
  for (int a = 0; a < 3; ++a) qh[a] = __shfl_sync(0xffffffffu, mine, a);
  __syncwarp();
  build_stencil<R, K>(S, qh, p, false, lane);
  gather<R, K>(S, v, p, lane, w1);
  if (lane == 0) {
    store3(s.w0, b, w0);
    store3(s.qh, b, qh);
    store3(s.w1, b, w1);
  }
  double ftrap = 0.0;
  if (p.trap_k != 0.0 && lane < 3) {
    double d = mine - p.trap_c[lane];
    d = fma(-p.box[lane], rint(d * p.inv_box[lane]), d);
    ftrap = -p.trap_k * d;
    s.fe[3 * b + lane] = s.f[3 * b + lane] + ftrap;
  }
  return ftrap;
}

template <typename R, int K>
__global__ void __launch_bounds__(32 * kWarps) k_predict(BlobParams p, BlobState s, const R* __restrict__ v) {
  __shared__ WarpStencil<R, K> sten[kWarps];
  __shared__ double red[kWarps][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kWarps + wid;
  double ftrap = 0.0;
  if (b < s.nb) ftrap = predict_blob<R, K>(p, s, v, b, lane, sten[wid]);
  if (p.trap_k == 0.0) return;   // uniform over the launch
  if (lane < 3) red[wid][lane] = ftrap;
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w][threadIdx.x];
    atomicAdd(&s.scal[SC_K0 + threadIdx.x], p.dt * t);
  }
}

// Step 4 (Eq. delta_u_nph[_visc]): slip correction du and momentum change
// dp = m_e (u^n - J v~ - du); cdp = m~_f / (rho (m~_f + m_e)) dp for step 5.
template <typename R, int K>
__device__ __forceinline__ void dp_blob(const BlobParams& p, const BlobState& s, const R* __restrict__ vt, long long b,
                                        int lane, WarpStencil<R, K>& S) {
  double qh[3], jvt[3];
  load3(s.qh, b, qh);
  build_stencil<R, K>(S, qh, p, false, lane);
  gather<R, K>(S, vt, p, lane, jvt);
  if (lane < 3) {
    const int a = lane;
    const long long i = 3 * b + a;
    const double me = s.me[b];
    const double visc = 0.5 * (p.eta / p.rho) * p.dt;
    const double coef = p.mtf / (p.rho * (p.mtf + me));
    const double jv = pick3(jvt, a);
    double du = p.slip == 1 ? 0.0 : visc * s.g[i];
    if (p.slip == 2) du += s.w1[i] - s.w0[i];
    const double dp = me * (s.u[i] - jv - du);
    s.jvt[i] = jv;
    s.du[i] = du;
    s.dp[i] = dp;
    s.cdp[i] = coef * dp;
  }
}

template <typename R, int K>
__global__ void __launch_bounds__(32 * kWarps) k_dp(BlobParams p, BlobState s, const R* __restrict__ vt) {
  ICM_WARP_SETUP
  dp_blob<R, K>(p, s, vt, b, lane, S);
}

// Steps 6-8: J dv~, the source dp - m_e J dv~ of the viscous correction, and the
// momentum-conserving velocity u^{n+1} = J (v~ + dv~) + du (Eq. update_u).  The
// grid sum of the source feeds the FP64 momentum bookkeeping.
// Blob b of the steps 6-8 kernel; returns (in lane a < 3) component a of its source.
template <typename R, int K>
__device__ __forceinline__ double inertial_blob(const BlobParams& p, const BlobState& s, const R* __restrict__ dvt,
                                                long long b, int lane, WarpStencil<R, K>& S) {
  double qh[3], jd[3];
  load3(s.qh, b, qh);
  build_stencil<R, K>(S, qh, p, false, lane);
  gather<R, K>(S, dvt, p, lane, jd);
  double sr = 0.0;
  if (lane < 3) {
    const int a = lane;
    const long long i = 3 * b + a;
    const double jv = pick3(jd, a);
    sr = s.dp[i] - s.me[b] * jv;
    s.src[i] = sr;
    s.u[i] = s.jvt[i] + jv + s.du[i];
  }
  return sr;
}

template <typename R, int K>
__global__ void __launch_bounds__(32 * kWarps) k_inertial(BlobParams p, BlobState s, const R* __restrict__ dvt) {
  __shared__ double red[kWarps][3];
  __shared__ WarpStencil<R, K> sten[kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kWarps + wid;
  double src = 0.0;
  if (b < s.nb) src = inertial_blob<R, K>(p, s, dvt, b, lane, sten[wid]);
  if (lane < 3) red[wid][lane] = src;
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w][threadIdx.x];
    atomicAdd(&s.scal[SC_SUMSRC + threadIdx.x], t);
  }
}

// Step 9 (Eq. update_q): q^{n+1} = q^n + dt/2 (J^{n+1/2} v^{n+1} + J^{n+1/2} v^n).
// Inertial path: store the lagged slip term g = J^{n+1/2} L dv.  Neutral path:
// u^{n+1} = J^{n+1/2} v^{n+1}, g = 0.  Raises CFL / non-finite flags.
template <typename R, int K>
__device__ __forceinline__ void finish_blob(const BlobParams& p, const BlobState& s, const R* __restrict__ vn,
                                            const R* __restrict__ dv, int inertial, long long b, int lane,
                                            WarpStencil<R, K>& S) {
  double qh[3], jv[3], g[3] = {0.0, 0.0, 0.0};
  load3(s.qh, b, qh);
  build_stencil<R, K>(S, qh, p, false, lane);
  gather<R, K>(S, vn, p, lane, jv);
  if (inertial) {
    __syncwarp();
    build_stencil<R, K>(S, qh, p, true, lane);
    gather_lap<R, K>(S, dv, p, lane, g);
  }
  if (lane < 3) {
    const int a = lane;
    const long long i = 3 * b + a;
    const double jva = pick3(jv, a);
    const double u = inertial ? s.u[i] : jva;
    const double qn = wrap_pos(fma(0.5 * p.dt, jva + s.w1[i], s.q[i]), p.box[a], p.inv_box[a]);
    s.q[i] = qn;
    s.u[i] = u;
    s.g[i] = pick3(g, a);
    if (!isfinite(qn) || !isfinite(u)) atomicOr(s.err, DEV_ERR_NONFINITE);
    if (fabs(u) * p.dt > p.h) atomicOr(s.err, DEV_ERR_CFL);
  }
}

template <typename R, int K>
__global__ void __launch_bounds__(32 * kWarps) k_finish(BlobParams p, BlobState s, const R* __restrict__ vn,
                                                        const R* __restrict__ dv, int inertial) {
  ICM_WARP_SETUP
  finish_blob<R, K>(p, s, vn, dv, inertial, b, lane, S);
}

template <typename R, int K>
__global__ void __launch_bounds__(32 * kWarps) k_spread(BlobParams p, long long nb, const double* __restrict__ qv,
                                                        const double* __restrict__ vec, R* __restrict__ field) {
  __shared__ WarpStencil<R, K> sten[kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kWarps + wid;
  if (b >= nb) return;
  WarpStencil<R, K>& S = sten[wid];
  double q[3], f[3];
  load3(qv, b, q);
  load3(vec, b, f);
  build_stencil<R, K>(S, q, p, false, lane);
  scatter<R, K>(S, field, p, lane, f);
}

template <typename R, int K>
__global__ void __launch_bounds__(32 * kWarps) k_interp(BlobParams p, long long nb, const double* __restrict__ qv,
                                                        const R* __restrict__ field, int lap, double* __restrict__ out) {
  __shared__ WarpStencil<R, K> sten[kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kWarps + wid;
  if (b >= nb) return;
  WarpStencil<R, K>& S = sten[wid];
  double q[3], r[3];
  load3(qv, b, q);
  build_stencil<R, K>(S, q, p, lap != 0, lane);
  if (lap)
    gather_lap<R, K>(S, field, p, lane, r);
  else
    gather<R, K>(S, field, p, lane, r);
  if (lane == 0) store3(out, b, r);
}

// Thermal drift (Appendix B.2, Eq. thermal_drift, kernel-derivative form): component c
// gets kT m~_f/(m~_f + m_e) dV_f^-1 (1/h) phi'(s_c) phi(s_a) phi(s_b) at q^{n+1/2}.
// One warp per blob; lanes 0-8 build the weights and, for the component's own axis,
// the derivative weights.
template <typename R, int K>
__global__ void __launch_bounds__(32 * kWarps) k_spread_drift(BlobParams p, BlobState s, R* __restrict__ field) {
  __shared__ WarpStencil<R, K> sten[kWarps];
  __shared__ R dw[kWarps][3][K];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kWarps + wid;
  if (b >= s.nb) return;
  WarpStencil<R, K>& S = sten[wid];
  double q[3];
  load3(s.qh, b, q);
  build_stencil<R, K>(S, q, p, false, lane);
  if (lane < 3) {   // derivative weights of component `lane` along its own axis (offset 0)
    const double sa = q[lane] * p.inv_h;
    const double anc = Peskin<R, K>::anchor(sa);
    const R frac = (R)(sa - anc);
#pragma unroll
    for (int a = 0; a < K; ++a) dw[wid][lane][a] = Peskin<R, K>::dphi(frac + R(1 - a)) * (R)p.inv_h;
  }
  __syncwarp();
  const double mtf = p.mtf;
  const R amp = (R)(p.kT * mtf / (mtf + s.me[b]) / (p.h * p.h * p.h));
  constexpr int W3 = K * K * K, ITEMS = 3 * W3;
  for (int it = lane; it < ITEMS; it += 32) {
    const int c = it / W3, r = it - c * W3;
    const int a = r % K, bb = (r / K) % K, cz = r / (K * K);
    const int ix = wrap_add(S.first[c][0], a, p.nx);
    const int iy = wrap_add(S.first[c][1], bb, p.ny);
    const int iz = wrap_add(S.first[c][2], cz, p.nz);
    const R wx = c == 0 ? dw[wid][0][a] : S.w[c][0][a];
    const R wy = c == 1 ? dw[wid][1][bb] : S.w[c][1][bb];
    const R wz = c == 2 ? dw[wid][2][cz] : S.w[c][2][cz];
    const long long off = c * p.ncell + ix + (long long)p.nx * (iy + (long long)p.ny * iz);
    if (index_ok(off, 3 * p.ncell, p.err)) atomicAdd(field + off, wx * wy * wz * amp);
  }
}

inline unsigned nblocks(long long nb) { return (unsigned)((nb + kWarps - 1) / kWarps); }

// ---------------------------------------------------------------------------
// Stages over every member of a batch: one warp per blob of any member.  The member's
// kernel width is read at run time (uniform over the warp), the stencil lives in a
// shared slot large enough for either width, and the block-level sums of the
// single-simulation kernels become one FP64 atomic per warp and component (a block may
// hold blobs of several members).
// ---------------------------------------------------------------------------
template <typename R>
struct BatchSlot {
  __align__(16) unsigned char raw[sizeof(WarpStencil<R, 4>) > sizeof(WarpStencil<R, 3>) ? sizeof(WarpStencil<R, 4>)
                                                                                         : sizeof(WarpStencil<R, 3>)];
  template <int K> __device__ WarpStencil<R, K>& as() { return *reinterpret_cast<WarpStencil<R, K>*>(raw); }
};

#define ICM_BATCH_SETUP                                                 \
  __shared__ BatchSlot<R> slots[kWarps];                                \
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;            \
  const long long gb = (long long)blockIdx.x * kWarps + wid;            \
  if (gb >= nbt) return;                                                \
  const BlobMember& m = mem[member_of[gb]];                             \
  const BlobParams p = m.p;                                             \
  const BlobState s = m.s;                                              \
  const long long b = gb - m.b0;                                        \
  BatchSlot<R>& slot = slots[wid];

template <typename R>
__global__ void __launch_bounds__(32 * kWarps) k_bpredict(const BlobMember* __restrict__ mem,
                                                          const int* __restrict__ member_of, long long nbt) {
  ICM_BATCH_SETUP
  const R* v = (const R*)m.v;
  const double ft = p.kernel == 3 ? predict_blob<R, 3>(p, s, v, b, lane, slot.template as<3>())
                                  : predict_blob<R, 4>(p, s, v, b, lane, slot.template as<4>());
  if (p.trap_k != 0.0 && lane < 3) atomicAdd(&s.scal[SC_K0 + lane], p.dt * ft);
}

template <typename R>
__global__ void __launch_bounds__(32 * kWarps) k_bspread(const BlobMember* __restrict__ mem,
                                                         const int* __restrict__ member_of, long long nbt, int which) {
  ICM_BATCH_SETUP
  const double* vec = which == BV_FORCE ? m.fvec : (which == BV_CDP ? s.cdp : s.src);
  if (vec == nullptr) return;
  double q[3], f[3];
  load3(s.qh, b, q);
  load3(vec, b, f);
  R* field = (R*)m.work;
  if (p.kernel == 3) {
    build_stencil<R, 3>(slot.template as<3>(), q, p, false, lane);
    scatter<R, 3>(slot.template as<3>(), field, p, lane, f);
  } else {
    build_stencil<R, 4>(slot.template as<4>(), q, p, false, lane);
    scatter<R, 4>(slot.template as<4>(), field, p, lane, f);
  }
}

template <typename R>
__global__ void __launch_bounds__(32 * kWarps) k_bdp(const BlobMember* __restrict__ mem,
                                                     const int* __restrict__ member_of, long long nbt) {
  ICM_BATCH_SETUP
  const R* v = (const R*)m.v;
  if (p.kernel == 3)
    dp_blob<R, 3>(p, s, v, b, lane, slot.template as<3>());
  else
    dp_blob<R, 4>(p, s, v, b, lane, slot.template as<4>());
}

template <typename R>
__global__ void __launch_bounds__(32 * kWarps) k_binertial(const BlobMember* __restrict__ mem,
                                                           const int* __restrict__ member_of, long long nbt) {
  ICM_BATCH_SETUP
  const R* w = (const R*)m.work;
  const double sr = p.kernel == 3 ? inertial_blob<R, 3>(p, s, w, b, lane, slot.template as<3>())
                                  : inertial_blob<R, 4>(p, s, w, b, lane, slot.template as<4>());
  if (lane < 3) atomicAdd(&s.scal[SC_SUMSRC + lane], sr);
}

template <typename R>
__global__ void __launch_bounds__(32 * kWarps) k_bfinish(const BlobMember* __restrict__ mem,
                                                         const int* __restrict__ member_of, long long nbt) {
  ICM_BATCH_SETUP
  const R* v = (const R*)m.v;
  const R* dv = m.inertial ? (const R*)m.work : nullptr;
  if (p.kernel == 3)
    finish_blob<R, 3>(p, s, v, dv, m.inertial, b, lane, slot.template as<3>());
  else
    finish_blob<R, 4>(p, s, v, dv, m.inertial, b, lane, slot.template as<4>());
}
#undef ICM_BATCH_SETUP

// work = 0 for every member, in 16-byte stores over the members' concatenated work
// fields (register FFT sides are even, so 3 ncell R values are a whole number of 16-byte
// words): word i belongs to the member m with prefix[m] <= i < prefix[m + 1].
__global__ void k_bzero(const BlobMember* __restrict__ mem, const long long* __restrict__ prefix, int nm,
                        long long total) {
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int a = 0, b = nm - 1;
    while (a < b) {
      const int c = (a + b + 1) / 2;
      if (prefix[c] <= i) a = c; else b = c - 1;
    }
    reinterpret_cast<float4*>(mem[a].work)[i - prefix[a]] = z;
  }
}

__global__ void k_bscal_before(const BlobMember* __restrict__ mem) {
  const BlobMember& m = mem[blockIdx.x];
  const int a = threadIdx.x;
  if (a < 3) {
    double* scal = m.s.scal;
    scal[SC_K0 + a] = scal[SC_PBAR + a] + m.p.dt * scal[SC_SUMF + a];
    scal[SC_SUMSRC + a] = 0.0;
  }
}

__global__ void k_bscal_after(const BlobMember* __restrict__ mem) {
  const BlobMember& m = mem[blockIdx.x];
  const int a = threadIdx.x;
  double* scal = m.s.scal;
  if (a < 3) scal[SC_PBAR + a] = scal[SC_K0 + a] + (m.inertial ? scal[SC_SUMSRC + a] : 0.0);
  if (a == 0) {
    *m.step_dev += 1;
    *m.hist_dev = 1;
  }
}

// ---------------------------------------------------------------------------
// Row-block bins (count, scan, fill) and the elementwise updates of the fused step
// ---------------------------------------------------------------------------
// Blob b of nb: its stencil record, zeroed accumulators, and a count in every row
// block its stencil reaches.
template <typename R>
__device__ __forceinline__ void bin_count_one(const BlobParams& p, long long nb, const double* __restrict__ q,
                                              const RowBins& bins, long long b) {
  const double qb[3] = {q[3 * b], q[3 * b + 1], q[3 * b + 2]};
  BlobStencil<R> rec;
  const BlobSpan sp = make_stencil<R>(&rec, qb, p);
  reinterpret_cast<BlobStencil<R>*>(bins.geo)[b] = rec;
  for (int k = 0; k < bins.nacc; ++k) bins.acc[k * nb + b] = 0.0;
  for_each_row_block(sp, p, [&](int blk) { atomicAdd(&bins.count[blk], 1); });
}

template <typename R>
__global__ void k_bin_count(BlobParams p, long long nb, const double* __restrict__ q, RowBins bins) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  bin_count_one<R>(p, nb, q, bins, b);
}

// Exclusive scan of the counts (one block of 1024 threads); resets the counts for the
// next build.  Each thread sums a contiguous chunk; the 1024 chunk sums are scanned
// with warp shuffles and one shared array of warp totals (two barriers).
__device__ __forceinline__ void bin_scan_block(const RowBins& bins) {
  __shared__ int warp_tot[32];
  const int n = bins.nblocks, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (n + 1023) / 1024;
  const int lo = min(t * per, n), hi = min(lo + per, n);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += bins.count[i];
  int incl = sum;   // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += v;
    }
    warp_tot[lane] = x;   // inclusive over warps
  }
  __syncthreads();
  int run = incl - sum + (w > 0 ? warp_tot[w - 1] : 0);
  for (int i = lo; i < hi; ++i) {
    const int c = bins.count[i];
    bins.start[i] = run;
    bins.cursor[i] = run;
    bins.count[i] = 0;
    run += c;
  }
  if (t == 1023) bins.start[n] = warp_tot[31];
}

__global__ void __launch_bounds__(1024) k_bin_scan(RowBins bins) { bin_scan_block(bins); }

template <typename R>
__device__ __forceinline__ void bin_fill_one(const BlobParams& p, const double* __restrict__ q, const RowBins& bins,
                                             long long b) {
  const double qb[3] = {q[3 * b], q[3 * b + 1], q[3 * b + 2]};
  const BlobSpan sp = make_stencil<R>(nullptr, qb, p);
  for_each_row_block(sp, p, [&](int blk) {
    const int pos = atomicAdd(&bins.cursor[blk], 1);
    if (pos < bins.capacity) bins.list[pos] = (int)b;
  });
}

template <typename R>
__global__ void k_bin_fill(BlobParams p, long long nb, const double* __restrict__ q, RowBins bins) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  bin_fill_one<R>(p, q, bins, b);
}

// Step 4 from the gathered J v~ (element i = 3 b + a): slip correction, momentum
// change, its weighted copy.
__device__ __forceinline__ void dp_from_one(const BlobParams& p, const BlobState& s, const double* __restrict__ jvt,
                                            long long i) {
  const long long b = i / 3;
  const double me = s.me[b];
  const double visc = 0.5 * (p.eta / p.rho) * p.dt;
  const double coef = p.mtf / (p.rho * (p.mtf + me));
  const double jv = jvt[i];
  double du = p.slip == 1 ? 0.0 : visc * s.g[i];
  if (p.slip == 2) du += s.w1[i] - s.w0[i];
  const double dp = me * (s.u[i] - jv - du);
  s.jvt[i] = jv;
  s.du[i] = du;
  s.dp[i] = dp;
  s.cdp[i] = coef * dp;
}

__global__ void k_dp_from(BlobParams p, BlobState s, const double* __restrict__ jvt) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < 3 * s.nb) dp_from_one(p, s, jvt, i);
}

// Steps 6-8 from the gathered J dv~ (element i): the source of the viscous correction
// (returned) and u^{n+1}.
__device__ __forceinline__ double inertial_from_one(const BlobState& s, const double* __restrict__ jdvt, long long i) {
  const long long b = i / 3;
  const double jd = jdvt[i];
  const double sr = s.dp[i] - s.me[b] * jd;
  s.src[i] = sr;
  s.u[i] = s.jvt[i] + jd + s.du[i];
  return sr;
}

// Steps 6-8 from the gathered J dv~, with the grid sum of the source for the momentum
// bookkeeping.
__global__ void __launch_bounds__(256) k_inertial_from(BlobParams p, BlobState s, const double* __restrict__ jdvt) {
  __shared__ double red[3][256];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int a = (int)(i % 3);
  double sr = 0.0;
  if (i < 3 * s.nb) sr = inertial_from_one(s, jdvt, i);
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = c == a ? sr : 0.0;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) atomicAdd(&s.scal[SC_SUMSRC + threadIdx.x], red[threadIdx.x][0]);
}

// Step 9 from the gathered J v^{n+1} (= base + add) and J L dv (element i): positions,
// velocities, the lagged slip term, checks.
__device__ __forceinline__ void finish_from_one(const BlobParams& p, const BlobState& s,
                                                const double* __restrict__ base, const double* __restrict__ add,
                                                const double* __restrict__ g, int inertial, long long i) {
  const int a = (int)(i % 3);
  const double jv = base ? base[i] + add[i] : add[i];
  const double u = inertial ? s.u[i] : jv;
  const double qn = wrap_pos(fma(0.5 * p.dt, jv + s.w1[i], s.q[i]), p.box[a], p.inv_box[a]);
  s.q[i] = qn;
  s.u[i] = u;
  s.g[i] = inertial ? g[i] * (p.inv_h * p.inv_h) : 0.0;
  if (!isfinite(qn) || !isfinite(u)) atomicOr(s.err, DEV_ERR_NONFINITE);
  if (fabs(u) * p.dt > p.h) atomicOr(s.err, DEV_ERR_CFL);
}

// With step_dev set, block 0 also closes the step's FP64 bookkeeping (the momentum
// target P^{n+1} = K0 + the viscous correction's source sum, the time level and the
// history flag), which reads nothing this kernel writes.
__global__ void k_finish_from(BlobParams p, BlobState s, const double* __restrict__ base,
                              const double* __restrict__ add, const double* __restrict__ g, int inertial,
                              long long* __restrict__ step_dev, int* __restrict__ hist_dev) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < 3 * s.nb) finish_from_one(p, s, base, add, g, inertial, i);
  if (step_dev != nullptr && blockIdx.x == 0) {
    const int a = threadIdx.x;
    if (a < 3) s.scal[SC_PBAR + a] = s.scal[SC_K0 + a] + (inertial ? s.scal[SC_SUMSRC + a] : 0.0);
    if (a == 0) {
      *step_dev += 1;
      *hist_dev = 1;
    }
  }
}

// The same over every member of a batch: one thread per blob (bins) or per blob
// component (the elementwise steps); the member's accumulators are its bins.acc.
template <typename R>
__global__ void k_bbin_count(const BlobMember* __restrict__ mem, const int* __restrict__ member_of, long long nbt) {
  const long long gb = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gb >= nbt) return;
  const BlobMember& m = mem[member_of[gb]];
  bin_count_one<R>(m.p, m.s.nb, m.s.qh, m.bins, gb - m.b0);
}
__global__ void __launch_bounds__(1024) k_bbin_scan(const BlobMember* __restrict__ mem) {
  bin_scan_block(mem[blockIdx.x].bins);
}
template <typename R>
__global__ void k_bbin_fill(const BlobMember* __restrict__ mem, const int* __restrict__ member_of, long long nbt) {
  const long long gb = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gb >= nbt) return;
  const BlobMember& m = mem[member_of[gb]];
  bin_fill_one<R>(m.p, m.s.qh, m.bins, gb - m.b0);
}
__global__ void k_bdp_from(const BlobMember* __restrict__ mem, const int* __restrict__ member_of, long long nbt) {
  const long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gi >= 3 * nbt) return;
  const BlobMember& m = mem[member_of[gi / 3]];
  dp_from_one(m.p, m.s, m.bins.acc, gi - 3 * m.b0);
}
__global__ void k_binertial_from(const BlobMember* __restrict__ mem, const int* __restrict__ member_of,
                                 long long nbt) {
  const long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gi >= 3 * nbt) return;
  const BlobMember& m = mem[member_of[gi / 3]];
  const long long i = gi - 3 * m.b0;
  const double sr = inertial_from_one(m.s, m.bins.acc + 3 * m.s.nb, i);
  atomicAdd(&m.s.scal[SC_SUMSRC + (int)(i % 3)], sr);
}
__global__ void k_bfinish_from(const BlobMember* __restrict__ mem, const int* __restrict__ member_of,
                               long long nbt) {
  const long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gi >= 3 * nbt) return;
  const BlobMember& m = mem[member_of[gi / 3]];
  const long long i = gi - 3 * m.b0, nb = m.s.nb;
  const double* acc = m.bins.acc;   // J v~, J dv~, J dv, J L dv
  if (m.inertial)
    finish_from_one(m.p, m.s, m.s.jvt, acc + 6 * nb, acc + 9 * nb, 1, i);
  else
    finish_from_one(m.p, m.s, nullptr, acc, nullptr, 0, i);
}

inline unsigned eblocks(long long n) { return (unsigned)((n + 255) / 256); }

// ---------------------------------------------------------------------------
// WCA pair forces (Sec. IV.A, Eq. WCA) through a cell list at q^{n+1/2}
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wca_cell_axis(double x, double cell_inv, int n) {
  const int c = (int)(x * cell_inv);
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

__global__ void k_wca_count(BlobState s, WcaParams w) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= s.nb) return;
  int c[3];
  for (int a = 0; a < 3; ++a) c[a] = wca_cell_axis(s.qh[3 * b + a], w.cell_inv[a], w.nc[a]);
  atomicAdd(&w.count[c[0] + w.nc[0] * (c[1] + w.nc[1] * c[2])], 1);
}

__global__ void k_wca_fill(BlobState s, WcaParams w) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= s.nb) return;
  int c[3];
  for (int a = 0; a < 3; ++a) c[a] = wca_cell_axis(s.qh[3 * b + a], w.cell_inv[a], w.nc[a]);
  const int pos = atomicAdd(&w.cursor[c[0] + w.nc[0] * (c[1] + w.nc[1] * c[2])], 1);
  if (pos < s.nb) w.list[pos] = (int)b;
}

// F_i = sum_j 24 eps (2 s^12/r^14 - s^6/r^8) d_ij over the pairs within the cut-off,
// d_ij = q_i - q_j to the nearest image (FP64).
__global__ void __launch_bounds__(256) k_wca_force(BlobParams p, BlobState s, WcaParams w, int with_trap) {
  __shared__ double red[3][256];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double f[3] = {0.0, 0.0, 0.0};
  if (i < s.nb) {
    const double qi[3] = {s.qh[3 * i], s.qh[3 * i + 1], s.qh[3 * i + 2]};
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = wca_cell_axis(qi[a], w.cell_inv[a], w.nc[a]);
    const double s2 = w.sigma * w.sigma;
    for (int dz = w.lo[2]; dz <= w.hi[2]; ++dz)
      for (int dy = w.lo[1]; dy <= w.hi[1]; ++dy)
        for (int dx = w.lo[0]; dx <= w.hi[0]; ++dx) {
          const int cx = (c[0] + dx + w.nc[0]) % w.nc[0], cy = (c[1] + dy + w.nc[1]) % w.nc[1];
          const int cz = (c[2] + dz + w.nc[2]) % w.nc[2];
          const int cell = cx + w.nc[0] * (cy + w.nc[1] * cz);
          const int e = w.start[cell + 1];
          for (int k = w.start[cell]; k < e; ++k) {
            const int j = w.list[k];
            if (j == i) continue;
            double d[3], r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
              const double x = qi[a] - s.qh[3 * j + a];
              d[a] = fma(-p.box[a], rint(x * p.inv_box[a]), x);
              r2 = fma(d[a], d[a], r2);
            }
            if (r2 >= w.rc2) continue;
            const double s6 = (s2 / r2) * (s2 / r2) * (s2 / r2);
            const double mag = 24.0 * w.eps * (2.0 * s6 * s6 - s6) / r2;
            for (int a = 0; a < 3; ++a) f[a] = fma(mag, d[a], f[a]);
          }
        }
    for (int a = 0; a < 3; ++a) s.fe[3 * i + a] = (with_trap ? s.fe[3 * i + a] : s.f[3 * i + a]) + f[a];
  }
  for (int a = 0; a < 3; ++a) red[a][threadIdx.x] = f[a];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int a = 0; a < 3; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) atomicAdd(&s.scal[SC_K0 + threadIdx.x], p.dt * red[threadIdx.x][0]);
}

}  // namespace

template <typename R>
void build_row_bins(const BlobParams& p, long long nb, const double* q, RowBins bins, cudaStream_t st) {
  if (nb <= 0) return;
  k_bin_count<R><<<eblocks(nb), 256, 0, st>>>(p, nb, q, bins);
  k_bin_scan<<<1, 1024, 0, st>>>(bins);
  k_bin_fill<R><<<eblocks(nb), 256, 0, st>>>(p, nb, q, bins);
}
template void build_row_bins<float>(const BlobParams&, long long, const double*, RowBins, cudaStream_t);
template void build_row_bins<double>(const BlobParams&, long long, const double*, RowBins, cudaStream_t);

void blob_wca_forces(const BlobParams& p, BlobState s, const WcaParams& w, bool with_trap, cudaStream_t st) {
  if (s.nb <= 0) return;
  k_wca_count<<<eblocks(s.nb), 256, 0, st>>>(s, w);
  RowBins cells;
  cells.count = w.count;
  cells.start = w.start;
  cells.cursor = w.cursor;
  cells.list = w.list;
  cells.geo = nullptr;
  cells.acc = nullptr;
  cells.nacc = 0;
  cells.nblocks = w.ncells;
  cells.capacity = s.nb;
  k_bin_scan<<<1, 1024, 0, st>>>(cells);
  k_wca_fill<<<eblocks(s.nb), 256, 0, st>>>(s, w);
  k_wca_force<<<eblocks(s.nb), 256, 0, st>>>(p, s, w, with_trap ? 1 : 0);
}

void blob_dp_from(const BlobParams& p, BlobState s, const double* jvt, cudaStream_t st) {
  if (s.nb > 0) k_dp_from<<<eblocks(3 * s.nb), 256, 0, st>>>(p, s, jvt);
}
void blob_inertial_from(const BlobParams& p, BlobState s, const double* jdvt, cudaStream_t st) {
  if (s.nb > 0) k_inertial_from<<<eblocks(3 * s.nb), 256, 0, st>>>(p, s, jdvt);
}
void blob_finish_from(const BlobParams& p, BlobState s, const double* base, const double* add, const double* g,
                      bool inertial, cudaStream_t st, long long* step_dev, int* hist_dev) {
  if (s.nb > 0)
    k_finish_from<<<eblocks(3 * s.nb), 256, 0, st>>>(p, s, base, add, g, inertial ? 1 : 0, step_dev, hist_dev);
}

#define ICM_KSWITCH(call3, call4) \
  if (p.kernel == 3) {            \
    call3;                        \
  } else {                        \
    call4;                        \
  }

template <typename R>
void batch_predict(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st) {
  if (nbt > 0) k_bpredict<R><<<nblocks(nbt), 32 * kWarps, 0, st>>>(m, member_of, nbt);
}
template <typename R>
void batch_spread(const BlobMember* m, const int* member_of, long long nbt, int which, cudaStream_t st) {
  if (nbt > 0) k_bspread<R><<<nblocks(nbt), 32 * kWarps, 0, st>>>(m, member_of, nbt, which);
}
template <typename R>
void batch_dp(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st) {
  if (nbt > 0) k_bdp<R><<<nblocks(nbt), 32 * kWarps, 0, st>>>(m, member_of, nbt);
}
template <typename R>
void batch_inertial(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st) {
  if (nbt > 0) k_binertial<R><<<nblocks(nbt), 32 * kWarps, 0, st>>>(m, member_of, nbt);
}
template <typename R>
void batch_finish(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st) {
  if (nbt > 0) k_bfinish<R><<<nblocks(nbt), 32 * kWarps, 0, st>>>(m, member_of, nbt);
}
void batch_zero_work(const BlobMember* m, const long long* prefix16, int nm, long long total16, cudaStream_t st) {
  if (nm <= 0 || total16 <= 0) return;
  const unsigned g = (unsigned)std::min<long long>((total16 + 255) / 256, 4096);
  k_bzero<<<g, 256, 0, st>>>(m, prefix16, nm, total16);
}
template <typename R>
void batch_bins(const BlobMember* m, const int* member_of, long long nbt, int nm, cudaStream_t st) {
  if (nbt <= 0 || nm <= 0) return;
  k_bbin_count<R><<<eblocks(nbt), 256, 0, st>>>(m, member_of, nbt);
  k_bbin_scan<<<nm, 1024, 0, st>>>(m);
  k_bbin_fill<R><<<eblocks(nbt), 256, 0, st>>>(m, member_of, nbt);
}
void batch_dp_from(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st) {
  if (nbt > 0) k_bdp_from<<<eblocks(3 * nbt), 256, 0, st>>>(m, member_of, nbt);
}
void batch_inertial_from(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st) {
  if (nbt > 0) k_binertial_from<<<eblocks(3 * nbt), 256, 0, st>>>(m, member_of, nbt);
}
void batch_finish_from(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st) {
  if (nbt > 0) k_bfinish_from<<<eblocks(3 * nbt), 256, 0, st>>>(m, member_of, nbt);
}
void batch_scalars_before(const BlobMember* m, int nm, cudaStream_t st) {
  if (nm > 0) k_bscal_before<<<nm, 32, 0, st>>>(m);
}
void batch_scalars_after(const BlobMember* m, int nm, cudaStream_t st) {
  if (nm > 0) k_bscal_after<<<nm, 32, 0, st>>>(m);
}
#define ICM_BINST(R)                                                                                       \
  template void batch_predict<R>(const BlobMember*, const int*, long long, cudaStream_t);                \
  template void batch_spread<R>(const BlobMember*, const int*, long long, int, cudaStream_t);            \
  template void batch_dp<R>(const BlobMember*, const int*, long long, cudaStream_t);                     \
  template void batch_inertial<R>(const BlobMember*, const int*, long long, cudaStream_t);               \
  template void batch_finish<R>(const BlobMember*, const int*, long long, cudaStream_t);                 \
  template void batch_bins<R>(const BlobMember*, const int*, long long, int, cudaStream_t);
ICM_BINST(float)
ICM_BINST(double)
#undef ICM_BINST

template <typename R>
void blob_predict(const BlobParams& p, BlobState s, const R* v, cudaStream_t st) {
  if (s.nb <= 0) return;
  ICM_KSWITCH((k_predict<R, 3><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, v)),
              (k_predict<R, 4><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, v)))
}
template <typename R>
void blob_spread(const BlobParams& p, long long nb, const double* q, const double* vec, R* field, cudaStream_t st) {
  if (nb <= 0) return;
  ICM_KSWITCH((k_spread<R, 3><<<nblocks(nb), 32 * kWarps, 0, st>>>(p, nb, q, vec, field)),
              (k_spread<R, 4><<<nblocks(nb), 32 * kWarps, 0, st>>>(p, nb, q, vec, field)))
}
namespace {
// Block tree sum of three per-thread values into red[3][256]; the result is in red[.][0].
__device__ __forceinline__ void block_sum3(double (&red)[3][256], const double v[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) red[a][threadIdx.x] = v[a];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int a = 0; a < 3; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + h];
    __syncthreads();
  }
}

// Per-block compensated sums of w_i x[3 i + a] -> partial[a * gridDim.x + block].
__global__ void __launch_bounds__(256) k_rows_partial(const double* __restrict__ x, const double* __restrict__ w,
                                                      long long n, double* __restrict__ partial) {
  __shared__ double red[3][256];
  double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double wi = w ? w[i] : 1.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double y = wi * x[3 * i + a] - c[a];
      const double t = s[a] + y;
      c[a] = (t - s[a]) - y;
      s[a] = t;
    }
  }
  block_sum3(red, s);
  if (threadIdx.x < 3) partial[threadIdx.x * gridDim.x + blockIdx.x] = red[threadIdx.x][0];
}

// out[a] = init[a] + compensated sum of the np partials of component a.
__global__ void __launch_bounds__(256) k_rows_final(const double* __restrict__ partial, int np,
                                                    const double* __restrict__ init, double* __restrict__ out) {
  __shared__ double red[3][256];
  double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < np; i += blockDim.x)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double y = partial[a * np + i] - c[a];
      const double t = s[a] + y;
      c[a] = (t - s[a]) - y;
      s[a] = t;
    }
  block_sum3(red, s);
  if (threadIdx.x < 3) out[threadIdx.x] = (init ? init[threadIdx.x] : 0.0) + red[threadIdx.x][0];
}
}  // namespace

namespace {
// The blob state a queued read returns, gathered into one contiguous device block:
// positions [3 nb], velocities [3 nb], then momentum [3], the time level and the error
// bits (their bit patterns in two doubles).
__global__ void k_snapshot(const double* __restrict__ q, const double* __restrict__ u, long long nb,
                           const double* __restrict__ ptot, const long long* __restrict__ step,
                           const int* __restrict__ err, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n3 = 3 * nb;
  if (i < n3) {
    out[i] = q[i];
    out[n3 + i] = u[i];
  }
  if (i == 0) {
    for (int a = 0; a < 3; ++a) out[2 * n3 + a] = ptot[a];
    out[2 * n3 + 3] = __longlong_as_double(*step);
    out[2 * n3 + 4] = __longlong_as_double((long long)*err);
  }
}
}  // namespace

void blob_snapshot(const double* q, const double* u, long long nb, const double* ptot, const long long* step,
                   const int* err, double* out, cudaStream_t st) {
  const long long n = nb > 0 ? 3 * nb : 1;
  k_snapshot<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(q, u, nb, ptot, step, err, out);
}

void rows_sum3(const double* x, const double* w, long long n, const double* init, double* out, double* partial,
               int npartial, cudaStream_t st) {
  long long g = (n + 255) / 256;
  if (g > npartial) g = npartial;
  if (g < 1) g = 1;
  k_rows_partial<<<(unsigned)g, 256, 0, st>>>(x, w, n, partial);
  k_rows_final<<<1, 256, 0, st>>>(partial, (int)g, init, out);
}

template <typename R>
void blob_momentum_change(const BlobParams& p, BlobState s, const R* vt, cudaStream_t st) {
  if (s.nb <= 0) return;
  ICM_KSWITCH((k_dp<R, 3><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, vt)),
              (k_dp<R, 4><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, vt)))
}
template <typename R>
void blob_inertial(const BlobParams& p, BlobState s, const R* dvt, cudaStream_t st) {
  if (s.nb <= 0) return;
  ICM_KSWITCH((k_inertial<R, 3><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, dvt)),
              (k_inertial<R, 4><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, dvt)))
}
template <typename R>
void blob_finish(const BlobParams& p, BlobState s, const R* v_new, const R* dv, bool inertial, cudaStream_t st) {
  if (s.nb <= 0) return;
  ICM_KSWITCH((k_finish<R, 3><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, v_new, dv, inertial ? 1 : 0)),
              (k_finish<R, 4><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, v_new, dv, inertial ? 1 : 0)))
}
template <typename R>
void blob_interp(const BlobParams& p, long long nb, const double* q, const R* field, bool laplacian, double* out,
                 cudaStream_t st) {
  if (nb <= 0) return;
  ICM_KSWITCH((k_interp<R, 3><<<nblocks(nb), 32 * kWarps, 0, st>>>(p, nb, q, field, laplacian ? 1 : 0, out)),
              (k_interp<R, 4><<<nblocks(nb), 32 * kWarps, 0, st>>>(p, nb, q, field, laplacian ? 1 : 0, out)))
}

template <typename R>
void blob_spread_drift(const BlobParams& p, BlobState s, R* field, cudaStream_t st) {
  if (s.nb <= 0) return;
  if (p.kernel == 3)
    k_spread_drift<R, 3><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, field);
  else
    k_spread_drift<R, 4><<<nblocks(s.nb), 32 * kWarps, 0, st>>>(p, s, field);
}

#define ICM_INST(R)                                                                                            \
  template void blob_predict<R>(const BlobParams&, BlobState, const R*, cudaStream_t);                        \
  template void blob_spread<R>(const BlobParams&, long long, const double*, const double*, R*, cudaStream_t); \
  template void blob_momentum_change<R>(const BlobParams&, BlobState, const R*, cudaStream_t);                \
  template void blob_inertial<R>(const BlobParams&, BlobState, const R*, cudaStream_t);                       \
  template void blob_finish<R>(const BlobParams&, BlobState, const R*, const R*, bool, cudaStream_t);          \
  template void blob_interp<R>(const BlobParams&, long long, const double*, const R*, bool, double*, cudaStream_t); \
  template void blob_spread_drift<R>(const BlobParams&, BlobState, R*, cudaStream_t);
ICM_INST(float)
ICM_INST(double)
#undef ICM_INST

}  // namespace icm
