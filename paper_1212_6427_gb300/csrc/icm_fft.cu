// 3D real-to-complex FFT Helmholtz solve and discrete projection on the MAC grid
// (arXiv:1212.6427, Sec. III.D and Appendix C: the periodic velocity and pressure
// systems are diagonalised by Fourier transforms).
//
// Layout.  A real face field is 3 components x [Nz][Ny][Nx] (x fastest).  The
// spectrum is 3 x [Nz][Ny][kxp] complex with kx = Nx/2+1 stored x wavenumbers.
//
// Passes (each one read + one write of the spectrum, tiles staged in shared
// memory, every global access a contiguous 128-byte row segment):
//   x forward : two real rows packed as one complex row, Nx-point FFT, split into
//               two half spectra (Hermitian symmetry).
//   y forward : in-place decimation-in-frequency stages; leaves ky in digit-reversed
//               storage order (the symbol tables are indexed by storage position).
//   z         : forward DIF, symbol P^/(a + b|d|^2) on all three components at once,
//               inverse DIT back to natural z order.
//   y inverse : DIT, digit-reversed -> natural order.
//   x inverse : Hermitian extension, Nx-point inverse FFT, two real rows out.
// Each stage of a pass is a radix-2/3/4/8/16 butterfly done in registers with the
// operands read from and written back to the same shared-memory positions.
#include <algorithm>
#include <cstdio>

#include <cooperative_groups.h>
#include <cuda.h>

#include "icm.h"
#include "icm_internal.h"
#include "icm_fft_reg.cuh"
#include "icm_rows.cuh"

// Each shard uses only part of the helpers below.
#pragma nv_diag_suppress 177

namespace icm {
namespace {

// ---------------------------------------------------------------------------
// Small DFTs in registers (forward, W = exp(-2 pi i / R)).
// ---------------------------------------------------------------------------
template <typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  const C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, cmul_mi(d13));
  a3 = cadd(d02, cmul_pi(d13));
}

// multiply by exp(-2 pi i m / 16); m is a compile-time constant after unrolling
template <typename R> __device__ __forceinline__ cplx_t<R> w16mul(cplx_t<R> a, int m) {
  const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173), r2 = R(0.70710678118654752440);
  R c, s;  // exp(-i t) = c - i s
  switch (m & 15) {
    case 0: return a;
    case 1: c = c1; s = s1; break;
    case 2: c = r2; s = r2; break;
    case 3: c = s1; s = c1; break;
    case 4: return cmul_mi(a);
    case 5: c = -s1; s = c1; break;
    case 6: c = -r2; s = r2; break;
    case 7: c = -c1; s = s1; break;
    case 8: return mk(-a.x, -a.y);
    case 9: c = -c1; s = -s1; break;
    case 10: c = -r2; s = -r2; break;
    case 11: c = -s1; s = -c1; break;
    case 12: return cmul_pi(a);
    case 13: c = s1; s = -c1; break;
    case 14: c = r2; s = -r2; break;
    default: c = c1; s = -s1; break;
  }
  return mk(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <typename R, int RAD> struct Dft;
template <typename R> struct Dft<R, 2> {
  __device__ __forceinline__ static void run(cplx_t<R>* a) {
    const cplx_t<R> t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};
template <typename R> struct Dft<R, 3> {
  __device__ __forceinline__ static void run(cplx_t<R>* a) {
    const R s = R(0.86602540378443864676);
    const cplx_t<R> t1 = cadd(a[1], a[2]);
    const cplx_t<R> t2 = mk(a[0].x - R(0.5) * t1.x, a[0].y - R(0.5) * t1.y);
    const cplx_t<R> d = csub(a[1], a[2]);
    const cplx_t<R> t3 = mk(s * d.x, s * d.y);
    a[0] = cadd(a[0], t1);
    a[1] = cadd(t2, cmul_mi(t3));
    a[2] = cadd(t2, cmul_pi(t3));
  }
};
template <typename R> struct Dft<R, 4> {
  __device__ __forceinline__ static void run(cplx_t<R>* a) { dft4(a[0], a[1], a[2], a[3]); }
};
template <typename R> struct Dft<R, 8> {
  // 8 = 2 x 4: b_k2[n1] = W8^(n1 k2) sum_n2 x[n1 + 4 n2] W2^(n2 k2); X[2 k1 + k2] = DFT4(b_k2)[k1]
  __device__ __forceinline__ static void run(cplx_t<R>* a) {
    cplx_t<R> b0[4], b1[4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      b0[n1] = cadd(a[n1], a[n1 + 4]);
      b1[n1] = w16mul<R>(csub(a[n1], a[n1 + 4]), 2 * n1);
    }
    dft4(b0[0], b0[1], b0[2], b0[3]);
    dft4(b1[0], b1[1], b1[2], b1[3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      a[2 * k1] = b0[k1];
      a[2 * k1 + 1] = b1[k1];
    }
  }
};
template <typename R> struct Dft<R, 16> {
  // 16 = 4 x 4: t[n1][k2] = W16^(n1 k2) DFT4_n2(x[n1 + 4 n2])[k2]; X[4 k1 + k2] = DFT4_n1(t[.][k2])[k1]
  __device__ __forceinline__ static void run(cplx_t<R>* a) {
    cplx_t<R> t[16];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      cplx_t<R> y0 = a[n1], y1 = a[n1 + 4], y2 = a[n1 + 8], y3 = a[n1 + 12];
      dft4(y0, y1, y2, y3);
      t[n1 * 4 + 0] = y0;
      t[n1 * 4 + 1] = w16mul<R>(y1, n1);
      t[n1 * 4 + 2] = w16mul<R>(y2, 2 * n1);
      t[n1 * 4 + 3] = w16mul<R>(y3, 3 * n1);
    }
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      cplx_t<R> z0 = t[k2], z1 = t[4 + k2], z2 = t[8 + k2], z3 = t[12 + k2];
      dft4(z0, z1, z2, z3);
      a[k2] = z0;
      a[4 + k2] = z1;
      a[8 + k2] = z2;
      a[12 + k2] = z3;
    }
  }
};

// One in-place stage over ncomp groups of NL interleaved lines: element (pos, line)
// of group c is s[c*cs + pos*LS + line].  Sub-transform length M, radix RAD.
// Forward (DIF): y[n1 + (M/R) k2] = W_M^(n1 k2) sum_n2 x[n1 + (M/R) n2] W_R^(n2 k2).
// Inverse: the exact (unnormalised) inverse of that map, via conj o DFT o conj.
template <typename R, int RAD, bool INV, int NL>
__device__ __forceinline__ void fft_stage(cplx_t<R>* s, int N, int M, int LS, int ncomp, int cs,
                                          const cplx_t<R>* tw, int tid, int nthr) {
  using C = cplx_t<R>;
  const int Mr = M / RAD;
  const int nbf = N / RAD;
  const int tws = N / M;
  const int total = nbf * NL * ncomp;
  const int str = Mr * LS;
  for (int it = tid; it < total; it += nthr) {
    const int line = it % NL;
    const int rest = it / NL;
    const int comp = rest / nbf;
    const int bf = rest - comp * nbf;
    const int blk = bf / Mr;
    const int n1 = bf - blk * Mr;
    C* p = s + comp * cs + (blk * M + n1) * LS + line;
    C a[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) a[r] = p[r * str];
    if (INV) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        a[r] = cconj(a[r]);
        if (r > 0) a[r] = cmul(a[r], tw[n1 * r * tws]);
      }
      Dft<R, RAD>::run(a);
#pragma unroll
      for (int r = 0; r < RAD; ++r) a[r] = cconj(a[r]);
    } else {
      Dft<R, RAD>::run(a);
#pragma unroll
      for (int r = 1; r < RAD; ++r) a[r] = cmul(a[r], tw[n1 * r * tws]);
    }
#pragma unroll
    for (int r = 0; r < RAD; ++r) p[r * str] = a[r];
  }
}

template <typename R, bool INV, int NL>
__device__ void run_fft(cplx_t<R>* s, const AxisPlan& P, int LS, int ncomp, int cs, const cplx_t<R>* tw,
                        int tid, int nthr) {
  int Ms[kMaxStages];
  int M = P.n;
  for (int k = 0; k < P.nstages; ++k) {
    Ms[k] = M;
    M /= P.radix[k];
  }
  for (int k = 0; k < P.nstages; ++k) {
    const int si = INV ? P.nstages - 1 - k : k;
    const int m = Ms[si];
    switch (P.radix[si]) {
      case 2: fft_stage<R, 2, INV, NL>(s, P.n, m, LS, ncomp, cs, tw, tid, nthr); break;
      case 3: fft_stage<R, 3, INV, NL>(s, P.n, m, LS, ncomp, cs, tw, tid, nthr); break;
      case 4: fft_stage<R, 4, INV, NL>(s, P.n, m, LS, ncomp, cs, tw, tid, nthr); break;
      case 8: fft_stage<R, 8, INV, NL>(s, P.n, m, LS, ncomp, cs, tw, tid, nthr); break;
      default: fft_stage<R, 16, INV, NL>(s, P.n, m, LS, ncomp, cs, tw, tid, nthr); break;
    }
    __syncthreads();
  }
}

constexpr int kThreads = 256;
constexpr int kXLines = 16;   // complex lines (= 32 real rows) per x-pass block
constexpr int kXLS = 17;      // padded line stride of the x pass (transposing loads)

template <typename R> constexpr int seg_lines() { return 128 / (int)sizeof(cplx_t<R>); }

template <typename R>
__device__ __forceinline__ void load_tables(cplx_t<R>* tw, int* pof, const AxisPlan& P, int tid) {
  const cplx_t<R>* g = (const cplx_t<R>*)P.tw;
  for (int i = tid; i < P.n; i += kThreads) {
    tw[i] = g[i];
    if (pof) pof[i] = P.pos_of_freq[i];
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_xfwd(const R* __restrict__ src, cplx_t<R>* __restrict__ spec,
                                                   AxisPlan P, int nrows, long long ncell, int kx, int kxp) {
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = P.n;
  C* lines = reinterpret_cast<C*>(smem_raw);
  C* tw = lines + N * kXLS;
  int* pof = reinterpret_cast<int*>(tw + N);
  const int tid = threadIdx.x;
  load_tables<R>(tw, pof, P, tid);
  const int comp = blockIdx.y % 3;
  const long long row0 = (long long)blockIdx.x * (2 * kXLines);
  const R* s = src + comp * ncell;
  for (int idx = tid; idx < 2 * kXLines * N; idx += kThreads) {
    const int rr = idx / N, x = idx - rr * N;
    const long long row = row0 + rr;
    const R val = row < nrows ? s[row * N + x] : R(0);
    reinterpret_cast<R*>(&lines[x * kXLS + (rr >> 1)])[rr & 1] = val;
  }
  __syncthreads();
  run_fft<R, false, kXLines>(lines, P, kXLS, 1, 0, tw, tid, kThreads);
  C* out = spec + (size_t)comp * nrows * kxp;
  for (int idx = tid; idx < kXLines * kx; idx += kThreads) {
    const int l = idx / kx, k = idx - l * kx;
    const C zk = lines[pof[k] * kXLS + l];
    const C zm = lines[pof[k == 0 ? 0 : N - k] * kXLS + l];
    const C x1 = mk((zk.x + zm.x) * R(0.5), (zk.y - zm.y) * R(0.5));
    const C x2 = cmul_mi(mk((zk.x - zm.x) * R(0.5), (zk.y + zm.y) * R(0.5)));
    const long long r1 = row0 + 2 * l;
    if (r1 < nrows) out[r1 * kxp + k] = x1;
    if (r1 + 1 < nrows) out[(r1 + 1) * kxp + k] = x2;
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_xinv(const cplx_t<R>* __restrict__ spec, R* __restrict__ dst,
                                                   R* __restrict__ dst2, int mode, AxisPlan P, int nrows,
                                                   long long ncell, int kxp) {
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = P.n;
  C* lines = reinterpret_cast<C*>(smem_raw);
  C* tw = lines + N * kXLS;
  int* pof = reinterpret_cast<int*>(tw + N);
  const int tid = threadIdx.x;
  load_tables<R>(tw, pof, P, tid);
  __syncthreads();
  const int comp = blockIdx.y % 3;
  const long long row0 = (long long)blockIdx.x * (2 * kXLines);
  const C* in = spec + (size_t)comp * nrows * kxp;
  const C zero = mk(R(0), R(0));
  for (int idx = tid; idx < kXLines * N; idx += kThreads) {
    const int l = idx / N, k = idx - l * N;
    const long long r1 = row0 + 2 * l;
    const bool direct = 2 * k <= N;
    const int kk = direct ? k : N - k;
    C a = r1 < nrows ? in[r1 * kxp + kk] : zero;
    C b = r1 + 1 < nrows ? in[(r1 + 1) * kxp + kk] : zero;
    if (!direct) {
      a = cconj(a);
      b = cconj(b);
    }
    if (k == 0 || 2 * k == N) {  // real by Hermitian symmetry: drop round-off imaginary parts
      a.y = R(0);
      b.y = R(0);
    }
    lines[pof[k] * kXLS + l] = mk(a.x - b.y, a.y + b.x);
  }
  __syncthreads();
  run_fft<R, true, kXLines>(lines, P, kXLS, 1, 0, tw, tid, kThreads);
  const size_t base = (size_t)comp * ncell;
  for (int idx = tid; idx < 2 * kXLines * N; idx += kThreads) {
    const int rr = idx / N, x = idx - rr * N;
    const long long row = row0 + rr;
    if (row >= nrows) continue;
    const R val = reinterpret_cast<const R*>(&lines[x * kXLS + (rr >> 1)])[rr & 1];
    const size_t o = base + (size_t)row * N + x;
    if (mode == OUT_STORE) {
      dst[o] = val;
    } else {
      dst[o] += val;
      dst2[o] = val;
    }
  }
}

template <typename R, bool INV>
__global__ void __launch_bounds__(kThreads) k_ypass(cplx_t<R>* __restrict__ spec, AxisPlan P, int nz, int kx,
                                                    int kxp) {
  using C = cplx_t<R>;
  constexpr int NL = seg_lines<R>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = P.n;
  C* lines = reinterpret_cast<C*>(smem_raw);
  C* tw = lines + N * NL;
  const int tid = threadIdx.x;
  load_tables<R>(tw, nullptr, P, tid);
  const int kx0 = blockIdx.x * NL;
  const int z = blockIdx.y, comp = blockIdx.z;
  C* base = spec + ((size_t)(comp * nz + z) * N) * kxp + kx0;
  const C zero = mk(R(0), R(0));
  for (int idx = tid; idx < N * NL; idx += kThreads) {
    const int t = idx % NL, y = idx / NL;
    lines[idx] = (kx0 + t < kx) ? base[(size_t)y * kxp + t] : zero;
  }
  __syncthreads();
  run_fft<R, INV, NL>(lines, P, NL, 1, 0, tw, tid, kThreads);
  for (int idx = tid; idx < N * NL; idx += kThreads) {
    const int t = idx % NL, y = idx / NL;
    if (kx0 + t < kx) base[(size_t)y * kxp + t] = lines[idx];
  }
}

template <typename R>
struct SymParams {
  R a, b, inv_ntot;
  R mean_scale;   // the symbol's scale on the mean mode: 1/(a ncell), 0 when a = 0
  const cplx_t<R>* dx; const R* ddx;
  const cplx_t<R>* dy; const R* ddy;
  const cplx_t<R>* dz; const R* ddz;
  const double* k0sum;
  double k0mul;   // k0scale / ncell
};

// P^ w / (a + b|d|^2) / ncell on one wave vector: (P^ w)_a = w_a - conj(d_a)(d . w)/|d|^2,
// identity on the mean mode, whose value is replaced by the FP64 bookkeeping if given
// (and which is zero when a = 0).
// 1/x: the hardware reciprocal in FP32 (within one ulp: a few roundings more than two
// divisions per wave vector, far inside the FP32 path's tolerance), exact division in FP64.
template <typename R> __device__ __forceinline__ R recip(R x);
template <> __device__ __forceinline__ float recip<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));   // within one ulp; x is never denormal here
  return r;
}
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }

template <typename R>
__device__ __forceinline__ void apply_symbol(cplx_t<R>& c0, cplx_t<R>& c1, cplx_t<R>& c2, cplx_t<R> d0,
                                             cplx_t<R> d1, cplx_t<R> d2, R dd, const SymParams<R>& sp,
                                             bool mean_mode) {
  // FP32: one reciprocal r = 1/(|d|^2 (a + b|d|^2)) serves both divisions; |d|^2 = 0
  // only on the mean mode, whose scale is precomputed.
  const R den = sp.a + sp.b * dd;
  const R prod = dd * den;
  const R r = sizeof(R) == 4 ? recip<R>(prod > R(0) ? prod : R(1)) : R(0);
  if (dd > R(0)) {
    const cplx_t<R> div = cadd(cadd(cmul(d0, c0), cmul(d1, c1)), cmul(d2, c2));
    const R inv_dd = sizeof(R) == 4 ? den * r : recip<R>(dd);
    const cplx_t<R> q = mk(div.x * inv_dd, div.y * inv_dd);
    c0 = csub(c0, cmul(cconj(d0), q));
    c1 = csub(c1, cmul(cconj(d1), q));
    c2 = csub(c2, cmul(cconj(d2), q));
  }
  // a = 0 (the steady Stokes solve): the mean mode has no solution and is dropped
  R scale;
  if (sizeof(R) == 4)
    scale = prod > R(0) ? sp.inv_ntot * (dd * r) : (dd > R(0) ? R(0) : sp.mean_scale);
  else
    scale = den > R(0) ? sp.inv_ntot * recip<R>(den) : R(0);
  c0 = cscale(c0, scale);
  c1 = cscale(c1, scale);
  c2 = cscale(c2, scale);
  if (mean_mode && sp.k0sum != nullptr) {
    c0 = mk((R)(sp.k0sum[0] * sp.k0mul), R(0));
    c1 = mk((R)(sp.k0sum[1] * sp.k0mul), R(0));
    c2 = mk((R)(sp.k0sum[2] * sp.k0mul), R(0));
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_zsym(cplx_t<R>* __restrict__ spec, AxisPlan P, int ny, int kx,
                                                   int kxp, SymParams<R> sp) {
  using C = cplx_t<R>;
  constexpr int NL = seg_lines<R>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = P.n;  // nz
  C* lines = reinterpret_cast<C*>(smem_raw);
  const int cs = N * NL;
  C* tw = lines + 3 * cs;
  const int tid = threadIdx.x;
  load_tables<R>(tw, nullptr, P, tid);
  const int kx0 = blockIdx.x * NL;
  const int py = blockIdx.y;
  const size_t zstride = (size_t)ny * kxp;
  const size_t cstride = (size_t)N * zstride;
  C* base = spec + (size_t)py * kxp + kx0;
  const C zero = mk(R(0), R(0));
  for (int idx = tid; idx < 3 * cs; idx += kThreads) {
    const int c = idx / cs, rem = idx - c * cs;
    const int t = rem % NL, z = rem / NL;
    lines[idx] = (kx0 + t < kx) ? base[c * cstride + z * zstride + t] : zero;
  }
  __syncthreads();
  run_fft<R, false, NL>(lines, P, NL, 3, cs, tw, tid, kThreads);
  const C dyv = sp.dy[py];
  const R ddy = sp.ddy[py];
  for (int idx = tid; idx < cs; idx += kThreads) {
    const int t = idx % NL, pz = idx / NL;
    const int k = kx0 + t;
    if (k >= kx) continue;
    const C d0 = sp.dx[k], d2 = sp.dz[pz];
    const R dd = sp.ddx[k] + ddy + sp.ddz[pz];
    C c0 = lines[idx], c1 = lines[cs + idx], c2 = lines[2 * cs + idx];
    apply_symbol<R>(c0, c1, c2, d0, dyv, d2, dd, sp, k == 0 && py == 0 && pz == 0);
    lines[idx] = c0;
    lines[cs + idx] = c1;
    lines[2 * cs + idx] = c2;
  }
  __syncthreads();
  run_fft<R, true, NL>(lines, P, NL, 3, cs, tw, tid, kThreads);
  for (int idx = tid; idx < 3 * cs; idx += kThreads) {
    const int c = idx / cs, rem = idx - c * cs;
    const int t = rem % NL, z = rem / NL;
    if (kx0 + t < kx) base[c * cstride + z * zstride + t] = lines[idx];
  }
}

// ---------------------------------------------------------------------------
// Two-stage register passes (sides listed in fft_split).
// ---------------------------------------------------------------------------
constexpr int kXPad = 16;   // x pass: one padding slot every 16 positions (bank spread)
__host__ __device__ constexpr int xrow(int n) { return n + n / kXPad; }
__device__ __forceinline__ int xaddr(int l, int p, int N) { return l * xrow(N) + p + p / kXPad; }
// x passes with blob work: the staged task records follow the rows and twiddles
template <typename R, int N> constexpr size_t stage_offset() {
  return ((size_t)kXLines * xrow(N) * sizeof(cplx_t<R>) + N * sizeof(cplx_t<R>) + 15) / 16 * 16;
}
// Blob task records staged per block (the rest are read in place).  The forward x
// pass stages 128, which keeps its FP32 blocks of sides up to 256 at four per SM
// (registers capped to match); the inverse pass, which holds its loads in flight in
// registers and would spill under that cap, stages one per thread.
constexpr int kStageF = 128;
template <typename R, int N, int S> size_t smem_x2b() { return stage_offset<R, N>() + S * sizeof(StagedTask<R>); }
template <typename R, int N> constexpr int xf2_min_blocks() { return sizeof(R) == 4 && N <= 256 ? 4 : 1; }
// Complex lines per block of the x passes without blob work: FP32 sides up to 128 take
// more than 16, so that the first stage (R2 items per line) fills the block's threads.
// With blob work a block is one 32-row bin (16 lines).
template <typename R, int N, int R2> constexpr int x_plain_lines() {
  return sizeof(R) != 4 || N > 128 ? kXLines : (kThreads / R2 >= 64 ? 64 : 32);
}
// The inverse x pass of FP32 sides up to 256 runs lean at four blocks per SM: its
// spectrum loads go in two batches, the old values of the adding modes are loaded
// just before the output, and 128 records are staged.  Otherwise (and for the
// two-output mode, which would spill) all loads are in flight at once and one record
// per thread is staged.
template <typename R, int N, int MODE> constexpr bool xi2_lean() {
  return sizeof(R) == 4 && N <= 256 && MODE != OUT_ADD_AND_STORE2;
}
template <typename R, int N, int MODE> constexpr int xi2_stage() { return xi2_lean<R, N, MODE>() ? 128 : kThreads; }

// The z pass holds all three components of its tile, so it takes 8 kx lines
// (64-byte rows in FP32) to keep two blocks per SM; one thread per first-stage item
// (3 components x R2 x 8), so the loads of all three components are in flight together.
constexpr int kZLines = 8;
template <typename R, int N, int R1, int R2>
constexpr int zsym2_threads() { return 3 * R2 * kZLines > 1024 ? 1024 : 3 * R2 * kZLines; }
// Threads of the plain z pass: one first-stage item each, except where the second stage
// with the symbol in registers (R1 items per line) would leave most of them idle: then
// R1 per line, and the first stage loops over its items.
template <typename R, int N, int R1, int R2>
constexpr int zplain_threads() {
  return (sizeof(R) == 4 && R2 <= 12 && 2 * R1 < 3 * R2) ? R1 * kZLines : zsym2_threads<R, N, R1, R2>();
}

// The work of one z tile (3 components x N z x NL kx lines, kx0..kx0+NL-1, storage y
// position py): forward z FFT, symbol, inverse z FFT.  The first stage reads the tile
// from global memory (FROM_SMEM false) or from `buf`, where a TMA copy has put it.
// Row of the z tile that holds spectral row R2 blk + n: within each block of R2 rows,
// odd blocks swap adjacent rows (R2 even).  The second FFT stage reads the same n of
// four consecutive blocks per warp; NL-line rows are 64 bytes in FP32, so without the
// swap the two blocks a half-warp touches would share banks.
template <int R2>
__device__ __forceinline__ int zrow(int blk, int n) {
  return R2 % 2 == 0 ? R2 * blk + (n ^ (blk & 1)) : R2 * blk + n;
}

template <typename R, int N, int R1, int R2, bool FROM_SMEM, int NT>
__device__ __forceinline__ void zsym_tile(cplx_t<R>* __restrict__ buf, const cplx_t<R>* __restrict__ tw,
                                          cplx_t<R>* __restrict__ base, size_t cs, size_t zs, int kx0, int py, int kx,
                                          const SymParams<R>& sp, const cplx_t<R>* __restrict__ dzt,
                                          const R* __restrict__ ddzt, int tid) {
  using C = cplx_t<R>;
  constexpr int NL = kZLines;
  constexpr bool HOLD3 = sizeof(R) == 4 && R2 <= 12;   // 3 x R2 complex in registers
  const C zero = mk(R(0), R(0));
  if constexpr (FROM_SMEM) {
    static_assert(NT == 3 * R2 * NL, "one first-stage item per thread");
    const int line = tid % NL, rest = tid / NL, n1 = rest % R2, c = rest / R2;
    C a[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) a[r] = buf[(c * N + n1 + R2 * r) * NL + line];
    stage_a_fwd<R, R1, R2>(a, tw + n1);
    // the tile landed in natural row order: every thread reads before the swapped writes
    if (R2 % 2 == 0) __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) buf[(c * N + zrow<R2>(k2, n1)) * NL + line] = a[k2];
  } else {
    for (int it = tid; it < 3 * R2 * NL; it += NT) {
      const int line = it % NL, rest = it / NL, n1 = rest % R2, c = rest / R2;
      const bool ok = kx0 + line < kx;
      C a[R1];
#pragma unroll
      for (int r = 0; r < R1; ++r) a[r] = ok ? base[c * cs + (size_t)(n1 + R2 * r) * zs + line] : zero;
      stage_a_fwd<R, R1, R2>(a, tw + n1);
#pragma unroll
      for (int k2 = 0; k2 < R1; ++k2) buf[(c * N + zrow<R2>(k2, n1)) * NL + line] = a[k2];
    }
  }
  __syncthreads();
  const C dyv = sp.dy[py];
  const R ddy = sp.ddy[py];
  if (HOLD3) {
    for (int it = tid; it < R1 * NL; it += NT) {
      const int line = it % NL, blk = it / NL, k = kx0 + line;
      if (k >= kx) continue;
      C b[3][R2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int n = 0; n < R2; ++n) b[c][n] = buf[(c * N + zrow<R2>(blk, n)) * NL + line];
        SDft<R, R2>::run(b[c]);
      }
      const C d0 = sp.dx[k];
      const R ddx = sp.ddx[k];
#pragma unroll
      for (int k1 = 0; k1 < R2; ++k1) {
        const int pz = R2 * blk + k1;
        apply_symbol<R>(b[0][k1], b[1][k1], b[2][k1], d0, dyv, dzt[pz], ddx + ddy + ddzt[pz], sp,
                        k == 0 && py == 0 && pz == 0);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sdft_inv<R, R2>(b[c]);
#pragma unroll
        for (int n = 0; n < R2; ++n) buf[(c * N + zrow<R2>(blk, n)) * NL + line] = b[c][n];
      }
    }
  } else {
    for (int it = tid; it < 3 * R1 * NL; it += NT) {
      const int line = it % NL, rest = it / NL, blk = rest % R1, c = rest / R1;
      C b[R2];
#pragma unroll
      for (int n = 0; n < R2; ++n) b[n] = buf[(c * N + zrow<R2>(blk, n)) * NL + line];
      SDft<R, R2>::run(b);
#pragma unroll
      for (int n = 0; n < R2; ++n) buf[(c * N + zrow<R2>(blk, n)) * NL + line] = b[n];
    }
    __syncthreads();
    // NT is a multiple of NL, so a thread keeps its line (and its x symbol) in every round
    static_assert(NT % NL == 0, "fixed line per thread");
    const int kt = kx0 + tid % NL;
    const C dxt = sp.dx[kt < kx ? kt : 0];
    const R dxy = sp.ddx[kt < kx ? kt : 0] + ddy;
    for (int it = tid; it < N * NL; it += NT) {
      const int pr = it / NL;                                  // row of the tile
      const int pz = zrow<R2>(pr / R2, pr % R2);               // its spectral row (the swap is an involution)
      if (kt >= kx) continue;
      C& c0 = buf[it];
      C& c1 = buf[N * NL + it];
      C& c2 = buf[2 * N * NL + it];
      apply_symbol<R>(c0, c1, c2, dxt, dyv, dzt[pz], dxy + ddzt[pz], sp, kt == 0 && py == 0 && pz == 0);
    }
    __syncthreads();
    for (int it = tid; it < 3 * R1 * NL; it += NT) {
      const int line = it % NL, rest = it / NL, blk = rest % R1, c = rest / R1;
      C b[R2];
#pragma unroll
      for (int n = 0; n < R2; ++n) b[n] = buf[(c * N + zrow<R2>(blk, n)) * NL + line];
      sdft_inv<R, R2>(b);
#pragma unroll
      for (int n = 0; n < R2; ++n) buf[(c * N + zrow<R2>(blk, n)) * NL + line] = b[n];
    }
  }
  __syncthreads();
  for (int it = tid; it < 3 * R2 * NL; it += NT) {
    const int line = it % NL, rest = it / NL, n1 = rest % R2, c = rest / R2;
    if (kx0 + line >= kx) continue;
    C a[R1];
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) a[k2] = buf[(c * N + zrow<R2>(k2, n1)) * NL + line];
    stage_a_inv<R, R1, R2>(a, tw + n1);
#pragma unroll
    for (int n2 = 0; n2 < R1; ++n2) base[c * cs + (size_t)(n1 + R2 * n2) * zs + line] = a[n2];
  }
}

template <typename R, int N, int R1, int R2>
__global__ void __launch_bounds__(zplain_threads<R, N, R1, R2>(), sizeof(R) == 4 ? 2 : 1)
    k_zsym2(cplx_t<R>* __restrict__ spec, const cplx_t<R>* __restrict__ gtw, int ny, int kx, int kxp, SymParams<R> sp,
            const RepFft* __restrict__ reps) {
  using C = cplx_t<R>;
  if (reps != nullptr) {   // replica blockIdx.z of a group solve
    const RepFft& rp = reps[blockIdx.z];
    spec = reinterpret_cast<C*>(rp.spec);
    sp.a = (R)rp.a;
    sp.b = (R)rp.b;
    sp.mean_scale = rp.a > 0.0 ? (R)((double)sp.inv_ntot / rp.a) : R(0);
    sp.k0sum = rp.k0sum;
    sp.k0mul = rp.k0mul;
  }
  constexpr int NL = kZLines;
  constexpr int NT = zplain_threads<R, N, R1, R2>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [3][N][NL]
  C* tw = buf + 3 * N * NL;                  // [N] first-stage twiddles, [k2][n1]
  const int tid = threadIdx.x;
  load_stage_twiddles<R, R1, R2>(tw, gtw, tid, NT);
  const int kx0 = blockIdx.x * NL, py = blockIdx.y;
  const size_t zs = (size_t)ny * kxp, cs = (size_t)N * zs;
  __syncthreads();
  zsym_tile<R, N, R1, R2, false, NT>(buf, tw, spec + (size_t)py * kxp + kx0, cs, zs, kx0, py, kx, sp, sp.dz, sp.ddz, tid);
}

// ---------------------------------------------------------------------------
// Persistent z pass fed by the tensor memory accelerator: a block loops over tiles,
// and while it transforms one tile (three 16-float x N boxes, one per component)
// the copy of its next tile lands in the other shared-memory buffer.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the barrier, giving up after limit_ns of global time
// (half a second unless given).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = 500000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}

// GRP: tiles of every replica of a group (reps, nrep; the map covers the group buffer).
template <typename R, int N, int R1, int R2, bool GRP = false>
__global__ void __launch_bounds__(zsym2_threads<R, N, R1, R2>(), sizeof(R) == 4 ? 2 : 1)
    k_zsym_tma(const __grid_constant__ CUtensorMap zmap, cplx_t<R>* __restrict__ spec,
               const cplx_t<R>* __restrict__ gtw, int ny, int kx, int kxp, int ntx, SymParams<R> sp, int* err,
               const RepFft* __restrict__ reps, int nrep) {
  using C = cplx_t<R>;
  constexpr int NL = kZLines;
  constexpr int NT = zsym2_threads<R, N, R1, R2>();
  constexpr int TILE = 3 * N * NL;
  constexpr uint32_t TILE_BYTES = TILE * sizeof(C);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // tensor copies land on 128-byte aligned shared addresses
  unsigned char* aligned = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  C* bufs = reinterpret_cast<C*>(aligned);             // [2 stages][3][N][NL]
  C* tw = bufs + 2 * TILE;                             // [N]
  C* zdz = tw + N;                                     // [N] z symbols (every tile uses them)
  R* zddz = reinterpret_cast<R*>(zdz + N);             // [N]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(zdz + N) + (N * sizeof(R) + 7) / 8;   // [2]
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  load_stage_twiddles<R, R1, R2>(tw, gtw, tid, NT);
  for (int i = tid; i < N; i += NT) {
    zdz[i] = sp.dz[i];
    zddz[i] = sp.ddz[i];
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // tiles: ntx x ny per spectrum; with reps, replica e = t / (ntx ny) of the table, whose
  // spectrum is the slot-th of the group buffer the map covers (components 3 slot ..)
  const int tpm = ntx * ny;
  const int ntiles = GRP ? tpm * nrep : tpm;
  const size_t zs = (size_t)ny * kxp, cs = (size_t)N * zs;
  auto issue = [&](int t, int st) {
    const int e = GRP ? t / tpm : 0, tt = t - e * tpm;
    const int kx0 = (tt % ntx) * NL, py = tt / ntx;
    const int c0 = GRP ? 3 * reps[e].slot : 0;
    // order this block's earlier generic-proxy writes of the buffer before the copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&mbar[st], TILE_BYTES);
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load_4d(bufs + st * TILE + c * N * NL, &zmap, 2 * kx0, py, 0, c0 + c, &mbar[st]);
  };
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) issue(t, 0);
  int i = 0;
  bool pending_other = false;
  for (; t < ntiles; ++i, t += gridDim.x) {
    const int st = i & 1;
    if (tid == 0) {
      pending_other = t + (int)gridDim.x < ntiles;
      if (pending_other) issue(t + gridDim.x, st ^ 1);
      s_ok = mbar_wait_bounded(&mbar[st], (i >> 1) & 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) break;
    const int e = GRP ? t / tpm : 0, tt = t - e * tpm;
    const int kx0 = (tt % ntx) * NL, py = tt / ntx;
    C* sbase = spec;
    SymParams<R> spt = sp;
    if constexpr (GRP) {   // the replica's spectrum and symbol
      const RepFft& rp = reps[e];
      sbase = reinterpret_cast<C*>(rp.spec);
      spt.a = (R)rp.a;
      spt.b = (R)rp.b;
      spt.mean_scale = rp.a > 0.0 ? (R)((double)sp.inv_ntot / rp.a) : R(0);
      spt.k0sum = rp.k0sum;
      spt.k0mul = rp.k0mul;
    }
    // (checked build) the tile's row and its last column lie inside the padded spectrum
    if (index_ok(py, ny, err) && index_ok(kx0 + NL - 1, kxp, err))
      zsym_tile<R, N, R1, R2, true, NT>(bufs + st * TILE, tw, sbase + (size_t)py * kxp + kx0, cs, zs, kx0, py, kx,
                                        spt, zdz, zddz, tid);
    __syncthreads();
  }
  if (tid == 0 && !s_ok && t < ntiles) {
    // A copy that has not landed after half a second: report it and leave.  Before
    // leaving, give both copies that may still be in flight into this block's shared
    // memory (the next tile's and the late one) another bounded wait.  If either is
    // still outstanding after that, the block's shared memory may yet be written after
    // it exits: the step's results are undefined and the host, which sees ICM_ETIMEOUT
    // at its next icm_sync, must destroy the simulation (as after ICM_ECUDA).
    atomicOr(err, DEV_ERR_TIMEOUT);
    if (pending_other) mbar_wait_bounded(&mbar[(i & 1) ^ 1], ((i + 1) >> 1) & 1);
    mbar_wait_bounded(&mbar[i & 1], (i >> 1) & 1);
  }
}

// First-stage radix of the z split a plan selects (fft_split_z_alt; the axis split
// where there is no other).
template <int N, int R1>
constexpr int zalt_r1() {
  return N == 32 ? 4 : N == 48 ? 12 : N == 64 ? 16 : N == 96 ? 8 : N == 128 ? 8 : N == 192 ? 12 : N == 256 ? 32 : R1;
}

// z planes per block of the y pass: short FP32 sides take several, so that the first
// stage (R2 items per line and plane) finds work for most of the block's threads.
template <typename R, int N, int R2>
constexpr int y_planes() {
  return sizeof(R) != 4 || N > 64 ? 1 : (R2 * seg_lines<R>() * 4 <= kThreads ? 4 : 2);
}

template <typename R, int N, int R1, int R2, bool INV>
__global__ void __launch_bounds__(kThreads) k_ypass2(cplx_t<R>* __restrict__ spec, const cplx_t<R>* __restrict__ gtw,
                                                     int nz, int kx, int kxp, const RepFft* __restrict__ reps) {
  using C = cplx_t<R>;
  constexpr int NL = seg_lines<R>();
  constexpr int ZB = y_planes<R, N, R2>();
  if (reps != nullptr) spec = reinterpret_cast<C*>(reps[blockIdx.z / 3].spec);   // group solve: 3 components per replica
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [ZB][N][NL]
  C* tw = buf + ZB * N * NL;
  const int tid = threadIdx.x;
  // The forward pass walks the spectrum backwards (last component, last z planes, last
  // columns first): the x pass before it wrote those last, so the first blocks find
  // them in L2.  The inverse pass walks forwards.
  const int bx = INV ? blockIdx.x : gridDim.x - 1 - blockIdx.x;
  const int by = INV ? blockIdx.y : gridDim.y - 1 - blockIdx.y;
  const int kx0 = bx * NL, z0 = by * ZB, comp = INV ? blockIdx.z % 3 : 2 - blockIdx.z % 3;
  // plane z0 + zb of the component, columns kx0..
  C* base0 = spec + ((size_t)(comp * nz + z0) * N) * kxp + kx0;
  const C zero = mk(R(0), R(0));
  if (!INV) {
    // the loads of this thread's first item go out before the twiddle table is staged
    // (whose barrier they would otherwise wait behind)
    const auto load_item = [&](int it, C (&a)[R1]) {
      const int line = it % NL, rest = it / NL, n1 = rest % R2, zb = rest / R2;
      const bool ok = kx0 + line < kx && z0 + zb < nz;
      const C* base = base0 + (size_t)zb * N * kxp;
#pragma unroll
      for (int r = 0; r < R1; ++r) a[r] = ok ? base[(size_t)(n1 + R2 * r) * kxp + line] : zero;
    };
    C a[R1];
    if (tid < ZB * R2 * NL) load_item(tid, a);
    load_stage_twiddles<R, R1, R2>(tw, gtw, tid, kThreads);
    __syncthreads();
    for (int it = tid; it < ZB * R2 * NL; it += kThreads) {
      const int line = it % NL, rest = it / NL, n1 = rest % R2, zb = rest / R2;
      if (it != tid) load_item(it, a);
      stage_a_fwd<R, R1, R2>(a, tw + n1);
#pragma unroll
      for (int k2 = 0; k2 < R1; ++k2) buf[(zb * N + n1 + R2 * k2) * NL + line] = a[k2];
    }
    __syncthreads();
    for (int it = tid; it < ZB * R1 * NL; it += kThreads) {
      const int line = it % NL, rest = it / NL, blk = rest % R1, zb = rest / R1;
      if (kx0 + line >= kx || z0 + zb >= nz) continue;
      C* base = base0 + (size_t)zb * N * kxp;
      C b[R2];
#pragma unroll
      for (int n = 0; n < R2; ++n) b[n] = buf[(zb * N + R2 * blk + n) * NL + line];
      SDft<R, R2>::run(b);
#pragma unroll
      for (int k1 = 0; k1 < R2; ++k1) base[(size_t)(R2 * blk + k1) * kxp + line] = b[k1];
    }
  } else {
    // the second stage comes first and needs no twiddles: its loads go out first, the
    // table is staged after it, before the barrier the first stage waits at anyway
    for (int it = tid; it < ZB * R1 * NL; it += kThreads) {
      const int line = it % NL, rest = it / NL, blk = rest % R1, zb = rest / R1;
      const bool ok = kx0 + line < kx && z0 + zb < nz;
      const C* base = base0 + (size_t)zb * N * kxp;
      C b[R2];
#pragma unroll
      for (int k1 = 0; k1 < R2; ++k1) b[k1] = ok ? base[(size_t)(R2 * blk + k1) * kxp + line] : zero;
      sdft_inv<R, R2>(b);
#pragma unroll
      for (int n = 0; n < R2; ++n) buf[(zb * N + R2 * blk + n) * NL + line] = b[n];
    }
    load_stage_twiddles<R, R1, R2>(tw, gtw, tid, kThreads);
    __syncthreads();
    for (int it = tid; it < ZB * R2 * NL; it += kThreads) {
      const int line = it % NL, rest = it / NL, n1 = rest % R2, zb = rest / R2;
      if (kx0 + line >= kx || z0 + zb >= nz) continue;
      C* base = base0 + (size_t)zb * N * kxp;
      C a[R1];
#pragma unroll
      for (int k2 = 0; k2 < R1; ++k2) a[k2] = buf[(zb * N + n1 + R2 * k2) * NL + line];
      stage_a_inv<R, R1, R2>(a, tw + n1);
#pragma unroll
      for (int n2 = 0; n2 < R1; ++n2) base[(size_t)(n1 + R2 * n2) * kxp + line] = a[n2];
    }
  }
}

// The x forward transform of the 32 rows row0.. (16 complex lines, two real rows each)
// of component comp into buf: frequency k of line l ends at position
// R2 (k mod R1) + k div R1 of the line.  BLOBS: before the transform, the blobs of row
// block `bin` spread rb.vec into the rows (in shared memory, where the first stage
// reads them; NST records staged by cp.async in `stage_mem`), added to src if src is
// set.  The first-stage twiddles tw are loaded by the caller; ends with a block barrier.
template <typename R, int N, int R1, int R2, bool BLOBS, int NST, int L = kXLines, bool MAYBE_NO_VEC = false>
__device__ __forceinline__ void x_forward_rows(cplx_t<R>* __restrict__ buf, const cplx_t<R>* __restrict__ tw,
                                               unsigned char* stage_mem, const R* __restrict__ src, long long row0,
                                               int nrows, long long ncell, int comp, int bin, const RowBlobs& rb,
                                               int tid) {
  using C = cplx_t<R>;
  static_assert(kRowBlock == 2 * kXLines, "row blocks are the x-pass blocks");
  static_assert(!BLOBS || L == kXLines, "blob work takes one row block per block");
  const bool dense = !BLOBS || src != nullptr;
  // blob work of this block; with MAYBE_NO_VEC none where the source vector is absent
  // (a replica of a group solve without forces), uniform over the block
  const bool blobs = BLOBS && (!MAYBE_NO_VEC || rb.vec != nullptr);
  // one first-stage item (line l, offset n1) per thread; its loads are issued first
  constexpr int ITEMS = L * R2;
  static_assert(ITEMS <= kThreads, "one first-stage item per thread");
  const int n1 = tid % R2, l = tid / R2;
  const long long r0 = row0 + 2 * l;
  const R* p0 = src + comp * ncell + r0 * N;
  const bool ok0 = dense && tid < ITEMS && r0 < nrows, ok1 = ok0 && r0 + 1 < nrows;
  C a[R1];
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int x = n1 + R2 * r;
    a[r] = mk(ok0 ? p0[x] : R(0), ok1 ? p0[N + x] : R(0));
  }
  if (blobs) {
    // this block's tasks: records staged by cp.async while the buffer is zeroed
    StagedTask<R>* stage = reinterpret_cast<StagedTask<R>*>(stage_mem);
    const BlobStencil<R>* rec = reinterpret_cast<const BlobStencil<R>*>(rb.geo);
    const int s0 = rb.start[bin], e = rb.start[bin + 1];
    const int nst = min(e - s0, NST);
    if (tid < nst) stage_task<R>(&stage[tid], rec, rb.list[s0 + tid], comp, rb.vec);
    cp_async_commit();
    for (int i = tid; i < L * xrow(N); i += kThreads) buf[i] = mk(R(0), R(0));
    cp_async_wait_all();
    __syncthreads();
    R* rows = reinterpret_cast<R*>(buf);
    const double inv_dvf = rb.p.inv_h * rb.p.inv_h * rb.p.inv_h;
    const auto line = [](int ln, int x) { return xaddr(ln, x, N); };
    const bool plane = rb.p.ny % kRowBlock == 0;   // the block is part of one z plane
    const int z0 = (int)row0 / rb.p.ny, y0 = (int)row0 % rb.p.ny;
    if (tid < nst) {
      const StagedTask<R>& t = stage[tid];
      spread_one<R, N>(rows, (int)row0, plane, z0, y0, t.first, t.w, (R)(t.vec * inv_dvf), rb.p, line);
    }
    for (int i = s0 + NST + tid; i < e; i += kThreads) {   // beyond the staged tasks
      const int b = rb.list[i];
      spread_one<R, N>(rows, (int)row0, plane, z0, y0, *reinterpret_cast<const int4*>(rec[b].first[comp]),
                       &rec[b].w[comp][0][0], (R)(rb.vec[3 * b + comp] * inv_dvf), rb.p, line);
    }
  }
  __syncthreads();
  if (tid < ITEMS) {
    if (blobs) {
#pragma unroll
      for (int r = 0; r < R1; ++r) a[r] = cadd(a[r], buf[xaddr(l, n1 + R2 * r, N)]);
    }
    stage_a_fwd<R, R1, R2>(a, tw + n1);
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) buf[xaddr(l, n1 + R2 * k2, N)] = a[k2];
  }
  __syncthreads();
  for (int it = tid; it < L * R1; it += kThreads) {
    const int blk = it % R1, l = it / R1;
    C b[R2];
#pragma unroll
    for (int n = 0; n < R2; ++n) b[n] = buf[xaddr(l, R2 * blk + n, N)];
    SDft<R, R2>::run(b);
#pragma unroll
    for (int k1 = 0; k1 < R2; ++k1) buf[xaddr(l, R2 * blk + k1, N)] = b[k1];
  }
  __syncthreads();
}

// The two half spectra of line l at wavenumber k from the transformed lines in buf.
template <typename R, int N, int R1, int R2>
__device__ __forceinline__ void split_half_spectra(const cplx_t<R>* __restrict__ buf, int l, int k, cplx_t<R>& x1,
                                                   cplx_t<R>& x2) {
  using C = cplx_t<R>;
  const int km = k == 0 ? 0 : N - k;
  const C zk = buf[xaddr(l, R2 * (k % R1) + k / R1, N)];
  const C zm = buf[xaddr(l, R2 * (km % R1) + km / R1, N)];
  x1 = mk((zk.x + zm.x) * R(0.5), (zk.y - zm.y) * R(0.5));
  x2 = cmul_mi(mk((zk.x - zm.x) * R(0.5), (zk.y + zm.y) * R(0.5)));
}

// x forward pass: x_forward_rows, then the half spectra of the rows to spec.
// GRP: a group solve whose replicas carry their own blob work (reps[i].rb); otherwise rb.
template <typename R, int N, int R1, int R2, bool BLOBS, bool GRP = false>
__global__ void __launch_bounds__(kThreads, xf2_min_blocks<R, N>()) k_xfwd2(const R* __restrict__ src, cplx_t<R>* __restrict__ spec,
                                                    const cplx_t<R>* __restrict__ gtw, int nrows, long long ncell,
                                                    int kx, int kxp, RowBlobs rb, const RepFft* __restrict__ reps) {
  using C = cplx_t<R>;
  if ((!BLOBS || GRP) && reps != nullptr) {   // replica blockIdx.y / 3 of a group solve
    const RepFft& rp = reps[blockIdx.y / 3];
    src = reinterpret_cast<const R*>(rp.src);
    spec = reinterpret_cast<C*>(rp.spec);
  }
  constexpr int L = BLOBS ? kXLines : x_plain_lines<R, N, R2>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [L][xrow(N)]
  C* tw = buf + L * xrow(N);
  const int tid = threadIdx.x;
  load_stage_twiddles<R, R1, R2>(tw, gtw, tid, kThreads);
  const int comp = blockIdx.y % 3;
  const long long row0 = (long long)blockIdx.x * (2 * L);
  if constexpr (GRP)
    x_forward_rows<R, N, R1, R2, BLOBS, kStageF, L, true>(buf, tw, smem_raw + stage_offset<R, N>(), src, row0, nrows,
                                                       ncell, comp, blockIdx.x, *reps[blockIdx.y / 3].rb, tid);
  else
    x_forward_rows<R, N, R1, R2, BLOBS, kStageF, L>(buf, tw, smem_raw + stage_offset<R, N>(), src, row0, nrows,
                                                 ncell, comp, blockIdx.x, rb, tid);
  C* out = spec + (size_t)comp * nrows * kxp;
  // the two half spectra of line l at wavenumber k (kx = N/2 + 1 of them)
  const auto split = [&](int l, int k) {
    C x1, x2;
    split_half_spectra<R, N, R1, R2>(buf, l, k, x1, x2);
    const long long r1 = row0 + 2 * l;
    if (r1 < nrows) out[r1 * kxp + k] = x1;
    if (r1 + 1 < nrows) out[(r1 + 1) * kxp + k] = x2;
  };
  // k < N/2 with a compile-time (mostly power-of-two) index split, then k = N/2
  constexpr int H = N / 2;
  for (int it = tid; it < L * H; it += kThreads) split(it / H, it % H);
  if (tid < L) split(tid, H);
}

// ---------------------------------------------------------------------------
// Forward x and y passes fused on thread-block clusters (FP32, Nx = Ny = N, N a
// multiple of 32).  A cluster of N/32 blocks holds one z plane of one component:
// block r transforms rows y = 32 r .. 32 r + 31 along x (with the blob spread, as
// k_xfwd2) and keeps their half spectra in its shared memory; after a cluster barrier
// it transforms kx columns 16 r .. 16 r + 15 along y (rank 0 also the Nyquist column
// N/2), reading the rows of every block of the cluster through distributed shared
// memory, and writes them to the spectrum exactly as the y pass does.  The half
// spectrum thus never makes the round trip through HBM between the two passes.
// ---------------------------------------------------------------------------
constexpr int kYL = 17;   // lines of the y buffer: 16 kx columns (+ the Nyquist column)
template <int N> constexpr int xy_pitch() { return N / 2 + 1; }
template <int N> size_t smem_xyf() {
  return (size_t)(kYL * N + N + kRowBlock * xy_pitch<N>()) * sizeof(cplx_t<float>);
}

template <int N, int R1, int R2, bool BLOBS>
__global__ void __launch_bounds__(kThreads, 3) k_xyf(const float* __restrict__ src, cplx_t<float>* __restrict__ spec,
                                                     const cplx_t<float>* __restrict__ gtw, int nz, long long ncell,
                                                     int kxp, RowBlobs rb) {
  using R = float;
  using C = cplx_t<R>;
  namespace cg = cooperative_groups;
  constexpr int CL = N / kRowBlock;   // blocks per cluster
  constexpr int XP = xy_pitch<N>();
  constexpr int H = N / 2;
  static_assert(kYL * N == kXLines * xrow(N), "the y lines overlay the x rows");
  static_assert(kRowBlock % R2 == 0, "a first-stage item's rows lie in one block");
  static_assert(R1 * 16 <= kThreads && R2 * 16 <= kThreads, "one y item per thread");
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // x rows [16][xrow(N)], later the y lines [N][kYL]
  C* tw = buf + kYL * N;                     // first-stage twiddles (the y side is the x side)
  C* X = tw + N;                             // half spectra of this block's rows [32][XP]
  const int tid = threadIdx.x;
  const int rank = blockIdx.x, z = blockIdx.y, comp = blockIdx.z;
  load_stage_twiddles<R, R1, R2>(tw, gtw, tid, kThreads);
  const long long row0 = (long long)z * N + kRowBlock * rank;
  x_forward_rows<R, N, R1, R2, BLOBS, 0>(buf, tw, nullptr, src, row0, N * nz, ncell, comp, z * CL + rank, rb, tid);
  for (int it = tid; it < kXLines * H; it += kThreads) {
    const int l = it / H, k = it % H;
    C x1, x2;
    split_half_spectra<R, N, R1, R2>(buf, l, k, x1, x2);
    X[(2 * l) * XP + k] = x1;
    X[(2 * l + 1) * XP + k] = x2;
  }
  if (tid < kXLines) {
    C x1, x2;
    split_half_spectra<R, N, R1, R2>(buf, tid, H, x1, x2);
    X[(2 * tid) * XP + H] = x1;
    X[(2 * tid + 1) * XP + H] = x2;
  }
  cluster.sync();   // the half spectra of every block are complete; buf is free
  C* Y = buf;
  const int kx0 = 16 * rank;
  // y, first stage: item (line, n1) reads rows n1 + R2 r of column k from their blocks
  const auto stage_a = [&](int line, int n1, int k) {
    C a[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      constexpr int kR = kRowBlock;
      const int sblk = (R2 * r) / kR;
      const C* Xs = cluster.map_shared_rank(X, sblk);
      a[r] = Xs[(n1 + R2 * r - kR * sblk) * XP + k];
    }
    stage_a_fwd<R, R1, R2>(a, tw + n1);
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) Y[(n1 + R2 * k2) * kYL + line] = a[k2];
  };
  if (tid < R2 * 16) stage_a(tid % 16, tid / 16, kx0 + tid % 16);
  if (rank == 0 && tid < R2) stage_a(16, tid, H);
  cluster.sync();   // every remote read is done (blocks may leave); the y lines are complete
  C* base = spec + ((size_t)(comp * nz + z) * N) * kxp;
  // y, second stage: to the spectrum in storage order, as the y pass writes it
  const auto stage_b = [&](int line, int blk, int k) {
    C b[R2];
#pragma unroll
    for (int n = 0; n < R2; ++n) b[n] = Y[(R2 * blk + n) * kYL + line];
    SDft<R, R2>::run(b);
#pragma unroll
    for (int k1 = 0; k1 < R2; ++k1) base[(size_t)(R2 * blk + k1) * kxp + k] = b[k1];
  };
  if (tid < R1 * 16) stage_b(tid % 16, tid / 16, kx0 + tid % 16);
  if (rank == 0 && tid < R1) stage_b(16, tid, H);
}
#define ICM_XY_SIDES(X) X(32, 8, 4) X(64, 8, 8) X(128, 16, 8) X(256, 16, 16)

// MODE OUT_STORE: dst = x.  OUT_ADD_AND_STORE2: dst += x, dst2 = x.  OUT_ADD: dst += x.
// OUT_NONE: nothing stored.  The old dst values of the adding modes are loaded at
// kernel start so that they are in flight during the FFT (lean variant: before the
// last stage).  GATHER 1: the blobs of
// this row block add the part of J x in these rows to rb.acc; GATHER 2: also J L x
// (without 1/h^2) to rb.acc_lap.  x stays in shared memory for the gathers.
// GRP: a group solve whose replicas gather into their own accumulators (reps[i].rb).
template <typename R, int N, int R1, int R2, int MODE, int GATHER, bool GRP = false>
__global__ void __launch_bounds__(kThreads, xi2_lean<R, N, MODE>() ? 4 : 1) k_xinv2(const cplx_t<R>* __restrict__ spec, R* __restrict__ dst,
                                                    R* __restrict__ dst2, const cplx_t<R>* __restrict__ gtw,
                                                    int nrows, long long ncell, int kxp, RowBlobs rb0,
                                                    const RepFft* __restrict__ reps) {
  using C = cplx_t<R>;
  if ((GATHER == 0 || GRP) && reps != nullptr) {   // replica blockIdx.y / 3 of a group solve
    const RepFft& rp = reps[blockIdx.y / 3];
    spec = reinterpret_cast<const C*>(rp.spec);
    dst = reinterpret_cast<R*>(rp.dst);
    dst2 = reinterpret_cast<R*>(rp.dst2);
  }
  const RowBlobs& rb = GRP ? *reps[blockIdx.y / 3].rb : rb0;
  constexpr bool ADDS = MODE == OUT_ADD_AND_STORE2 || MODE == OUT_ADD;
  constexpr bool LEAN = xi2_lean<R, N, MODE>();
  constexpr int NST = xi2_stage<R, N, MODE>();
  // (the two-output mode keeps 16 lines: more would hold all its loads in registers)
  constexpr int L = GATHER || MODE == OUT_ADD_AND_STORE2 ? kXLines : x_plain_lines<R, N, R2>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw = buf + L * xrow(N);
  const int tid = threadIdx.x;
  load_stage_twiddles<R, R1, R2>(tw, gtw, tid, kThreads);
  // Rows are taken backwards (last component, last row blocks first): the inverse y pass
  // before this one wrote them last, so the first blocks find them in L2.
  const int comp = 2 - blockIdx.y % 3;
  const int bx = gridDim.x - 1 - blockIdx.x;
  const long long row0 = (long long)bx * (2 * L);
  const C* in = spec + (size_t)comp * nrows * kxp;
  const C zero = mk(R(0), R(0));
  const size_t cb = (size_t)comp * ncell;
  // this thread's output positions: line l = tid / R2, x = n1 + R2 n2, rows r0 and r0 + 1
  constexpr int OUTS = (L * R2 + kThreads - 1) / kThreads;
  R old0[ADDS ? OUTS * R1 : 1], old1[ADDS ? OUTS * R1 : 1];
  const auto load_old = [&](int o) {
    const int it = tid + o * kThreads;
    const int n1 = it % R2, l = it / R2;
    const long long r0 = row0 + 2 * l;
#pragma unroll
    for (int n2 = 0; n2 < R1; ++n2) {
      const int x = n1 + R2 * n2;
      old0[o * R1 + n2] = (it < L * R2 && r0 < nrows) ? dst[cb + (size_t)r0 * N + x] : R(0);
      old1[o * R1 + n2] = (it < L * R2 && r0 + 1 < nrows) ? dst[cb + (size_t)(r0 + 1) * N + x] : R(0);
    }
  };
  if (ADDS && !LEAN) {
#pragma unroll
    for (int o = 0; o < OUTS; ++o) load_old(o);
  }
  constexpr int LOADS = (L * N + kThreads - 1) / kThreads;   // compile-time: loads in flight together
  constexpr int BATCH = LEAN ? (LOADS + 1) / 2 : LOADS;
  int g0 = 0, ge = 0;
#pragma unroll
  for (int j0 = 0; j0 < LOADS; j0 += BATCH) {
    C av[BATCH], bv[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int it = tid + (j0 + j) * kThreads;
      const int k = it % N, l = it / N;
      const long long r1 = row0 + 2 * l;
      const int kk = 2 * k <= N ? k : N - k;
      const bool ok = j0 + j < LOADS && it < L * N;
      av[j] = (ok && r1 < nrows) ? in[r1 * kxp + kk] : zero;
      bv[j] = (ok && r1 + 1 < nrows) ? in[(r1 + 1) * kxp + kk] : zero;
    }
    // the gathers' records: staged by cp.async while the spectrum loads are in flight
    if (GATHER && j0 == 0) {
      StagedTask<R>* stage = reinterpret_cast<StagedTask<R>*>(smem_raw + stage_offset<R, N>());
      g0 = rb.start[bx];
      ge = rb.start[bx + 1];
      if (tid < min(ge - g0, NST))
        stage_task<R>(&stage[tid], reinterpret_cast<const BlobStencil<R>*>(rb.geo), rb.list[g0 + tid], comp, nullptr);
      cp_async_commit();
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int it = tid + (j0 + j) * kThreads;
      if (j0 + j >= LOADS || it >= L * N) continue;
      const int k = it % N, l = it / N;
      C a = av[j], b = bv[j];
      if (2 * k > N) {
        a = cconj(a);
        b = cconj(b);
      }
      if (k == 0 || 2 * k == N) {
        a.y = R(0);
        b.y = R(0);
      }
      buf[xaddr(l, R2 * (k % R1) + k / R1, N)] = mk(a.x - b.y, a.y + b.x);
    }
  }
  __syncthreads();
  for (int it = tid; it < L * R1; it += kThreads) {
    const int blk = it % R1, l = it / R1;
    C b[R2];
#pragma unroll
    for (int k1 = 0; k1 < R2; ++k1) b[k1] = buf[xaddr(l, R2 * blk + k1, N)];
    sdft_inv<R, R2>(b);
#pragma unroll
    for (int n = 0; n < R2; ++n) buf[xaddr(l, R2 * blk + n, N)] = b[n];
  }
  __syncthreads();
#pragma unroll
  for (int o = 0; o < OUTS; ++o) {
    const int it = tid + o * kThreads;
    if (it >= L * R2) break;
    const int n1 = it % R2, l = it / R2;
    if (ADDS && LEAN) load_old(o);   // in flight during the last stage
    C a[R1];
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) a[k2] = buf[xaddr(l, n1 + R2 * k2, N)];
    stage_a_inv<R, R1, R2>(a, tw + n1);
    if (GATHER) {
      // the same positions this thread read: in place
#pragma unroll
      for (int n2 = 0; n2 < R1; ++n2) buf[xaddr(l, n1 + R2 * n2, N)] = a[n2];
    }
    if (MODE == OUT_NONE) continue;
    const long long r0 = row0 + 2 * l;
#pragma unroll
    for (int n2 = 0; n2 < R1; ++n2) {
      const int x = n1 + R2 * n2;
      if (r0 < nrows) {
        const size_t ox = cb + (size_t)r0 * N + x;
        if (MODE == OUT_STORE) {
          dst[ox] = a[n2].x;
        } else {
          dst[ox] = old0[o * R1 + n2] + a[n2].x;
          if (MODE == OUT_ADD_AND_STORE2) dst2[ox] = a[n2].x;
        }
      }
      if (r0 + 1 < nrows) {
        const size_t ox = cb + (size_t)(r0 + 1) * N + x;
        if (MODE == OUT_STORE) {
          dst[ox] = a[n2].y;
        } else {
          dst[ox] = old1[o * R1 + n2] + a[n2].y;
          if (MODE == OUT_ADD_AND_STORE2) dst2[ox] = a[n2].y;
        }
      }
    }
  }
  if (GATHER) {
    cp_async_wait_all();
    __syncthreads();
    const R* rows = reinterpret_cast<const R*>(buf);
    const StagedTask<R>* stage = reinterpret_cast<const StagedTask<R>*>(smem_raw + stage_offset<R, N>());
    const BlobStencil<R>* rec = reinterpret_cast<const BlobStencil<R>*>(rb.geo);
    const auto line = [](int l, int x) { return xaddr(l, x, N); };
    const bool plane = rb.p.ny % kRowBlock == 0;   // the block is part of one z plane
    const int z0 = (int)row0 / rb.p.ny, y0 = (int)row0 % rb.p.ny;
    if (tid < min(ge - g0, NST)) {
      const StagedTask<R>& t = stage[tid];
      R j, jl;
      gather_one<R, N, GATHER == 2>(rows, (int)row0, plane, z0, y0, t.first, t.w, rb.p, line, j, jl);
      atomicAdd(&rb.acc[3 * t.b + comp], (double)j);
      if (GATHER == 2) atomicAdd(&rb.acc_lap[3 * t.b + comp], (double)jl);
    }
    for (int i = g0 + NST + tid; i < ge; i += kThreads) {   // beyond the staged tasks
      const int b = rb.list[i];
      R j, jl;
      gather_one<R, N, GATHER == 2>(rows, (int)row0, plane, z0, y0, *reinterpret_cast<const int4*>(rec[b].first[comp]),
                                    &rec[b].w[comp][0][0], rb.p, line, j, jl);
      atomicAdd(&rb.acc[3 * b + comp], (double)j);
      if (GATHER == 2) atomicAdd(&rb.acc_lap[3 * b + comp], (double)jl);
    }
  }
}

template <typename R, int N> size_t smem_ztma() {
  return 2 * 3 * (size_t)N * kZLines * sizeof(cplx_t<R>) + 2 * N * sizeof(cplx_t<R>) + (N * sizeof(R) + 7) / 8 * 8 + 16 + 128;
}
template <typename R, int N> size_t smem_z2() { return 3 * (size_t)N * kZLines * sizeof(cplx_t<R>) + N * sizeof(cplx_t<R>); }
template <typename R, int N, int R2> size_t smem_y2() {
  return (size_t)y_planes<R, N, R2>() * N * seg_lines<R>() * sizeof(cplx_t<R>) + N * sizeof(cplx_t<R>);
}
template <typename R, int N, int R1, int R2, bool GRP>
void launch_ztma(int grid, const CUtensorMap& map, cplx_t<R>* spec, const cplx_t<R>* tw, const FftCtx<R>& f, int kxz,
                 const SymParams<R>& sp, const RepFft* reps, int G, cudaStream_t st) {
  k_zsym_tma<R, N, R1, R2, GRP><<<grid, zsym2_threads<R, N, R1, R2>(), smem_ztma<R, N>(), st>>>(
      map, spec, tw, f.ny, f.kx, f.kxp, kxz, sp, f.err, reps, G);
}

template <typename R, int N, int R1, int R2>
void launch_zplain(dim3 grid, cplx_t<R>* spec, const cplx_t<R>* tw, const FftCtx<R>& f, const SymParams<R>& sp,
                   const RepFft* reps, cudaStream_t st) {
  k_zsym2<R, N, R1, R2><<<grid, zplain_threads<R, N, R1, R2>(), smem_z2<R, N>(), st>>>(spec, tw, f.ny, f.kx, f.kxp,
                                                                                    sp, reps);
}

template <typename R, int N, int L> size_t smem_x2() { return (size_t)L * xrow(N) * sizeof(cplx_t<R>) + N * sizeof(cplx_t<R>); }
// Blocks of a plain x pass over nrows rows (2 x_plain_lines rows per block).
template <typename R, int N, int R2> int xgrid(int nrows) {
  constexpr int L = x_plain_lines<R, N, R2>();
  return (nrows + 2 * L - 1) / (2 * L);
}

// Every side with register kernels, as (N, R1, R2); must agree with fft_split.
#define ICM_FFT_SIDES(X) \
  X(32, 8, 4)            \
  X(48, 16, 3)           \
  X(64, 8, 8)            \
  X(96, 16, 6)           \
  X(128, 16, 8)          \
  X(192, 16, 12)         \
  X(256, 16, 16)         \
  X(384, 32, 12)         \
  X(512, 32, 16)

template <typename R> size_t smem_x(int n) { return (size_t)n * kXLS * sizeof(cplx_t<R>) + n * sizeof(cplx_t<R>) + n * sizeof(int); }
template <typename R> size_t smem_y(int n) { return (size_t)n * seg_lines<R>() * sizeof(cplx_t<R>) + n * sizeof(cplx_t<R>); }
template <typename R> size_t smem_z(int n) { return 3 * (size_t)n * seg_lines<R>() * sizeof(cplx_t<R>) + n * sizeof(cplx_t<R>); }

// Sides of the fused x-y forward pass whose clusters the device can hold.
int g_xy_sides = 0;   // bit per entry of ICM_XY_SIDES

template <typename R>
void set_xf_attributes() {
  const int big = 227 * 1024;
#define ICM_ATTR(N, R1, R2)                                                                                        \
  cudaFuncSetAttribute(k_xfwd2<R, N, R1, R2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);           \
  cudaFuncSetAttribute(k_xfwd2<R, N, R1, R2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);            \
  cudaFuncSetAttribute(k_xfwd2<R, N, R1, R2, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  ICM_FFT_SIDES(ICM_ATTR)
#undef ICM_ATTR
  cudaFuncSetAttribute(k_xfwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if constexpr (sizeof(R) == 4) {
  int bit = 0, sides = 0;
#define ICM_ATTR(N, R1, R2)                                                                                        \
  {                                                                                                                \
    bool ok = true;                                                                                                \
    for (int b = 0; b < 2; ++b) {                                                                                  \
      const void* fn = b ? (const void*)k_xyf<N, R1, R2, true> : (const void*)k_xyf<N, R1, R2, false>;             \
      ok &= cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_xyf<N>()) == cudaSuccess; \
      cudaLaunchConfig_t cfg = {};                                                                                 \
      cfg.gridDim = dim3(N / kRowBlock, 1, 3);                                                                     \
      cfg.blockDim = dim3(kThreads);                                                                               \
      cfg.dynamicSmemBytes = smem_xyf<N>();                                                                        \
      cudaLaunchAttribute at;                                                                                      \
      at.id = cudaLaunchAttributeClusterDimension;                                                                 \
      at.val.clusterDim.x = N / kRowBlock;                                                                         \
      at.val.clusterDim.y = 1;                                                                                     \
      at.val.clusterDim.z = 1;                                                                                     \
      cfg.attrs = &at;                                                                                             \
      cfg.numAttrs = 1;                                                                                            \
      int nc = 0;                                                                                                  \
      ok &= cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc > 0;                                \
    }                                                                                                              \
    if (ok) sides |= 1 << bit;                                                                                     \
    ++bit;                                                                                                         \
  }
  ICM_XY_SIDES(ICM_ATTR)
#undef ICM_ATTR
  cudaGetLastError();
  g_xy_sides = sides;
  }
}

template <typename R>
void set_xi_attributes() {
  const int big = 227 * 1024;
#define ICM_ATTR(N, R1, R2)                                                                                        \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_STORE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);    \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_ADD_AND_STORE2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_STORE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);    \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_NONE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);     \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_ADD, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);     \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_STORE, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_NONE, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);  \
  cudaFuncSetAttribute(k_xinv2<R, N, R1, R2, OUT_ADD, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  ICM_FFT_SIDES(ICM_ATTR)
#undef ICM_ATTR
  cudaFuncSetAttribute(k_xinv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

template <typename R>
void set_yz_attributes() {
  const int big = 227 * 1024;
#define ICM_ATTR(N, R1, R2)                                                                               \
  cudaFuncSetAttribute(k_zsym2<R, N, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);         \
  cudaFuncSetAttribute(k_zsym2<R, N, zalt_r1<N, R1>(), N / zalt_r1<N, R1>()>,                              \
                       cudaFuncAttributeMaxDynamicSharedMemorySize, big);                                   \
  if (N <= 256) {                                                                                           \
    cudaFuncSetAttribute(k_zsym_tma<R, N, zalt_r1<N, R1>(), N / zalt_r1<N, R1>()>,                         \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ztma<R, N>());              \
    cudaFuncSetAttribute(k_zsym_tma<R, N, zalt_r1<N, R1>(), N / zalt_r1<N, R1>(), true>,                   \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ztma<R, N>());              \
  }                                                                                                         \
  if (N <= 256) /* exactly its need: the kernel also holds static shared memory */                          \
    cudaFuncSetAttribute(k_zsym_tma<R, N, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ztma<R, N>()); \
  if (N <= 256)                                                                                             \
    cudaFuncSetAttribute(k_zsym_tma<R, N, R1, R2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                         (int)smem_ztma<R, N>());                                                           \
  cudaFuncSetAttribute(k_ypass2<R, N, R1, R2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
  cudaFuncSetAttribute(k_ypass2<R, N, R1, R2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  ICM_FFT_SIDES(ICM_ATTR)
#undef ICM_ATTR
  cudaFuncSetAttribute(k_ypass<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_ypass<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_zsym<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace

// This file is compiled as six objects in parallel (-DICM_FFT_SHARD=k): for FP32,
// k = 0 the forward x passes and the precision-independent code, 1 the y and z
// passes, 2 the inverse x passes; k = 3, 4, 5 the same for FP64.  Without the macro
// one object holds everything.
#ifndef ICM_FFT_SHARD
#define ICM_FFT_SHARD -1
#endif
#define ICM_SHARD(k) (ICM_FFT_SHARD < 0 || ICM_FFT_SHARD == (k))

// SMs of the current device (persistent grids), read once.
inline int device_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    nsm = n > 0 ? n : 1;
  }
  return nsm;
}

template <typename R> void fft_prepare_xf() { set_xf_attributes<R>(); }
template <typename R> void fft_prepare_xi() { set_xi_attributes<R>(); }
template <typename R> void fft_prepare_yz() { set_yz_attributes<R>(); }

template <typename R>
void fft_x_forward(const FftCtx<R>& f, const R* src, cudaStream_t st) {
  const int nrows = f.ny * f.nz;
  const int xblocks = (nrows + 2 * kXLines - 1) / (2 * kXLines);
  const cplx_t<R>* tw = (const cplx_t<R>*)f.px.tw;
  switch (f.nx) {
#define ICM_CASE(N, R1, R2) \
  case N: k_xfwd2<R, N, R1, R2, false><<<dim3(xgrid<R, N, R2>(nrows), 3), kThreads, smem_x2<R, N, x_plain_lines<R, N, R2>()>(), st>>>(src, f.spec, tw, nrows, f.ncell, f.kx, f.kxp, RowBlobs{}, nullptr); return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  k_xfwd<R><<<dim3(xblocks, 3), kThreads, smem_x<R>(f.nx), st>>>(src, f.spec, f.px, nrows, f.ncell, f.kx, f.kxp);
}

template <typename R>
void fft_y(const FftCtx<R>& f, bool inverse, cudaStream_t st) {
  constexpr int NL = seg_lines<R>();
  const int kxt = (f.kx + NL - 1) / NL;
  const cplx_t<R>* tw = (const cplx_t<R>*)f.py.tw;
  const dim3 grid(kxt, f.nz, 3);
  switch (f.ny) {
#define ICM_CASE(N, R1, R2)                                                                                   \
  case N:                                                                                                     \
    if (inverse)                                                                                              \
      k_ypass2<R, N, R1, R2, true><<<dim3(kxt, (f.nz + y_planes<R, N, R2>() - 1) / y_planes<R, N, R2>(), 3), kThreads, smem_y2<R, N, R2>(), st>>>(f.spec, tw, f.nz, f.kx, f.kxp, nullptr);  \
    else                                                                                                      \
      k_ypass2<R, N, R1, R2, false><<<dim3(kxt, (f.nz + y_planes<R, N, R2>() - 1) / y_planes<R, N, R2>(), 3), kThreads, smem_y2<R, N, R2>(), st>>>(f.spec, tw, f.nz, f.kx, f.kxp, nullptr); \
    return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  if (inverse)
    k_ypass<R, true><<<dim3(kxt, f.nz, 3), kThreads, smem_y<R>(f.ny), st>>>(f.spec, f.py, f.nz, f.kx, f.kxp);
  else
    k_ypass<R, false><<<dim3(kxt, f.nz, 3), kThreads, smem_y<R>(f.ny), st>>>(f.spec, f.py, f.nz, f.kx, f.kxp);
}

template <typename R>
void fft_z_symbol(const FftCtx<R>& f, double a, double b, const double* k0sum, double k0scale, cudaStream_t st) {
  constexpr int NL = seg_lines<R>();
  const int kxt = (f.kx + NL - 1) / NL;
  SymParams<R> sp;
  sp.a = (R)a;
  sp.b = (R)b;
  sp.inv_ntot = (R)(1.0 / (double)f.ncell);
  sp.mean_scale = a > 0.0 ? (R)(1.0 / (a * (double)f.ncell)) : R(0);
  sp.dx = f.dx; sp.ddx = f.ddx;
  sp.dy = f.dy; sp.ddy = f.ddy;
  sp.dz = f.dz; sp.ddz = f.ddz;
  sp.k0sum = k0sum;
  sp.k0mul = k0scale / (double)f.ncell;
  const cplx_t<R>* tw = (const cplx_t<R>*)f.pz.tw;
  const int kxz = (f.kx + kZLines - 1) / kZLines;
  if (f.zmap != nullptr && f.nz <= 256) {
    const int nsm = device_sms();
    const int ntiles = kxz * f.ny;
    const int grid = ntiles < 2 * nsm ? ntiles : 2 * nsm;
    const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(f.zmap);
    switch (f.nz) {
#define ICM_CASE(N, R1, R2)                                                                                            \
  case N:                                                                                                              \
    if (N <= 256) {                                                                                                    \
      if (f.zalt)                                                                                                      \
        launch_ztma<R, N, zalt_r1<N, R1>(), N / zalt_r1<N, R1>(), false>(grid, map, f.spec, tw, f, kxz, sp, nullptr, 1, st); \
      else                                                                                                             \
        launch_ztma<R, N, R1, R2, false>(grid, map, f.spec, tw, f, kxz, sp, nullptr, 1, st);                         \
      return;                                                                                                          \
    }                                                                                                                  \
    break;
      ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
      default: break;
    }
  }
  switch (f.nz) {
#define ICM_CASE(N, R1, R2)                                                                                     \
  case N:                                                                                                       \
    if (f.zalt)                                                                                                 \
      launch_zplain<R, N, zalt_r1<N, R1>(), N / zalt_r1<N, R1>()>(dim3(kxz, f.ny), f.spec, tw, f, sp, nullptr, st); \
    else                                                                                                        \
      launch_zplain<R, N, R1, R2>(dim3(kxz, f.ny), f.spec, tw, f, sp, nullptr, st);                            \
    return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  k_zsym<R><<<dim3(kxt, f.ny), kThreads, smem_z<R>(f.nz), st>>>(f.spec, f.pz, f.ny, f.kx, f.kxp, sp);
}

template <typename R>
void fft_x_inverse(const FftCtx<R>& f, R* dst, R* dst2, int mode, cudaStream_t st) {
  const int nrows = f.ny * f.nz;
  const int xblocks = (nrows + 2 * kXLines - 1) / (2 * kXLines);
  const cplx_t<R>* tw = (const cplx_t<R>*)f.px.tw;
  switch (f.nx) {
#define ICM_CASE(N, R1, R2) \
  case N:                                                                                                              \
    if (mode == OUT_STORE)                                                                                             \
      k_xinv2<R, N, R1, R2, OUT_STORE, 0><<<dim3(xgrid<R, N, R2>(nrows), 3), kThreads, smem_x2<R, N, x_plain_lines<R, N, R2>()>(), st>>>(f.spec, dst, dst2, tw, nrows, f.ncell, f.kxp, RowBlobs{}, nullptr); \
    else                                                                                                               \
      k_xinv2<R, N, R1, R2, OUT_ADD_AND_STORE2, 0><<<dim3((nrows + 2 * kXLines - 1) / (2 * kXLines), 3), kThreads, smem_x2<R, N, kXLines>(), st>>>(f.spec, dst, dst2, tw, nrows, f.ncell, f.kxp, RowBlobs{}, nullptr); \
    return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  k_xinv<R><<<dim3(xblocks, 3), kThreads, smem_x<R>(f.nx), st>>>(f.spec, dst, dst2, mode, f.px, nrows, f.ncell,
                                                                 f.kxp);
}

#if ICM_SHARD(0)
bool fft_has_blob_passes(int nx) {
  int r1 = 0, r2 = 0;
  return fft_split(nx, r1, r2);
}

bool fft_has_group_passes(int nx, int ny, int nz) {
  int r1 = 0, r2 = 0;
  return fft_split(nx, r1, r2) && fft_split(ny, r1, r2) && fft_split(nz, r1, r2);
}
#endif

template <typename R>
void fft_x_forward_blobs(const FftCtx<R>& f, const R* src, const RowBlobs& rb, cudaStream_t st) {
  const int nrows = f.ny * f.nz;
  const int xblocks = (nrows + 2 * kXLines - 1) / (2 * kXLines);
  const cplx_t<R>* tw = (const cplx_t<R>*)f.px.tw;
  switch (f.nx) {
#define ICM_CASE(N, R1, R2) \
  case N: k_xfwd2<R, N, R1, R2, true><<<dim3(xblocks, 3), kThreads, smem_x2b<R, N, kStageF>(), st>>>(src, f.spec, tw, nrows, f.ncell, f.kx, f.kxp, rb, nullptr); return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  record_error(ICM_EINVAL, "x pass with blob work requested for a side without register FFT kernels");
}

#if ICM_SHARD(0)
bool fft_has_xy_passes(int precision, int nx, int ny) {
  if (precision != 32 || nx != ny) return false;
  int bit = 0;
#define ICM_CASE(N, R1, R2) \
  if (nx == N) return (g_xy_sides >> bit) & 1; \
  ++bit;
  ICM_XY_SIDES(ICM_CASE)
#undef ICM_CASE
  return false;
}
#endif

template <typename R>
void fft_xy_forward(const FftCtx<R>& f, const R* src, const RowBlobs* rb, cudaStream_t st) {
  if constexpr (sizeof(R) != 4) {
    record_error(ICM_EINVAL, "fused x-y pass in FP64");
  } else {
  if (!fft_has_xy_passes(32, f.nx, f.ny)) {
    record_error(ICM_EINVAL, "fused x-y pass on an unsupported grid");
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  const float* s32 = reinterpret_cast<const float*>(src);
  cplx_t<float>* sp = reinterpret_cast<cplx_t<float>*>(f.spec);
  const cplx_t<float>* tw = reinterpret_cast<const cplx_t<float>*>(f.px.tw);
  const RowBlobs none{};
  switch (f.nx) {
#define ICM_CASE(N, R1, R2)                                                                                          \
  case N:                                                                                                            \
    cfg.gridDim = dim3(N / kRowBlock, f.nz, 3);                                                                      \
    cfg.dynamicSmemBytes = smem_xyf<N>();                                                                            \
    at.val.clusterDim.x = N / kRowBlock;                                                                             \
    if (rb)                                                                                                          \
      cudaLaunchKernelEx(&cfg, k_xyf<N, R1, R2, true>, s32, sp, tw, f.nz, f.ncell, f.kxp, *rb);                      \
    else                                                                                                             \
      cudaLaunchKernelEx(&cfg, k_xyf<N, R1, R2, false>, s32, sp, tw, f.nz, f.ncell, f.kxp, none);                    \
    return;
    ICM_XY_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  }
}

template <typename R>
void fft_x_inverse_blobs(const FftCtx<R>& f, R* dst, int mode, const RowBlobs& rb, cudaStream_t st) {
  const int nrows = f.ny * f.nz;
  const int xblocks = (nrows + 2 * kXLines - 1) / (2 * kXLines);
  const cplx_t<R>* tw = (const cplx_t<R>*)f.px.tw;
  const dim3 grid(xblocks, 3);
  switch (f.nx) {
#define ICM_CASE(N, R1, R2)                                                                                              \
  case N:                                                                                                                \
    if (mode == OUT_STORE)                                                                                               \
      k_xinv2<R, N, R1, R2, OUT_STORE, 1><<<grid, kThreads, smem_x2b<R, N, xi2_stage<R, N, OUT_STORE>()>(), st>>>(f.spec, dst, nullptr, tw, nrows, f.ncell, f.kxp, rb, nullptr); \
    else if (mode == OUT_NONE)                                                                                           \
      k_xinv2<R, N, R1, R2, OUT_NONE, 1><<<grid, kThreads, smem_x2b<R, N, xi2_stage<R, N, OUT_NONE>()>(), st>>>(f.spec, dst, nullptr, tw, nrows, f.ncell, f.kxp, rb, nullptr); \
    else                                                                                                                 \
      k_xinv2<R, N, R1, R2, OUT_ADD, 2><<<grid, kThreads, smem_x2b<R, N, xi2_stage<R, N, OUT_ADD>()>(), st>>>(f.spec, dst, nullptr, tw, nrows, f.ncell, f.kxp, rb, nullptr); \
    return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  record_error(ICM_EINVAL, "x pass with blob work requested for a side without register FFT kernels");
}

template <typename R>
void spectral_solve(const FftCtx<R>& f, const R* src, R* dst, R* dst2, int mode, double a, double b,
                    const double* k0sum, double k0scale, cudaStream_t st) {
  fft_x_forward<R>(f, src, st);
  fft_y<R>(f, false, st);
  fft_z_symbol<R>(f, a, b, k0sum, k0scale, st);
  fft_y<R>(f, true, st);
  fft_x_inverse<R>(f, dst, dst2, mode, st);
}

// Group solve: the five passes of spectral_solve, each one launch over G replicas of
// the same grid (register sides only; the plain z pass).  In the x passes blockIdx.y
// is 3 x replica + component, in the y pass blockIdx.z, in the z pass blockIdx.z is
// the replica; the pointers and symbol constants come from the table.
template <typename R>
void fft_x_forward_group(const FftCtx<R>& f, const RepFft* reps, int G, cudaStream_t st, bool blobs) {
  const int nrows = f.ny * f.nz;
  const int xblocks = (nrows + 2 * kXLines - 1) / (2 * kXLines);
  const cplx_t<R>* tw = (const cplx_t<R>*)f.px.tw;
  switch (f.nx) {
#define ICM_CASE(N, R1, R2) \
  case N:                                                                                                              \
    if (blobs)                                                                                                         \
      k_xfwd2<R, N, R1, R2, true, true><<<dim3(xblocks, 3 * G), kThreads, smem_x2b<R, N, kStageF>(), st>>>(nullptr, nullptr, tw, nrows, f.ncell, f.kx, f.kxp, RowBlobs{}, reps); \
    else                                                                                                               \
      k_xfwd2<R, N, R1, R2, false><<<dim3(xgrid<R, N, R2>(nrows), 3 * G), kThreads, smem_x2<R, N, x_plain_lines<R, N, R2>()>(), st>>>(nullptr, nullptr, tw, nrows, f.ncell, f.kx, f.kxp, RowBlobs{}, reps); \
    return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  record_error(ICM_EINVAL, "group solve on a side without register FFT kernels");
}

template <typename R>
void fft_yz_group(const FftCtx<R>& f, const RepFft* reps, int G, int which, cudaStream_t st, const void* gzmap) {
  const cplx_t<R>* twy = (const cplx_t<R>*)f.py.tw;
  const cplx_t<R>* twz = (const cplx_t<R>*)f.pz.tw;
  constexpr int NL = seg_lines<R>();
  const int kxt = (f.kx + NL - 1) / NL;
  const int kxz = (f.kx + kZLines - 1) / kZLines;
  if (which == 1) {   // z FFT, symbol, inverse z FFT
    SymParams<R> sp;
    sp.a = R(0);
    sp.b = R(0);
    sp.inv_ntot = (R)(1.0 / (double)f.ncell);
    sp.mean_scale = R(0);   // per replica, from the table
    sp.dx = f.dx; sp.ddx = f.ddx;
    sp.dy = f.dy; sp.ddy = f.ddy;
    sp.dz = f.dz; sp.ddz = f.ddz;
    sp.k0sum = nullptr;
    sp.k0mul = 0.0;
    if (gzmap != nullptr && f.nz <= 256) {
      const int grid = std::min(kxz * f.ny * G, 2 * device_sms());
      const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(gzmap);
      switch (f.nz) {
#define ICM_CASE(N, R1, R2)                                                                                            \
  case N:                                                                                                              \
    if (N <= 256) {                                                                                                    \
      if (f.zalt)                                                                                                      \
        launch_ztma<R, N, zalt_r1<N, R1>(), N / zalt_r1<N, R1>(), true>(grid, map, nullptr, twz, f, kxz, sp, reps, G, st); \
      else                                                                                                             \
        launch_ztma<R, N, R1, R2, true>(grid, map, nullptr, twz, f, kxz, sp, reps, G, st);                           \
      return;                                                                                                          \
    }                                                                                                                  \
    break;
        ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
        default: break;
      }
    }
    switch (f.nz) {
#define ICM_CASE(N, R1, R2)                                                                                     \
  case N:                                                                                                       \
    if (f.zalt)                                                                                                 \
      launch_zplain<R, N, zalt_r1<N, R1>(), N / zalt_r1<N, R1>()>(dim3(kxz, f.ny, G), nullptr, twz, f, sp, reps, st); \
    else                                                                                                        \
      launch_zplain<R, N, R1, R2>(dim3(kxz, f.ny, G), nullptr, twz, f, sp, reps, st);                          \
    return;
      ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
      default: break;
    }
  } else {            // y FFT: which 0 forward, 2 inverse
    switch (f.ny) {
#define ICM_CASE(N, R1, R2)                                                                                             \
  case N:                                                                                                               \
    if (which == 2)                                                                                                     \
      k_ypass2<R, N, R1, R2, true><<<dim3(kxt, (f.nz + y_planes<R, N, R2>() - 1) / y_planes<R, N, R2>(), 3 * G), kThreads, smem_y2<R, N, R2>(), st>>>(nullptr, twy, f.nz, f.kx, f.kxp, reps); \
    else                                                                                                                \
      k_ypass2<R, N, R1, R2, false><<<dim3(kxt, (f.nz + y_planes<R, N, R2>() - 1) / y_planes<R, N, R2>(), 3 * G), kThreads, smem_y2<R, N, R2>(), st>>>(nullptr, twy, f.nz, f.kx, f.kxp, reps); \
    return;
      ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
      default: break;
    }
  }
  record_error(ICM_EINVAL, "group solve on a side without register FFT kernels");
}

template <typename R>
void fft_x_inverse_group(const FftCtx<R>& f, const RepFft* reps, int G, int mode, cudaStream_t st, bool gathers) {
  const int nrows = f.ny * f.nz;
  const int xblocks = (nrows + 2 * kXLines - 1) / (2 * kXLines);
  const cplx_t<R>* tw = (const cplx_t<R>*)f.px.tw;
  switch (f.nx) {
#define ICM_CASE(N, R1, R2)                                                                                             \
  case N:                                                                                                               \
    if (gathers && mode == OUT_STORE)                                                                                   \
      k_xinv2<R, N, R1, R2, OUT_STORE, 1, true><<<dim3(xblocks, 3 * G), kThreads, smem_x2b<R, N, xi2_stage<R, N, OUT_STORE>()>(), st>>>(nullptr, nullptr, nullptr, tw, nrows, f.ncell, f.kxp, RowBlobs{}, reps); \
    else if (gathers && mode == OUT_NONE)                                                                               \
      k_xinv2<R, N, R1, R2, OUT_NONE, 1, true><<<dim3(xblocks, 3 * G), kThreads, smem_x2b<R, N, xi2_stage<R, N, OUT_NONE>()>(), st>>>(nullptr, nullptr, nullptr, tw, nrows, f.ncell, f.kxp, RowBlobs{}, reps); \
    else if (gathers)                                                                                                   \
      k_xinv2<R, N, R1, R2, OUT_ADD, 2, true><<<dim3(xblocks, 3 * G), kThreads, smem_x2b<R, N, xi2_stage<R, N, OUT_ADD>()>(), st>>>(nullptr, nullptr, nullptr, tw, nrows, f.ncell, f.kxp, RowBlobs{}, reps); \
    else if (mode == OUT_STORE)                                                                                         \
      k_xinv2<R, N, R1, R2, OUT_STORE, 0><<<dim3(xgrid<R, N, R2>(nrows), 3 * G), kThreads, smem_x2<R, N, x_plain_lines<R, N, R2>()>(), st>>>(nullptr, nullptr, nullptr, tw, nrows, f.ncell, f.kxp, RowBlobs{}, reps); \
    else                                                                                                                \
      k_xinv2<R, N, R1, R2, OUT_ADD_AND_STORE2, 0><<<dim3((nrows + 2 * kXLines - 1) / (2 * kXLines), 3 * G), kThreads, smem_x2<R, N, kXLines>(), st>>>(nullptr, nullptr, nullptr, tw, nrows, f.ncell, f.kxp, RowBlobs{}, reps); \
    return;
    ICM_FFT_SIDES(ICM_CASE)
#undef ICM_CASE
    default: break;
  }
  record_error(ICM_EINVAL, "group solve on a side without register FFT kernels");
}

template <typename R>
void spectral_solve_group(const FftCtx<R>& f, const RepFft* reps, int G, int mode, cudaStream_t st,
                          const void* gzmap, bool blobs) {
  fft_x_forward_group<R>(f, reps, G, st, blobs);
  fft_yz_group<R>(f, reps, G, 0, st, nullptr);
  fft_yz_group<R>(f, reps, G, 1, st, gzmap);
  fft_yz_group<R>(f, reps, G, 2, st, nullptr);
  fft_x_inverse_group<R>(f, reps, G, mode, st, blobs);
}

#if ICM_SHARD(0)
// Failure-path check of the bounded wait (no GPU fault): one thread arms an mbarrier
// for 16 bytes of a transaction that is never issued, so its phase cannot complete;
// the bounded wait gives up after limit_ns and raises the timeout bit, exactly as the
// TMA z pass does when a copy does not land.  No copy is in flight when it returns.
__global__ void k_wait_timeout(int* err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_expect_tx(&bar, 16);
  if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
}

void debug_wait_timeout(int* err, long long limit_ns, cudaStream_t st) {
  k_wait_timeout<<<1, 32, 0, st>>>(err, (unsigned long long)limit_ns);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The spectrum as a 4-D tensor (floats along kx, y, z, component) and the box one z
// tile of one component occupies: 2 kZLines floats x 1 x nz x 1.  Wave numbers past
// kx read as zeros.
bool make_zmap(void* map, const void* spec, int precision, int kx, int kxp, int ny, int nz, int ncomp) {
  int r1 = 0, r2 = 0;
  if (nz > 256 || !fft_split(nz, r1, r2)) return false;
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || p == nullptr) {
      cudaGetLastError();
      return false;
    }
    fn = (EncodeTiledFn)p;
  }
  const cuuint64_t es = precision == 32 ? 4 : 8;
  const cuuint64_t dims[4] = {(cuuint64_t)(2 * kx), (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)ncomp};
  const cuuint64_t strides[3] = {2 * (cuuint64_t)kxp * es, 2 * (cuuint64_t)kxp * es * ny,
                                 2 * (cuuint64_t)kxp * es * ny * nz};
  const cuuint32_t box[4] = {2 * kZLines, 1, (cuuint32_t)nz, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(reinterpret_cast<CUtensorMap*>(map),
                        precision == 32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                        const_cast<void*>(spec), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

#endif

#define ICM_INST_XF(R, KW)                                                                               \
  KW template void fft_x_forward<R>(const FftCtx<R>&, const R*, cudaStream_t);                           \
  KW template void fft_x_forward_blobs<R>(const FftCtx<R>&, const R*, const RowBlobs&, cudaStream_t);    \
  KW template void fft_x_forward_group<R>(const FftCtx<R>&, const RepFft*, int, cudaStream_t, bool);      \
  KW template void fft_xy_forward<R>(const FftCtx<R>&, const R*, const RowBlobs*, cudaStream_t);         \
  KW template void fft_prepare_xf<R>();
#define ICM_INST_XI(R, KW)                                                                               \
  KW template void fft_x_inverse<R>(const FftCtx<R>&, R*, R*, int, cudaStream_t);                        \
  KW template void fft_x_inverse_blobs<R>(const FftCtx<R>&, R*, int, const RowBlobs&, cudaStream_t);     \
  KW template void fft_x_inverse_group<R>(const FftCtx<R>&, const RepFft*, int, int, cudaStream_t, bool); \
  KW template void fft_prepare_xi<R>();
#define ICM_INST_YZ(R, KW)                                                                               \
  KW template void fft_y<R>(const FftCtx<R>&, bool, cudaStream_t);                                       \
  KW template void fft_z_symbol<R>(const FftCtx<R>&, double, double, const double*, double, cudaStream_t); \
  KW template void fft_yz_group<R>(const FftCtx<R>&, const RepFft*, int, int, cudaStream_t, const void*); \
  KW template void fft_prepare_yz<R>();
#define ICM_NONE
#if ICM_SHARD(0)
ICM_INST_XF(float, ICM_NONE)
#else
ICM_INST_XF(float, extern)
#endif
#if ICM_SHARD(1)
ICM_INST_YZ(float, ICM_NONE)
#else
ICM_INST_YZ(float, extern)
#endif
#if ICM_SHARD(2)
ICM_INST_XI(float, ICM_NONE)
#else
ICM_INST_XI(float, extern)
#endif
#if ICM_SHARD(3)
ICM_INST_XF(double, ICM_NONE)
#else
ICM_INST_XF(double, extern)
#endif
#if ICM_SHARD(4)
ICM_INST_YZ(double, ICM_NONE)
#else
ICM_INST_YZ(double, extern)
#endif
#if ICM_SHARD(5)
ICM_INST_XI(double, ICM_NONE)
#else
ICM_INST_XI(double, extern)
#endif

#if ICM_SHARD(0)
void fft_prepare() {
  fft_prepare_xf<float>();
  fft_prepare_yz<float>();
  fft_prepare_xi<float>();
  fft_prepare_xf<double>();
  fft_prepare_yz<double>();
  fft_prepare_xi<double>();
}

template void spectral_solve<float>(const FftCtx<float>&, const float*, float*, float*, int, double, double,
                                    const double*, double, cudaStream_t);
template void spectral_solve<double>(const FftCtx<double>&, const double*, double*, double*, int, double, double,
                                     const double*, double, cudaStream_t);
template void spectral_solve_group<float>(const FftCtx<float>&, const RepFft*, int, int, cudaStream_t, const void*,
                                          bool);
template void spectral_solve_group<double>(const FftCtx<double>&, const RepFft*, int, int, cudaStream_t,
                                           const void*, bool);
#endif
#undef ICM_NONE
#undef ICM_INST_XF
#undef ICM_INST_XI
#undef ICM_INST_YZ

}  // namespace icm
