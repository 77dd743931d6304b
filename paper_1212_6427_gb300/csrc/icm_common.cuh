// Device-side building blocks shared by the ICM kernels (sm_103a).
//
// Complex helpers, the Philox4x32-10 generator (Salmon et al., SC'11), the
// Box-Muller transform, and the Peskin 3-/4-point kernel functions
// (arXiv:1212.6427, Sec. III.A.1, Eq. JS_invariance).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace icm {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };
template <typename R> using cplx_t = typename Cplx<R>::T;

__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// multiply by -i and +i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return mk(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C cmul_pi(C a) { return mk(-a.y, a.x); }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Philox4x32-10.  Round: words 0 and 2 are multiplied (full 64-bit products) by
// two constants; the high halves are xored with words 1, 3 and the key; the key
// is bumped by two Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    // one widening 32 x 32 -> 64-bit multiply per word gives both halves
    const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// The ten round keys of one key (round r uses the key bumped r times), formed once so
// that a kernel drawing many numbers reads them as constants instead of bumping the
// key in every call.
struct PhiloxRoundKeys { uint32_t k0[10], k1[10]; };
inline PhiloxRoundKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxRoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return rk;
}
__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, const PhiloxRoundKeys& rk) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = u32x4{hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0};
  }
  return c;
}

// Box-Muller: two 32-bit words -> two unit normals (cos branch, sin branch).
// u = (x + 1/2) 2^-32 in (0, 1).
template <typename R> struct BoxMuller;
template <> struct BoxMuller<double> {
  __device__ __forceinline__ static void apply(uint32_t a, uint32_t b, double& z0, double& z1) {
    const double u1 = ((double)a + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)b + 0.5) * 2.3283064365386963e-10;
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
  }
};
template <> struct BoxMuller<float> {
  __device__ __forceinline__ static void apply(uint32_t a, uint32_t b, float& z0, float& z1) {
    // u = (x + 1/2) 2^-32 with one rounding: exact for x < 2^23 (u < 2^-9, the tail
    // of the normal), relative error <= 2^-24 above
    const float u1 = fmaf(__uint2float_rn(a), 2.3283064365386963e-10f, 1.16415321826934814e-10f);
    const float u2 = fmaf(__uint2float_rn(b), 2.3283064365386963e-10f, 1.16415321826934814e-10f);
    // -2 ln u1 = -2 ln(2) log2(u1); the hardware log2 and reciprocal square root are
    // accurate to ~2^-22 relative, far inside the FP32 path's tolerance.  u1 may round
    // to 1, where the radius is 0: the floor keeps x * rsqrt(x) finite.
    const float x = fmaxf(-1.38629436111989061f * __log2f(u1), 1e-30f);
    const float rad = x * rsqrtf(x);
    float s, c;
    __sincosf(6.28318530717958648f * u2, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
  }
};

// The key as two words (the round keys formed in every call).
struct PhiloxKey { uint32_t k0, k1; };
__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, PhiloxKey k) { return philox4x32_10(c, k.k0, k.k1); }

// The 6 stress normals of one cell and step: (xx, yy, zz, xy, xz, yz).  Counters
// (cell, step, call, 0), key (seed_lo, seed_hi): call 0 of the cell gives xx, yy, zz,
// xy; call 1 serves two z planes: at the cell of plane 2m its words 0-1 give xz, yz of
// that cell, words 2-3 those of the cell above it (plane 2m + 1).  `odd`: the cell's
// plane is odd (its call 1 is the one at cell - plane).  KEYS: PhiloxKey or
// PhiloxRoundKeys.
template <typename R, typename KEYS>
__device__ __forceinline__ void cell_normals(uint32_t cell, uint32_t plane, bool odd, uint32_t step, const KEYS& key,
                                             R z[6]) {
  const u32x4 a = philox4x32_10(u32x4{cell, step, 0u, 0u}, key);
  const u32x4 b = philox4x32_10(u32x4{odd ? cell - plane : cell, step, 1u, 0u}, key);
  BoxMuller<R>::apply(a.x, a.y, z[0], z[1]);
  BoxMuller<R>::apply(a.z, a.w, z[2], z[3]);
  BoxMuller<R>::apply(odd ? b.z : b.x, odd ? b.w : b.y, z[4], z[5]);
}

// ---------------------------------------------------------------------------
// Peskin kernel functions of r in grid units.
// 3-point: (1 + sqrt(1 - 3 r^2))/3 for |r| <= 1/2, (5 - 3|r| - sqrt(1 - 3(1-|r|)^2))/6
//          for 1/2 <= |r| <= 3/2.  4-point: (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2))/8 for
//          |r| <= 1, (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2))/8 for 1 <= |r| <= 2.
// ---------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ R rsqrt0(R x) { return sqrt(x > R(0) ? x : R(0)); }

template <typename R, int K> struct Peskin;
template <typename R> struct Peskin<R, 3> {
  static constexpr int W = 3;
  __device__ __forceinline__ static R phi(R r) {
    r = fabs(r);
    if (r <= R(0.5)) return (R(1) + rsqrt0<R>(R(1) - R(3) * r * r)) / R(3);
    if (r <= R(1.5)) {
      const R t = R(1) - r;
      return (R(5) - R(3) * r - rsqrt0<R>(R(1) - R(3) * t * t)) / R(6);
    }
    return R(0);
  }
  // derivative: -r/sqrt(1-3r^2) inside, sign(r)(-3 - 3t/sqrt(1-3t^2))/6, t = 1-|r|, outside
  __device__ __forceinline__ static R dphi(R r) {
    const R a = fabs(r);
    if (a <= R(0.5)) return -r / sqrt(R(1) - R(3) * r * r);
    if (a <= R(1.5)) {
      const R t = R(1) - a;
      const R d = (R(-3) - R(3) * t / sqrt(R(1) - R(3) * t * t)) / R(6);   // d phi / d|r|
      return r < R(0) ? -d : d;
    }
    return R(0);
  }
  // first node of the support: round-half-up(s) - 1
  __device__ __forceinline__ static long long first(double s) { return (long long)floor(s + 0.5) - 1; }
  // the cell that fixes the support (its node 'first' + 1), as a double: round-half-up(s)
  __device__ __forceinline__ static double anchor(double s) { return floor(s + 0.5); }
};
template <typename R> struct Peskin<R, 4> {
  static constexpr int W = 4;
  __device__ __forceinline__ static R phi(R r) {
    r = fabs(r);
    if (r <= R(1)) return (R(3) - R(2) * r + rsqrt0<R>(R(1) + R(4) * r - R(4) * r * r)) / R(8);
    if (r <= R(2)) return (R(5) - R(2) * r - rsqrt0<R>(R(-7) + R(12) * r - R(4) * r * r)) / R(8);
    return R(0);
  }
  // derivative: sign(r)(-2 + (2-4|r|)/sqrt(1+4|r|-4r^2))/8 inside,
  // sign(r)(-2 - (6-4|r|)/sqrt(-7+12|r|-4r^2))/8 outside
  __device__ __forceinline__ static R dphi(R r) {
    const R a = fabs(r);
    R d;   // d phi / d|r|
    if (a <= R(1))
      d = (R(-2) + (R(2) - R(4) * a) / sqrt(R(1) + R(4) * a - R(4) * a * a)) / R(8);
    else if (a <= R(2))
      d = (R(-2) - (R(6) - R(4) * a) / sqrt(R(-7) + R(12) * a - R(4) * a * a)) / R(8);
    else
      return R(0);
    return r < R(0) ? -d : d;
  }
  __device__ __forceinline__ static long long first(double s) { return (long long)floor(s) - 1; }
  __device__ __forceinline__ static double anchor(double s) { return floor(s); }
};

// Status bits the device raises (read back by icm_sync).
enum : int { DEV_ERR_CFL = 1, DEV_ERR_NONFINITE = 2, DEV_ERR_TIMEOUT = 4, DEV_ERR_INDEX = 8 };

// Index checks of the checked build (compiled with -DICM_INDEX_CHECKS=1, the library
// libicm_checked.so): true when 0 <= i < n; otherwise the check raises DEV_ERR_INDEX in
// *err (if err is set) and returns false, and the caller skips the access.  It never
// traps.  In the ordinary build it is always true and compiles away.
#ifndef ICM_INDEX_CHECKS
#define ICM_INDEX_CHECKS 0
#endif
__device__ __forceinline__ bool index_ok(long long i, long long n, int* err) {
#if ICM_INDEX_CHECKS
  if (i >= 0 && i < n) return true;
  if (err != nullptr) atomicOr(err, DEV_ERR_INDEX);
  return false;
#else
  (void)i;
  (void)n;
  (void)err;
  return true;
#endif
}

}  // namespace icm
