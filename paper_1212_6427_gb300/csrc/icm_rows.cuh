// Blob work done inside the x passes of the FFT, one row block at a time.
//
// An x-pass block owns 32 consecutive rows (y + Ny z) of one velocity component.
// Blobs are binned by the row blocks their extended support (w + 2 nodes per axis,
// union over the three staggered components) touches, so a block finds the blobs
// it must serve in its bin:
//   * spreading (Sec. III.A.1, (S F)_k = dV_f^-1 sum_i phi(q_i - r_k) F_i): the
//     block adds the blobs' contributions to its rows in shared memory before its
//     transform, instead of a zeroed field, a scatter kernel and a field read;
//   * interpolation ((J v)_i = sum_k phi(q_i - r_k) v_k) and its Laplacian form
//     (J L v): the block adds the part of each blob's sum that lies in its rows to
//     an FP64 accumulator, instead of writing the field and gathering it again.
// The bin builder evaluates every blob's 1-D kernel weights once per step (FP64
// anchor, R weights) into a BlobStencil record; a (blob, row block, component) task
// in an x pass only loads the record of its component and multiplies.
#pragma once

#include "icm_internal.h"

namespace icm {
namespace {

constexpr int kRowBlock = 32;   // rows per x-pass block (two rows per complex line)

// Anchor cell of a support: node 'first' + 1, where first = round-half-up(s) - 1
// (3-point) or floor(s) - 1 (4-point), s = q/h - offset.
__device__ __forceinline__ double anchor_of(double s, int kernel) { return kernel == 3 ? floor(s + 0.5) : floor(s); }

__device__ __forceinline__ int wrap_i(int i, int n) {
  const int m = i % n;
  return m < 0 ? m + n : m;
}

// Per blob and component c: first node (wrapped) along x, y, z, and the w <= 4
// weights along each axis (entries past w are zero).  16-byte aligned rows so that
// a task loads its component with vector loads.
template <typename R>
struct __align__(16) BlobStencil {
  int first[3][4];    // [component][axis], entry 3 unused
  R w[3][3][4];       // [component][axis][node]
};

static_assert(sizeof(BlobStencil<double>) <= kStencilBytes && sizeof(BlobStencil<float>) <= kStencilBytes,
              "stencil record size");

// First and last node of the extended support along y and z, unwrapped (the bins
// need the union of the three components' supports).
struct BlobSpan {
  int lo[2], hi[2];
};

// The span of a blob at q and, if out is set, its stencil record.
template <typename R>
__device__ __forceinline__ BlobSpan make_stencil(BlobStencil<R>* out, const double q[3], const BlobParams& p) {
  BlobSpan sp;
  const int n[3] = {p.nx, p.ny, p.nz};
  const int K = p.kernel;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    int anc[2];
    R fr[2];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const double s = fma(q[ax], p.inv_h, o == 0 ? 0.0 : -0.5);
      const double a = anchor_of(s, K);
      anc[o] = (int)a;
      fr[o] = (R)(s - a);
    }
    if (ax > 0) {
      sp.lo[ax - 1] = min(anc[0], anc[1]) - 2;
      sp.hi[ax - 1] = max(anc[0], anc[1]) + K - 1;
    }
    if (out) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int o = c == ax ? 0 : 1;
        out->first[c][ax] = wrap_i(anc[o] - 1, n[ax]);
#pragma unroll
        for (int a = 0; a < 4; ++a)
          out->w[c][ax][a] = a >= K ? R(0)
                                    : (K == 3 ? Peskin<R, 3>::phi(fr[o] + R(1 - a)) : Peskin<R, 4>::phi(fr[o] + R(1 - a)));
      }
    }
  }
  if (out) {
    out->first[0][3] = 0;
    out->first[1][3] = 0;
    out->first[2][3] = 0;
  }
  return sp;
}

// The wrapped segments of the unwrapped node range [lo, hi] on a side of n nodes, in
// ascending order: at most two.
__device__ __forceinline__ int wrapped_segments(int lo, int hi, int n, int seg[2][2]) {
  if (hi - lo + 1 >= n) {
    seg[0][0] = 0;
    seg[0][1] = n - 1;
    return 1;
  }
  const int a = wrap_i(lo, n), b = wrap_i(hi, n);
  if (a <= b) {
    seg[0][0] = a;
    seg[0][1] = b;
    return 1;
  }
  seg[0][0] = 0;
  seg[0][1] = b;
  seg[1][0] = a;
  seg[1][1] = n - 1;
  return 2;
}

// Calls f(b) once for every row block that the extended support touches.  Rows
// y + Ny z are visited in ascending order (wrapped z, then wrapped y), so the block
// index never decreases and a repeat can only be the last block seen.
template <typename F>
__device__ __forceinline__ void for_each_row_block(const BlobSpan& sp, const BlobParams& p, F f) {
  int zs[2][2], ys[2][2];
  const int nzs = wrapped_segments(sp.lo[1], sp.hi[1], p.nz, zs);
  const int nys = wrapped_segments(sp.lo[0], sp.hi[0], p.ny, ys);
  int last = -1;
  for (int i = 0; i < nzs; ++i)
    for (int z = zs[i][0]; z <= zs[i][1]; ++z)
      for (int j = 0; j < nys; ++j) {
        const int b0 = (ys[j][0] + p.ny * z) / kRowBlock, b1 = (ys[j][1] + p.ny * z) / kRowBlock;
        for (int b = max(b0, last + 1); b <= b1; ++b) f(b);
        last = max(last, b1);
      }
}

__device__ __forceinline__ int wrap_add1(int a, int b, int n) {
  const int t = a + b;
  return t >= n ? t - n : t;
}

// The stencil of one component, loaded from the record.
template <typename R, int K>
struct CompStencil {
  int fx, fy, fz;
  R wx[K], wy[K], wz[K];
};

template <typename R, int K>
__device__ __forceinline__ void load_comp(CompStencil<R, K>& S, const BlobStencil<R>* rec, int comp) {
  const int4 f = *reinterpret_cast<const int4*>(rec->first[comp]);
  S.fx = f.x;
  S.fy = f.y;
  S.fz = f.z;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    S.wx[a] = rec->w[comp][0][a];
    S.wy[a] = rec->w[comp][1][a];
    S.wz[a] = rec->w[comp][2][a];
  }
}

// Rows of the block are held as complex lines: line l = rows 2l (real part) and
// 2l + 1 (imaginary part); position x of line l at complex index line(l, x).
template <typename LINE>
__device__ __forceinline__ int lane_of(int r, int x, LINE line) { return 2 * line(r >> 1, x) + (r & 1); }

// Add one blob's spread contribution (component comp, amp = vec_comp / dV_f) to the
// rows [row0, row0 + 32) held in `rows`.
template <typename R, int K, int N, typename LINE>
__device__ __forceinline__ void spread_task(R* rows, int row0, const CompStencil<R, K>& S, R amp, const BlobParams& p,
                                            LINE line) {
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const int zrow = p.ny * wrap_add1(S.fz, c, p.nz) - row0;
    if (zrow + p.ny <= 0 || zrow >= kRowBlock) continue;   // the whole plane is outside
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const int r = zrow + wrap_add1(S.fy, b, p.ny);
      if (r < 0 || r >= kRowBlock) continue;
      const R wyz = S.wy[b] * S.wz[c] * amp;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        const int x = wrap_add1(S.fx, a, N);
        if (index_ok(x, N, p.err)) atomicAdd(&rows[lane_of(r, x, line)], S.wx[a] * wyz);
      }
    }
  }
}

// Part of (J field)_comp of one blob that lies in the rows held in `rows`.
template <typename R, int K, int N, typename LINE>
__device__ __forceinline__ R gather_task(const R* rows, int row0, const CompStencil<R, K>& S, const BlobParams& p,
                                         LINE line) {
  R acc = R(0);
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const int zrow = p.ny * wrap_add1(S.fz, c, p.nz) - row0;
    if (zrow + p.ny <= 0 || zrow >= kRowBlock) continue;
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const int r = zrow + wrap_add1(S.fy, b, p.ny);
      if (r < 0 || r >= kRowBlock) continue;
      R t = R(0);
#pragma unroll
      for (int a = 0; a < K; ++a) {
        const int x = wrap_add1(S.fx, a, N);
        if (index_ok(x, N, p.err)) t += S.wx[a] * rows[lane_of(r, x, line)];
      }
      acc += S.wy[b] * S.wz[c] * t;
    }
  }
  return acc;
}

// Zero-padded K + 2 weights (one node earlier) and their second differences.
template <typename R, int K>
__device__ __forceinline__ void extend(const R w[K], R we[K + 2], R d2[K + 2]) {
#pragma unroll
  for (int a = 0; a < K + 2; ++a) {
    const R c = (a >= 1 && a <= K) ? w[a - 1] : R(0);
    const R lo = (a >= 2) ? w[a - 2] : R(0);
    const R hi = (a <= K - 1) ? w[a] : R(0);
    we[a] = c;
    d2[a] = lo - R(2) * c + hi;
  }
}

// Part of (J L field)_comp in the rows: the gather with the discrete Laplacian of the
// weights (L is symmetric), without the 1/h^2 factor.
template <typename R, int K, int N, typename LINE>
__device__ __forceinline__ R gather_lap_task(const R* rows, int row0, const CompStencil<R, K>& S, const BlobParams& p,
                                             LINE line) {
  constexpr int E = K + 2;
  R wx[E], wy[E], wz[E], dx[E], dy[E], dz[E];
  extend<R, K>(S.wx, wx, dx);
  extend<R, K>(S.wy, wy, dy);
  extend<R, K>(S.wz, wz, dz);
  const int fx = S.fx == 0 ? N - 1 : S.fx - 1;
  const int fy = S.fy == 0 ? p.ny - 1 : S.fy - 1;
  const int fz = S.fz == 0 ? p.nz - 1 : S.fz - 1;
  R acc = R(0);
#pragma unroll 1
  for (int c = 0; c < E; ++c) {
    const int zrow = p.ny * wrap_add1(fz, c, p.nz) - row0;
    if (zrow + p.ny <= 0 || zrow >= kRowBlock) continue;
#pragma unroll
    for (int b = 0; b < E; ++b) {
      const int r = zrow + wrap_add1(fy, b, p.ny);
      if (r < 0 || r >= kRowBlock) continue;
      R t0 = R(0), t1 = R(0);   // sum w_x v and sum d2_x v along the row
#pragma unroll
      for (int a = 0; a < E; ++a) {
        const int x = wrap_add1(fx, a, N);
        const R v = index_ok(x, N, p.err) ? rows[lane_of(r, x, line)] : R(0);
        t0 += wx[a] * v;
        t1 += dx[a] * v;
      }
      acc += t1 * wy[b] * wz[c] + t0 * (dy[b] * wz[c] + wy[b] * dz[c]);
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Sides with Ny a multiple of 32: a row block is 32 consecutive y of one z plane
// (z0, y0..y0+31), so a task touches at most one plane of its stencil.  The same
// sums as above, with the plane index computed instead of tested node by node.
// ---------------------------------------------------------------------------
template <typename R, int K>
__device__ __forceinline__ R pick(const R w[K], int c) {
  R v = w[0];
#pragma unroll
  for (int k = 1; k < K; ++k) v = c == k ? w[k] : v;
  return v;
}

template <typename R, int K, int N, typename LINE>
__device__ __forceinline__ void spread_plane(R* rows, int z0, int y0, const CompStencil<R, K>& S, R amp,
                                             const BlobParams& p, LINE line) {
  int c = z0 - S.fz;
  if (c < 0) c += p.nz;
  if (c >= K) return;
  const R wz = pick<R, K>(S.wz, c) * amp;
  int xo[K];
#pragma unroll
  for (int a = 0; a < K; ++a) xo[a] = lane_of(0, wrap_add1(S.fx, a, N), line);
  if (!index_ok(S.fx, N, p.err) || !index_ok(S.fy, p.ny, p.err)) return;
#pragma unroll
  for (int b = 0; b < K; ++b) {
    const int r = wrap_add1(S.fy, b, p.ny) - y0;
    if ((unsigned)r >= (unsigned)kRowBlock) continue;
    const int rb = lane_of(r, 0, line);
    const R wyz = S.wy[b] * wz;
#pragma unroll
    for (int a = 0; a < K; ++a) atomicAdd(&rows[rb + xo[a]], S.wx[a] * wyz);
  }
}

template <typename R, int K, int N, typename LINE>
__device__ __forceinline__ R gather_plane(const R* rows, int z0, int y0, const CompStencil<R, K>& S,
                                          const BlobParams& p, LINE line) {
  int c = z0 - S.fz;
  if (c < 0) c += p.nz;
  if (c >= K) return R(0);
  int xo[K];
#pragma unroll
  for (int a = 0; a < K; ++a) xo[a] = lane_of(0, wrap_add1(S.fx, a, N), line);
  if (!index_ok(S.fx, N, p.err) || !index_ok(S.fy, p.ny, p.err)) return R(0);
  R acc = R(0);
#pragma unroll
  for (int b = 0; b < K; ++b) {
    const int r = wrap_add1(S.fy, b, p.ny) - y0;
    if ((unsigned)r >= (unsigned)kRowBlock) continue;
    const int rb = lane_of(r, 0, line);
    R t = R(0);
#pragma unroll
    for (int a = 0; a < K; ++a) t += S.wx[a] * rows[rb + xo[a]];
    acc += S.wy[b] * t;
  }
  return acc * pick<R, K>(S.wz, c);
}

template <typename R, int K, int N, typename LINE>
__device__ __forceinline__ R gather_lap_plane(const R* rows, int z0, int y0, const CompStencil<R, K>& S,
                                              const BlobParams& p, LINE line) {
  constexpr int E = K + 2;
  const int fz = S.fz == 0 ? p.nz - 1 : S.fz - 1;
  int c = z0 - fz;
  if (c < 0) c += p.nz;
  if (c >= E) return R(0);
  R wx[E], wy[E], wz[E], dx[E], dy[E], dz[E];
  extend<R, K>(S.wx, wx, dx);
  extend<R, K>(S.wy, wy, dy);
  extend<R, K>(S.wz, wz, dz);
  const R wzc = pick<R, E>(wz, c), dzc = pick<R, E>(dz, c);
  const int fx = S.fx == 0 ? N - 1 : S.fx - 1;
  const int fy = S.fy == 0 ? p.ny - 1 : S.fy - 1;
  int xo[E];
#pragma unroll
  for (int a = 0; a < E; ++a) xo[a] = lane_of(0, wrap_add1(fx, a, N), line);
  if (!index_ok(fx, N, p.err) || !index_ok(fy, p.ny, p.err)) return R(0);
  R acc = R(0);
#pragma unroll
  for (int b = 0; b < E; ++b) {
    const int r = wrap_add1(fy, b, p.ny) - y0;
    if ((unsigned)r >= (unsigned)kRowBlock) continue;
    const int rb = lane_of(r, 0, line);
    R t0 = R(0), t1 = R(0);
#pragma unroll
    for (int a = 0; a < E; ++a) {
      const R v = rows[rb + xo[a]];
      t0 += wx[a] * v;
      t1 += dx[a] * v;
    }
    acc += t1 * wy[b] * wzc + t0 * (dy[b] * wzc + wy[b] * dzc);
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Staging of a block's task records in shared memory (cp.async, issued at kernel
// start so that the dependent loads bin start -> blob id -> record overlap the
// block's field or spectrum loads).
// ---------------------------------------------------------------------------
template <typename R>
struct __align__(16) StagedTask {
  int4 first;     // first nodes of the component along x, y, z
  R w[12];        // weights [axis][node]
  double vec;     // spread source of the component (FP64); unused by gathers
  int b;          // blob id
};

__device__ __forceinline__ uint32_t rows_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(rows_smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(rows_smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy the record of component comp of blob b (and its source value) into slot.
template <typename R>
__device__ __forceinline__ void stage_task(StagedTask<R>* slot, const BlobStencil<R>* rec, int b, int comp,
                                           const double* vec) {
  cp_async16(&slot->first, &rec[b].first[comp][0]);
  const char* w = reinterpret_cast<const char*>(&rec[b].w[comp][0][0]);
  char* d = reinterpret_cast<char*>(slot->w);
#pragma unroll
  for (int k = 0; k < (int)(12 * sizeof(R) / 16); ++k) cp_async16(d + 16 * k, w + 16 * k);
  if (vec != nullptr) cp_async8(&slot->vec, vec + 3 * b + comp);
  slot->b = b;
}

template <typename R, int K>
__device__ __forceinline__ void comp_from(CompStencil<R, K>& S, int4 f, const R* w) {
  S.fx = f.x;
  S.fy = f.y;
  S.fz = f.z;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    S.wx[a] = w[a];
    S.wy[a] = w[4 + a];
    S.wz[a] = w[8 + a];
  }
}

// One spread task: plane path when the block lies in one z plane, generic otherwise.
template <typename R, int N, typename LINE>
__device__ __forceinline__ void spread_one(R* rows, int row0, bool plane, int z0, int y0, int4 f, const R* w,
                                           R amp, const BlobParams& p, LINE line) {
  if (p.kernel == 3) {
    CompStencil<R, 3> S;
    comp_from<R, 3>(S, f, w);
    if (plane)
      spread_plane<R, 3, N>(rows, z0, y0, S, amp, p, line);
    else
      spread_task<R, 3, N>(rows, row0, S, amp, p, line);
  } else {
    CompStencil<R, 4> S;
    comp_from<R, 4>(S, f, w);
    if (plane)
      spread_plane<R, 4, N>(rows, z0, y0, S, amp, p, line);
    else
      spread_task<R, 4, N>(rows, row0, S, amp, p, line);
  }
}

// One gather task: the parts of J and (LAP) J L of the component in these rows.
template <typename R, int N, bool LAP, typename LINE>
__device__ __forceinline__ void gather_one(const R* rows, int row0, bool plane, int z0, int y0, int4 f,
                                           const R* w, const BlobParams& p, LINE line, R& j, R& jl) {
  jl = R(0);
  if (p.kernel == 3) {
    CompStencil<R, 3> S;
    comp_from<R, 3>(S, f, w);
    j = plane ? gather_plane<R, 3, N>(rows, z0, y0, S, p, line) : gather_task<R, 3, N>(rows, row0, S, p, line);
    if (LAP)
      jl = plane ? gather_lap_plane<R, 3, N>(rows, z0, y0, S, p, line)
                 : gather_lap_task<R, 3, N>(rows, row0, S, p, line);
  } else {
    CompStencil<R, 4> S;
    comp_from<R, 4>(S, f, w);
    j = plane ? gather_plane<R, 4, N>(rows, z0, y0, S, p, line) : gather_task<R, 4, N>(rows, row0, S, p, line);
    if (LAP)
      jl = plane ? gather_lap_plane<R, 4, N>(rows, z0, y0, S, p, line)
                 : gather_lap_task<R, 4, N>(rows, row0, S, p, line);
  }
}

}  // namespace
}  // namespace icm
