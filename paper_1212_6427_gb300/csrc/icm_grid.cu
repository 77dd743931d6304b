// Grid kernels of the ICM step (arXiv:1212.6427, Sec. III.B-C):
//   * the explicit right-hand side of Eq. provisional_step-1, one fused pass:
//       r = (rho/dt) v + (eta/2) L v + div Sigma^n - (3/2 A^n - 1/2 A^{n-1}),
//     with the stochastic stress Sigma^n = sqrt(kT eta/(dV_f dt)) (W + W^T) drawn
//     from Philox4x32-10 on the fly (never stored) and A = div(rho v v^T) in
//     centred conservative (skew-adjoint) form, Adams-Bashforth in time
//     (Eq. Adams_Bashforth).  A^n overwrites A^{n-1} in place.
//   * FP64 compensated sums of face fields (momentum bookkeeping, Sec. II).
#include <algorithm>

#include "icm_internal.h"

namespace icm {
namespace {

constexpr int TX = 32, TY = 16;     // cells per block in x and y (one thread each)
constexpr int HX = TX + 2, HY = TY + 2;
constexpr int NT = TX * TY;         // threads per block
constexpr int NHALO = 2 * HX + 2 * TY;   // ring of halo cells around the TX x TY tile

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// Periodic index for any i (a tile can be several times wider than a short side).
__device__ __forceinline__ int wrapm(int i, int n) { return ((i % n) + n) % n; }

// Shared memory of the marching block.
//  * v: a ring of four velocity planes (three components, one-cell halo in x and y).
//    At plane k the block reads slots of planes k-1, k, k+1 and writes plane k+1's slot
//    before its barrier; that slot was last read by plane k-3, long finished.
//  * z: a ring of three planes of the stress normals that neighbours read (Z_xx, Z_yy,
//    Z_xy, Z_xz, Z_yz; Z_zz is only read by its own cell).  The normals of plane k+1
//    are written before plane k's barrier and read after plane k+1's; the slot was last
//    read at plane k-2.  Each thread keeps its own cell's normals in registers.
constexpr int kRing = 4, kZRing = 3;
template <typename R>
struct RhsSmem {
  R v[kRing][3][HY][HX];
  R z[kZRing][5][HY][HX];
};

// Halo cell h (0 <= h < NHALO) of the tile as (hx, hy) in the padded plane:
// bottom row, top row, left column, right column.
__device__ __forceinline__ void halo_cell(int h, int& hx, int& hy) {
  if (h < HX) {
    hx = h;
    hy = 0;
  } else if (h < 2 * HX) {
    hx = h - HX;
    hy = HY - 1;
  } else if (h < 2 * HX + TY) {
    hx = 0;
    hy = 1 + (h - 2 * HX);
  } else {
    hx = HX - 1;
    hy = 1 + (h - 2 * HX - TY);
  }
}

// The stress normals the tile's neighbours read from its halo cells, 144 per plane:
// Z_yy of the bottom row and Z_xx of the left column (the first Box-Muller pair of
// Philox call 0), Z_xy of the top row and of the right column (the second pair of call
// 0), Z_yz of the top row and Z_xz of the right column (the first pair of call 1).  Task
// tau = 32 warp + lane of warps 0-4 draws one of them: one Philox call and one
// Box-Muller pair per lane, the counter word, word pair and branch chosen per lane, so no
// warp diverges and none does more than one call.  The corners are read by no one.
struct HaloTask {
  int hx, hy;       // position in the padded plane
  int dst;          // z ring array: 0 xx, 1 yy, 2 xy, 3 xz, 4 yz
  uint32_t call;    // Philox counter word 2
  bool hi;          // Box-Muller on words (z, w) rather than (x, y)
  bool second;      // the sine branch rather than the cosine one
};
constexpr int kHaloTasks = 3 * TX + 3 * TY;   // 144
static_assert(kHaloTasks <= NT, "one halo task per thread at most");

__device__ __forceinline__ bool halo_task(int tau, HaloTask& t) {
  if (tau < TX) {                       // bottom row: Z_yy
    t = HaloTask{1 + tau, 0, 1, 0u, false, true};
  } else if (tau < TX + TY) {           // left column: Z_xx
    t = HaloTask{0, 1 + (tau - TX), 0, 0u, false, false};
  } else if (tau < 2 * TX + TY) {       // top row: Z_xy
    t = HaloTask{1 + (tau - TX - TY), HY - 1, 2, 0u, true, true};
  } else if (tau < 3 * TX + TY) {       // top row: Z_yz
    t = HaloTask{1 + (tau - 2 * TX - TY), HY - 1, 4, 1u, false, true};
  } else if (tau < 3 * TX + 2 * TY) {   // right column: Z_xy
    t = HaloTask{HX - 1, 1 + (tau - 3 * TX - TY), 2, 0u, true, true};
  } else if (tau < kHaloTasks) {        // right column: Z_xz
    t = HaloTask{HX - 1, 1 + (tau - 3 * TX - 2 * TY), 3, 1u, false, false};
  } else {
    return false;
  }
  return true;
}

// Philox of the RHS: with RK the round keys of the kernel parameters (read as
// constants), otherwise the key bumped in every call (parameters copied from memory).
template <bool RK>
__device__ __forceinline__ u32x4 rhs_philox(u32x4 c, const GridParams& g) {
  if constexpr (RK)
    return philox4x32_10(c, g.rk);
  else
    return philox4x32_10(c, g.key0, g.key1);
}

// Halo task t at flat cell index `cell` (plane `odd` or even) into slot `slot` of the z
// ring.  Its call-1 normals (Z_xz, Z_yz) on an odd plane are words 2-3 of the call at
// the cell one plane down (`plane` cells per plane).
template <typename R, bool RK>
__device__ __forceinline__ void gen_halo(RhsSmem<R>& sm, int slot, const HaloTask& t, uint32_t cell, uint32_t plane,
                                         bool odd, const GridParams& g, uint32_t step) {
  const bool up = t.call == 1u && odd;
  const u32x4 r = rhs_philox<RK>(u32x4{up ? cell - plane : cell, step, t.call, 0u}, g);
  const bool hi = t.hi || up;
  R c, sn;
  BoxMuller<R>::apply(hi ? r.z : r.x, hi ? r.w : r.y, c, sn);
  sm.z[slot][t.dst][t.hy][t.hx] = t.second ? sn : c;
}

// The own cell's normals of plane p (flat index `cell`) into z[] (registers) and the
// five that neighbours read into slot `slot` of the z ring.  The call-1 words of an
// even plane also hold the next plane's (Z_xz, Z_yz): kept in `next` (valid set) for
// the odd plane that follows in the march; an odd plane without them draws that call
// again at the cell below.
template <typename R, bool RK>
__device__ __forceinline__ void gen_own(RhsSmem<R>& sm, int slot, R (&z)[6], uint32_t cell, int p, uint32_t plane,
                                        const GridParams& g, uint32_t step, int lx, int ly, uint32_t (&next)[2],
                                        bool& valid) {
  const u32x4 a = rhs_philox<RK>(u32x4{cell, step, 0u, 0u}, g);
  BoxMuller<R>::apply(a.x, a.y, z[0], z[1]);
  BoxMuller<R>::apply(a.z, a.w, z[2], z[3]);
  uint32_t w0, w1;
  if ((p & 1) == 0) {
    const u32x4 b = rhs_philox<RK>(u32x4{cell, step, 1u, 0u}, g);
    w0 = b.x;
    w1 = b.y;
    next[0] = b.z;
    next[1] = b.w;
    valid = true;
  } else if (valid) {
    w0 = next[0];
    w1 = next[1];
    valid = false;
  } else {
    const u32x4 b = rhs_philox<RK>(u32x4{cell - plane, step, 1u, 0u}, g);
    w0 = b.z;
    w1 = b.w;
  }
  BoxMuller<R>::apply(w0, w1, z[4], z[5]);
  sm.z[slot][0][ly][lx] = z[0];
  sm.z[slot][1][ly][lx] = z[1];
  sm.z[slot][2][ly][lx] = z[3];
  sm.z[slot][3][ly][lx] = z[4];
  sm.z[slot][4][ly][lx] = z[5];
}

// Marching block of TX x TY cells.  A block takes a contiguous range of planes: with
// g.kz > 0 the kz planes of one tile (grid = tiles x ceil(nz / kz)); with g.kz == 0 the
// blocks are persistent (about two per SM) in groups of one block per tile of a tile
// row, and the groups split all tile-row planes evenly.  A range is marched tile by
// tile; each run starts with a prologue of two planes.  Per
// plane: the global loads of the plane after next are issued first, the stress normals
// of the next plane are drawn while they are in flight, then the plane is computed from
// the thread's registers (its own column) and shared memory (its neighbours).
// One run of the marching block: planes k0 .. kend-1 of tile `tile` (tiles x-fastest).
template <typename R, bool NOISE, bool RK>
__device__ __forceinline__ void rhs_run(RhsSmem<R>& sm, const R* __restrict__ v, R* __restrict__ adv,
                                        R* __restrict__ rhs, const GridParams& g, uint32_t step, bool hist,
                                        long long tile, int k0, int kend, int tx, int ty) {
  const int tid = tx + TX * ty;
  const int ntx = (g.nx + TX - 1) / TX;
  // offsets in 32 bits: 3 ncell <= 3 x 512^3 < 2^32
  const uint32_t nc = (uint32_t)g.ncell;
  const uint32_t plane = (uint32_t)g.nx * (uint32_t)g.ny;
  // r = cc v + ce (sum of the six neighbours) + div Sigma - AB2, with cc = rho/dt - 6 ce,
  // ce = (eta/2)/h^2; the 1/2 of every face or edge average of the advection is folded
  // into its factor aq = rho/(4h)
  const R ce = (R)(0.5 * g.eta / (g.h * g.h));
  const R cc = (R)(g.rho / g.dt - 3.0 * g.eta / (g.h * g.h));
  const R aq = g.advection ? (R)(0.25 * g.rho / g.h) : R(0);
  const double s_amp = sqrt(g.kT * g.eta / (g.h * g.h * g.h * g.dt));
  const R sd = (R)(2.0 * s_amp * (1.0 / g.h)), so = (R)(1.4142135623730951 * s_amp * (1.0 / g.h));
  const int lx = tx + 1, ly = ty + 1;
  {
    const int i0 = (int)(tile % ntx) * TX, j0 = (int)(tile / ntx) * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < g.nx && j < g.ny;
    // threads past a ragged edge hold the periodic images their neighbours read
    const uint32_t own = (uint32_t)wrapm(i, g.nx) + (uint32_t)g.nx * (uint32_t)wrapm(j, g.ny);
    // the halo cell whose velocities this thread loads, if any
    int hx = 0, hy = 0;
    const bool has_halo = tid < NHALO;
    uint32_t hoff = 0;
    if (has_halo) {
      halo_cell(tid, hx, hy);
      hoff = (uint32_t)wrapm(i0 - 1 + hx, g.nx) + (uint32_t)g.nx * (uint32_t)wrapm(j0 - 1 + hy, g.ny);
    }
    // the halo stress normal this thread draws, if any
    HaloTask ht{0, 0, 0, 0u, false, false};
    const bool hnoise = NOISE && halo_task(tid, ht);
    const uint32_t ncell = hnoise ? (uint32_t)(wrapm(i0 - 1 + ht.hx, g.nx) + g.nx * wrapm(j0 - 1 + ht.hy, g.ny)) : 0u;
    auto load = [&](R (&o)[3], R (&hv)[3], int k) {
      const uint32_t zo = plane * (uint32_t)wrapi(k, g.nz);
      const uint32_t a = zo + own;
#pragma unroll
      for (int c = 0; c < 3; ++c) o[c] = v[a + c * nc];
      if (has_halo) {
        const uint32_t b = zo + hoff;
#pragma unroll
        for (int c = 0; c < 3; ++c) hv[c] = v[b + c * nc];
      }
    };
    auto put = [&](int slot, const R (&o)[3], const R (&hv)[3]) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.v[slot][c][ly][lx] = o[c];
      if (has_halo) {
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.v[slot][c][hy][hx] = hv[c];
      }
    };
    // every thread is past the previous run's last plane before its slots are reused
    __syncthreads();
    R vp[3], vc[3], vn[3], vq[3], hq[3];   // own column: planes k-1, k, k+1, k+2; halo k+2
    R zc[6], zn[6], zzp = R(0);            // own normals: plane k, plane k+1, Z_zz of k-1
    load(vp, hq, k0 - 1);
    put(0, vp, hq);
    load(vc, hq, k0);
    put(1, vc, hq);
    load(vn, hq, k0 + 1);
    uint32_t next[2] = {0u, 0u};   // call-1 words of the plane after an even one
    bool nvalid = false;
    if (NOISE) {
      // plane k0-1: only the own cell's Z_zz is read (call 0); plane k0 into slot 1
      {
        const u32x4 a = rhs_philox<RK>(u32x4{own + plane * (uint32_t)wrapi(k0 - 1, g.nz), step, 0u, 0u}, g);
        R zxy;
        BoxMuller<R>::apply(a.z, a.w, zzp, zxy);
      }
      gen_own<R, RK>(sm, 1, zn, own + plane * (uint32_t)k0, k0, plane, g, step, lx, ly, next, nvalid);
      if (hnoise) gen_halo<R, RK>(sm, 1, ht, ncell + plane * (uint32_t)k0, plane, (k0 & 1) != 0, g, step);
    }
    for (int k = k0; k < kend; ++k) {
      const int kk = k - k0;
      const int sp = kk % kRing, sc = (kk + 1) % kRing, sn = (kk + 2) % kRing;
      const int zs = (kk + 1) % kZRing, zsn = (kk + 2) % kZRing;   // normals of planes k, k+1
      put(sn, vn, hq);                                         // plane k+1
      const uint32_t o = own + plane * (uint32_t)k;
      R ao[3] = {R(0), R(0), R(0)};
      if (active && hist) {
        ao[0] = adv[o];
        ao[1] = adv[o + nc];
        ao[2] = adv[o + 2 * nc];
      }
      if (k + 1 < kend) load(vq, hq, k + 2);                  // in flight during the noise
      if (NOISE) {
#pragma unroll
        for (int c = 0; c < 6; ++c) zc[c] = zn[c];
        const int p1 = wrapi(k + 1, g.nz);
        const uint32_t pk = plane * (uint32_t)p1;
        gen_own<R, RK>(sm, zsn, zn, own + pk, p1, plane, g, step, lx, ly, next, nvalid);
        if (hnoise) gen_halo<R, RK>(sm, zsn, ht, ncell + pk, plane, (p1 & 1) != 0, g, step);
      }
      __syncthreads();
      if (active) {
        const auto P = sm.v[sp];
        const auto C = sm.v[sc];
        const auto N = sm.v[sn];
        // component x
        const R x_c = vc[0], x_xp = C[0][ly][lx + 1], x_xm = C[0][ly][lx - 1];
        const R x_yp = C[0][ly + 1][lx], x_ym = C[0][ly - 1][lx], x_zp = vn[0], x_zm = vp[0];
        const R x_xpym = C[0][ly - 1][lx + 1], x_xpzm = P[0][ly][lx + 1];
        // component y
        const R y_c = vc[1], y_xp = C[1][ly][lx + 1], y_xm = C[1][ly][lx - 1];
        const R y_yp = C[1][ly + 1][lx], y_ym = C[1][ly - 1][lx], y_zp = vn[1], y_zm = vp[1];
        const R y_ypxm = C[1][ly + 1][lx - 1], y_ypzm = P[1][ly + 1][lx];
        // component z
        const R z_c = vc[2], z_xp = C[2][ly][lx + 1], z_xm = C[2][ly][lx - 1];
        const R z_yp = C[2][ly + 1][lx], z_ym = C[2][ly - 1][lx], z_zp = vn[2], z_zm = vp[2];
        const R z_zpxm = N[2][ly][lx - 1], z_zpym = N[2][ly - 1][lx];

        // edge products ut_a ut_b at edge index e, ut_a = (v_a[e] + v_a[e-e_b])/2 and
        // ut_b = (v_b[e] + v_b[e-e_a])/2, and the squared cell-centre averages, each
        // without its factor 1/4 (in aq)
        const R exy_c = (x_c + x_ym) * (y_c + y_xm);
        const R exy_yp = (x_yp + x_c) * (y_yp + y_ypxm);
        const R exy_xp = (x_xp + x_xpym) * (y_xp + y_c);
        const R exz_c = (x_c + x_zm) * (z_c + z_xm);
        const R exz_zp = (x_zp + x_c) * (z_zp + z_zpxm);
        const R exz_xp = (x_xp + x_xpzm) * (z_xp + z_c);
        const R eyz_c = (y_c + y_zm) * (z_c + z_ym);
        const R eyz_zp = (y_zp + y_c) * (z_zp + z_zpym);
        const R eyz_yp = (y_yp + y_ypzm) * (z_yp + z_c);
        const R ubx_c = x_xp + x_c, ubx_m = x_c + x_xm;
        const R uby_c = y_yp + y_c, uby_m = y_c + y_ym;
        const R ubz_c = z_zp + z_c, ubz_m = z_c + z_zm;
        const R ax = aq * (ubx_c * ubx_c - ubx_m * ubx_m + exy_yp - exy_c + exz_zp - exz_c);
        const R ay = aq * (uby_c * uby_c - uby_m * uby_m + exy_xp - exy_c + eyz_zp - eyz_c);
        const R az = aq * (ubz_c * ubz_c - ubz_m * ubz_m + exz_xp - exz_c + eyz_yp - eyz_c);
        const R nbx = x_xp + x_xm + x_yp + x_ym + x_zp + x_zm;
        const R nby = y_xp + y_xm + y_yp + y_ym + y_zp + y_zm;
        const R nbz = z_xp + z_xm + z_yp + z_ym + z_zp + z_zm;
        R fx = R(0), fy = R(0), fz = R(0);
        if (NOISE) {
          const auto Z = sm.z[zs];   // plane k: [0] xx, [1] yy, [2] xy, [3] xz, [4] yz
          // divergence of the stress at the faces: Sigma_aa at cells, Sigma_ab on edges
          fx = sd * (zc[0] - Z[0][ly][lx - 1]) + so * (Z[2][ly + 1][lx] - zc[3]) + so * (zn[4] - zc[4]);
          fy = sd * (zc[1] - Z[1][ly - 1][lx]) + so * (Z[2][ly][lx + 1] - zc[3]) + so * (zn[5] - zc[5]);
          fz = sd * (zc[2] - zzp) + so * (Z[3][ly][lx + 1] - zc[4]) + so * (Z[4][ly + 1][lx] - zc[5]);
        }
        if (!hist) {
          ao[0] = ax;
          ao[1] = ay;
          ao[2] = az;
        }
        adv[o] = ax;
        adv[o + nc] = ay;
        adv[o + 2 * nc] = az;
        rhs[o] = cc * x_c + ce * nbx + fx - (R(1.5) * ax - R(0.5) * ao[0]);
        rhs[o + nc] = cc * y_c + ce * nby + fy - (R(1.5) * ay - R(0.5) * ao[1]);
        rhs[o + 2 * nc] = cc * z_c + ce * nbz + fz - (R(1.5) * az - R(0.5) * ao[2]);
      }
      if (NOISE) zzp = zc[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vp[c] = vc[c];
        vc[c] = vn[c];
        vn[c] = vq[c];
      }
    }
  }
}

// A block takes a contiguous range [lo, hi) of planes: with g.kz > 0 the kz planes
// w = tile * nz + k of one tile (grid = tiles x ceil(nz / kz)); with g.kz == 0 the
// blocks are persistent (whole groups of one block per tile of a tile row, as many as
// the SMs hold at once) and a group's range is of tile-row planes u = row * nz + k, its
// block xt marching tile xt of each row.  A range is marched tile by tile.
template <typename R, bool NOISE>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) k_rhs(const R* __restrict__ v, R* __restrict__ adv,
                                                                      R* __restrict__ rhs, GridParams g,
                                                                      const long long* __restrict__ step_dev,
                                                                      const int* __restrict__ hist_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RhsSmem<R>& sm = *reinterpret_cast<RhsSmem<R>*>(smem_raw);
  const int ntx = (g.nx + TX - 1) / TX, nty = (g.ny + TY - 1) / TY;
  long long lo, hi;
  int xt = 0;
  if (g.kz > 0) {
    const long long tile = blockIdx.x + (long long)ntx * blockIdx.y;
    lo = tile * g.nz + (long long)blockIdx.z * g.kz;
    hi = min(lo + g.kz, (tile + 1) * g.nz);
  } else {
    // Persistent blocks in groups of ntx, one block per tile of a tile row: the groups
    // split the tile-row planes u = (tile row) nz + k evenly, and the blocks of a group
    // march the same planes side by side, so the halo columns a block reads are rows its
    // neighbours load at about the same time (found in L2, not fetched again).
    const int ngrp = gridDim.x / ntx, grp = blockIdx.x / ntx;
    xt = blockIdx.x - grp * ntx;
    const long long total = (long long)nty * g.nz;
    lo = total * grp / ngrp;
    hi = total * (grp + 1) / ngrp;
  }
  const uint32_t step = (uint32_t)(*step_dev);
  const bool hist = *hist_dev != 0;
  for (long long w = lo; w < hi;) {
    const long long q = w / g.nz;   // the tile (fixed marches) or the tile row (groups)
    const int k0 = (int)(w - q * g.nz);
    const int kend = (int)min((long long)g.nz, k0 + (hi - w));
    w += kend - k0;
    const long long tile = g.kz > 0 ? q : q * ntx + xt;
    rhs_run<R, NOISE, true>(sm, v, adv, rhs, g, step, hist, tile, k0, kend, threadIdx.x, threadIdx.y);
  }
}

// The right-hand side of every member of a batch: persistent blocks split the members'
// concatenated tile-planes evenly; a run never crosses from one member to the next.
template <typename R, bool NOISE>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) k_rhs_batch(const RhsMember<R>* __restrict__ mem,
                                                                            int nm, long long total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RhsSmem<R>& sm = *reinterpret_cast<RhsSmem<R>*>(smem_raw);
  const long long lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
  int mi = 0;   // the member holding w: the last with w0 <= w
  {
    int a = 0, b = nm - 1;
    while (a < b) {
      const int c = (a + b + 1) / 2;
      if (mem[c].w0 <= lo) a = c; else b = c - 1;
    }
    mi = a;
  }
  for (long long w = lo; w < hi;) {
    while (mi + 1 < nm && mem[mi + 1].w0 <= w) ++mi;
    const RhsMember<R>& m = mem[mi];
    const GridParams g = m.g;
    const long long end = mi + 1 < nm ? min(hi, mem[mi + 1].w0) : hi;
    const long long lw = w - m.w0;
    const long long tile = lw / g.nz;
    const int k0 = (int)(lw - tile * g.nz);
    const int kend = (int)min((long long)g.nz, k0 + (end - w));
    w += kend - k0;
    rhs_run<R, NOISE, false>(sm, m.v, m.adv, m.rhs, g, (uint32_t)(*m.step_dev), *m.hist_dev != 0, tile, k0, kend,
                      threadIdx.x, threadIdx.y);
  }
}

template <typename R>
__global__ void k_normals(GridParams g, uint32_t step, R* __restrict__ out) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  R z[6];
  const uint32_t plane = (uint32_t)g.nx * (uint32_t)g.ny;
  cell_normals<R>((uint32_t)c, plane, ((uint32_t)c / plane) & 1u, step, PhiloxKey{g.key0, g.key1}, z);
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
  const dim3 block(TX, TY);
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, 1);
  if (g.kz > 0) {
    grid.z = (g.nz + g.kz - 1) / g.kz;
  } else {
    // persistent: as many blocks as the SMs hold at once, never more than tile-planes
    static int resident[2] = {0, 0};
    int& res = resident[sizeof(R) == 4 ? 0 : 1];
    if (res == 0) {
      int dev = 0, nsm = 0, per = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (g.kT > 0.0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rhs<R, true>, NT, rhs_smem<R>());
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rhs<R, false>, NT, rhs_smem<R>());
      res = std::max(1, nsm) * std::max(1, per);
    }
    // whole groups of grid.x blocks (one per tile of a tile row), never more groups
    // than tile-row planes
    const long long rows = (long long)grid.y * g.nz;
    const long long ngrp = std::max<long long>(1, std::min<long long>(res / grid.x, rows));
    grid = dim3((unsigned)(ngrp * grid.x), 1, 1);
  }
  if (g.kT > 0.0)
    k_rhs<R, true><<<grid, block, rhs_smem<R>(), st>>>(v, adv, rhs, g, step_dev, hist_dev);
  else
    k_rhs<R, false><<<grid, block, rhs_smem<R>(), st>>>(v, adv, rhs, g, step_dev, hist_dev);
}

long long rhs_tile_planes(int nx, int ny, int nz) {
  return (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * nz;
}

template <typename R>
void batch_rhs(const RhsMember<R>* members, int nm, long long total, bool noise, cudaStream_t st) {
  if (nm <= 0 || total <= 0) return;
  static int resident[2] = {0, 0};
  int& res = resident[sizeof(R) == 4 ? 0 : 1];
  if (res == 0) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rhs_batch<R, true>, NT, rhs_smem<R>());
    res = std::max(1, nsm) * std::max(1, per);
  }
  const dim3 grid((unsigned)std::min<long long>(res, total)), block(TX, TY);
  if (noise)
    k_rhs_batch<R, true><<<grid, block, rhs_smem<R>(), st>>>(members, nm, total);
  else
    k_rhs_batch<R, false><<<grid, block, rhs_smem<R>(), st>>>(members, nm, total);
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
  cudaFuncSetAttribute(k_rhs_batch<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<float>());
  cudaFuncSetAttribute(k_rhs_batch<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<double>());
  cudaFuncSetAttribute(k_rhs_batch<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<float>());
  cudaFuncSetAttribute(k_rhs_batch<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)rhs_smem<double>());
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
  template void batch_rhs<R>(const RhsMember<R>*, int, long long, bool, cudaStream_t);                        \
  template void stress_normals<R>(const GridParams&, long long, R*, cudaStream_t);                           \
  template void field_sums<R>(const R*, long long, double*, double*, int, cudaStream_t);                      \
  template void convert_to_double<R>(const R*, double*, long long, cudaStream_t);                             \
  template void convert_from_double<R>(const double*, R*, long long, cudaStream_t);
ICM_INST(float)
ICM_INST(double)
#undef ICM_INST

}  // namespace icm
