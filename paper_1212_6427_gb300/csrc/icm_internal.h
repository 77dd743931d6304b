// Internal (non-ABI) declarations shared by the translation units of libicm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "icm_common.cuh"

struct icm_sim;

namespace icm {

// Record the message returned by icm_last_error for this thread; returns st.
int record_error(int st, const char* msg);

constexpr int kMaxSide = 512;
constexpr int kMaxStages = 12;

// Sides with two-stage register FFT kernels: N = r1 * r2 (first stage radix r1).
// The host plan of such an axis uses exactly these two radices, in this order.
inline bool fft_split(int n, int& r1, int& r2) {
  switch (n) {
    case 32: r1 = 8; r2 = 4; return true;
    case 48: r1 = 16; r2 = 3; return true;
    case 64: r1 = 8; r2 = 8; return true;
    case 96: r1 = 16; r2 = 6; return true;
    case 128: r1 = 16; r2 = 8; return true;
    case 192: r1 = 16; r2 = 12; return true;
    case 256: r1 = 16; r2 = 16; return true;
    case 384: r1 = 32; r2 = 12; return true;
    case 512: r1 = 32; r2 = 16; return true;
    default: return false;
  }
}

// The other two-stage split of a z side a plan may choose (plan z_split).  The z
// transform is internal to the z pass, so its split changes only the kernel and the
// storage order the z symbol tables follow.
inline bool fft_split_z_alt(int n, int& r1, int& r2) {
  switch (n) {
    case 32: r1 = 4; r2 = 8; return true;
    case 48: r1 = 12; r2 = 4; return true;
    case 64: r1 = 16; r2 = 4; return true;
    case 96: r1 = 8; r2 = 12; return true;
    case 128: r1 = 8; r2 = 16; return true;
    case 192: r1 = 12; r2 = 16; return true;
    case 256: r1 = 32; r2 = 8; return true;
    default: return false;
  }
}

// One axis of the 3D FFT: a mixed-radix factorisation N = prod radix[s] with
// in-place decimation-in-frequency stages.  The forward pass leaves frequency k
// at storage position pos_of_freq[k]; the inverse pass takes that order back to
// natural order, so the spectrum is never reordered.
struct AxisPlan {
  int n = 0;
  int nstages = 0;
  int radix[kMaxStages] = {0};
  const void* tw = nullptr;          // device: n complex, tw[m] = exp(-2 pi i m / n)
  const int* pos_of_freq = nullptr;  // device: n ints
};

// Everything the FFT passes need for one grid.
template <typename R>
struct FftCtx {
  int nx, ny, nz;
  int kx;        // nx/2 + 1 stored x wavenumbers
  int kxp;       // padded row length of the spectrum (multiple of 16)
  long long ncell;
  AxisPlan px, py, pz;
  // Discrete symbols d_a = (exp(i theta_a) - 1)/h and |d_a|^2: x by natural kx,
  // y and z by storage position of the forward pass.
  const cplx_t<R>* dx; const R* ddx;
  const cplx_t<R>* dy; const R* ddy;
  const cplx_t<R>* dz; const R* ddz;
  cplx_t<R>* spec;   // 3 * nz * ny * kxp complex scratch
  const void* zmap;  // host copy of the TMA descriptor of spec for the z pass (or null)
  int* err;          // device error bits (bounded waits report here)
  int zalt;          // 1: the z pass uses the other split of fft_split_z_alt (pz, dz, ddz follow it)
};

// Fill `map` (a 128-byte CUtensorMap) with the descriptor the TMA z pass uses for a
// spectrum buffer; returns false if TMA is unavailable for this shape.
bool make_zmap(void* map, const void* spec, int precision, int kx, int kxp, int ny, int nz, int ncomp = 3);

enum OutMode : int { OUT_STORE = 0, OUT_ADD_AND_STORE2 = 1, OUT_ADD = 2, OUT_NONE = 3 };

// x^ = P^ r^ / (a + b |d|^2) for the three components of src (real face field,
// 3*ncell values).  OUT_STORE: dst = x.  OUT_ADD_AND_STORE2: dst += x, dst2 = x.
// k0sum (device, 3 doubles, may be null): prescribed sum over the grid of each
// output component (the FP64 momentum bookkeeping of the mean mode).
// k0sum * k0scale is the prescribed grid sum (k0scale folds rho dV_f).
template <typename R>
void spectral_solve(const FftCtx<R>& f, const R* src, R* dst, R* dst2, int mode, double a, double b,
                    const double* k0sum, double k0scale, cudaStream_t st);

// The five passes of spectral_solve, for callers that time them one by one.
template <typename R> void fft_x_forward(const FftCtx<R>& f, const R* src, cudaStream_t st);
template <typename R> void fft_y(const FftCtx<R>& f, bool inverse, cudaStream_t st);
template <typename R>
void fft_z_symbol(const FftCtx<R>& f, double a, double b, const double* k0sum, double k0scale, cudaStream_t st);
template <typename R> void fft_x_inverse(const FftCtx<R>& f, R* dst, R* dst2, int mode, cudaStream_t st);

struct RowBlobs;
// One replica of a group solve: the same grid for every replica, launched once for all.
struct RepFft {
  const void* src;      // real face field (3 ncell)
  void* spec;           // spectrum scratch
  void* dst;            // output field
  void* dst2;           // second output (OUT_ADD_AND_STORE2)
  const double* k0sum;  // prescribed grid sums of the mean mode (or null)
  double a, b, k0mul;   // symbol a + b |d|^2 and k0sum scale (k0scale / ncell)
  int slot;             // spec = slot-th spectrum of a contiguous group buffer (tensor-map z pass)
  const RowBlobs* rb;   // the replica's blob work in the x passes (blob solves), or null
};
// spectral_solve for G replicas of the grid of f (register sides only): every pass is
// one launch over all replicas; reps is a device array of G entries.  With gzmap (a
// tensor map of a group buffer that holds every replica's spectrum, from make_zmap with
// ncomp = 3 x slots) the z pass is the persistent tensor-map one over all replicas'
// tiles; otherwise one block per z tile.  With blobs, every replica's x passes carry
// its blob work as the single-simulation fused passes do (reps[i].rb: the spread of
// rb->vec in the forward pass, when set, and the gathers of the inverse pass; mode
// OUT_STORE and OUT_NONE gather J, OUT_ADD also J L; src may be null).
template <typename R>
void spectral_solve_group(const FftCtx<R>& f, const RepFft* reps, int G, int mode, cudaStream_t st,
                          const void* gzmap = nullptr, bool blobs = false);
bool fft_has_group_passes(int nx, int ny, int nz);

// One-thread kernel whose bounded mbarrier wait runs out (a transaction that is never
// issued): raises DEV_ERR_TIMEOUT in err after limit_ns.  Tests the failure path only.
void debug_wait_timeout(int* err, long long limit_ns, cudaStream_t st);

// Peak FMA rate (flop/s, 2 per FMA) of this device in precision 32 or 64: independent
// FMA chains in every thread of blocks_per_sm 256-thread blocks per SM, `iters` FMAs
// per chain, the second of two launches timed with CUDA events on st.  -1 on error.
double fma_rate(int precision, int iters, int blocks_per_sm, cudaStream_t st, double* seconds);

// Raise the dynamic shared-memory limits of the kernels (call once, outside capture).
void fft_prepare();
void grid_prepare();

// ---------------------------------------------------------------------------
// Grid kernels (icm_grid.cu)
// ---------------------------------------------------------------------------
struct GridParams {
  int nx, ny, nz;
  long long ncell;
  double h, rho, eta, kT, dt;
  uint32_t key0, key1;
  PhiloxRoundKeys rk;   // the round keys of (key0, key1)
  int advection;
  int kz;           // z planes marched per block of the RHS kernel (>= 1)
};

// r = (rho/dt) v + (eta/2) L v + div Sigma^n - (3/2 A^n - 1/2 A^{n-1}); adv <- A^n.
// step_dev: device int64 time level (Philox counter word 1).  has_hist_dev: device
// int, 0 = no history (A^{n-1} := A^n); set to 1 by the kernel launch sequence.
template <typename R>
void explicit_rhs(const GridParams& g, const R* v, R* adv, R* rhs, const long long* step_dev,
                  const int* has_hist_dev, cudaStream_t st);

template <typename R>
void stress_normals(const GridParams& g, long long step, R* out, cudaStream_t st);

void philox_words(long long n, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                  uint32_t* out, cudaStream_t st);

// out[c] = sum over the grid of component c (FP64, compensated), 3 doubles.
template <typename R>
void field_sums(const R* v, long long ncell, double* out_dev, double* partial_dev, int npartial, cudaStream_t st);

template <typename R>
void convert_to_double(const R* src, double* dst, long long n, cudaStream_t st);
template <typename R>
void convert_from_double(const double* src, R* dst, long long n, cudaStream_t st);

// ---------------------------------------------------------------------------
// Blob kernels (icm_blob.cu)
// ---------------------------------------------------------------------------
struct BlobParams {
  int nx, ny, nz;
  long long ncell;
  double h, rho, eta, dt;
  int kernel;
  int slip;        // 0 visc, 1 zero, 2 full
  double mtf;      // m~_f = 3 rho dV / 2
  double inv_h;    // 1/h
  double box[3];   // periodic box lengths N h
  double inv_box[3];
  double kT;       // thermal energy (the thermal drift's weight)
  double trap_k;   // harmonic trap V = k r^2 / 2 about trap_c (0: none)
  double trap_c[3];
  int* err;        // device error bits (the checked build's index checks report here)
};

struct BlobState {
  long long nb;
  double* q;        // positions q^n (n,3)
  double* qh;       // midpoint q^{n+1/2}
  double* u;        // velocities
  const double* me; // excess masses
  const double* f;  // external forces (constant part)
  double* fe;       // forces at q^{n+1/2} (constant part + trap), written by the predictor
  double* g;        // lagged J L dv (slip term)
  double* w0;       // J^n v^n at q^n
  double* w1;       // J^{n+1/2} v^n
  double* jvt;      // J v~
  double* du;       // slip correction
  double* dp;       // momentum change
  double* cdp;      // m~_f/(rho(m~_f+m_e)) dp
  double* src;      // dp - m_e J dv~
  double* scal;     // device scalars (see ScalarSlot)
  int* err;         // device error bits
};

enum ScalarSlot : int {
  SC_PBAR = 0,      // [3] total fluid momentum rho dV_f sum v (FP64 bookkeeping)
  SC_SUMF = 3,      // [3] sum of external forces
  SC_SUMSRC = 6,    // [3] sum_i (dp_i - m_e,i J dv~_i) of this step
  SC_K0 = 9,        // [3] prescribed grid sum of the provisional solve output
  SC_K0B = 12,      // [3] prescribed grid sum of the viscous correction output
  SC_PTOT = 16,     // [3] total momentum (fluid + blob excess) for a host read
  SC_COUNT = 20
};

template <typename R> void blob_predict(const BlobParams& p, BlobState s, const R* v, cudaStream_t st);
template <typename R> void blob_spread(const BlobParams& p, long long nb, const double* q, const double* vec,
                                       R* field, cudaStream_t st);
template <typename R> void blob_momentum_change(const BlobParams& p, BlobState s, const R* vt, cudaStream_t st);
// out[a] = init[a] (0 if init is null) + sum_i w_i x[3 i + a] (w_i = 1 if w is null),
// FP64 compensated sums per thread, then over blocks (partial: 3 npartial doubles of
// scratch); out may not alias x, w or init.
void rows_sum3(const double* x, const double* w, long long n, const double* init, double* out, double* partial,
               int npartial, cudaStream_t st);
// positions and velocities of nb blobs, the momentum ptot [3], the time level and the error
// bits into out [6 nb + 5] (the last two as bit patterns), one launch.
void blob_snapshot(const double* q, const double* u, long long nb, const double* ptot, const long long* step,
                   const int* err, double* out, cudaStream_t st);
template <typename R> void blob_inertial(const BlobParams& p, BlobState s, const R* dvt, cudaStream_t st);
template <typename R> void blob_finish(const BlobParams& p, BlobState s, const R* v_new, const R* dv,
                                       bool inertial, cudaStream_t st);
template <typename R> void blob_interp(const BlobParams& p, long long nb, const double* q, const R* field,
                                       bool laplacian, double* out, cudaStream_t st);
// Thermal drift (Appendix B.2, Eq. thermal_drift): adds kT m~_f/(m~_f + m_e) dV_f^-1
// d/dq_a phi(q^{n+1/2} - r) to component a of field (atomics).
template <typename R> void blob_spread_drift(const BlobParams& p, BlobState s, R* field, cudaStream_t st);

// ---------------------------------------------------------------------------
// Blob work fused into the x passes (sides with register FFT kernels)
// ---------------------------------------------------------------------------
// Row-block bins: the blobs whose extended support touches each 32-row x-pass block.
// The builder also writes each blob's stencil geometry (anchor cells and fractional
// offsets, FP64 arithmetic done once) and zeroes the blob accumulators of the step.
struct RowBins {
  int* count;    // [nblocks], zero between builds
  int* start;    // [nblocks + 1]
  int* cursor;   // [nblocks]
  int* list;     // [capacity] blob ids
  void* geo;     // [nb] stencil records (R-typed, at most kStencilBytes each)
  double* acc;   // [nacc * nb] accumulators zeroed by the build
  int nacc;
  int nblocks;
  long long capacity;
};
constexpr int kBinsPerBlob = 49;   // capacity per blob: 7 x 7 (y, z) node pairs at most
constexpr int kStencilBytes = 336; // per-blob stencil record (FP64: 12 ints + 36 doubles)

// A blob source spread into the rows of x_fwd, or the accumulators x_inv gathers into.
struct RowBlobs {
  const int* start;
  const int* list;
  const void* geo;     // stencil records
  const double* vec;   // spread: per-blob vectors (n,3), spread as phi vec / dV_f
  double* acc;         // gather: J of the transform output, (n,3) accumulators
  double* acc_lap;     // gather: J L of the transform output without 1/h^2, (n,3)
  BlobParams p;
};
template <typename R>
void build_row_bins(const BlobParams& p, long long nb, const double* q, RowBins bins, cudaStream_t st);
// x passes with blob work: src may be null (the spread source only).
template <typename R>
void fft_x_forward_blobs(const FftCtx<R>& f, const R* src, const RowBlobs& rb, cudaStream_t st);
// Forward x and y passes fused on thread-block clusters (FP32, Nx = Ny in 32, 64, 128,
// 256, clusters the device can hold): the spectrum fft_x_forward(_blobs) + fft_y
// leave, without its HBM round trip in between.  rb: the blob spread, or null.
bool fft_has_xy_passes(int precision, int nx, int ny);
template <typename R>
void fft_xy_forward(const FftCtx<R>& f, const R* src, const RowBlobs* rb, cudaStream_t st);
// mode: OUT_STORE (dst = x), OUT_ADD (dst += x) or OUT_NONE; gathers J x into rb.acc
// and, if rb.acc_lap is set, J L x (without 1/h^2) into rb.acc_lap.
template <typename R>
void fft_x_inverse_blobs(const FftCtx<R>& f, R* dst, int mode, const RowBlobs& rb, cudaStream_t st);
bool fft_has_blob_passes(int nx);

// WCA pair forces (Sec. IV.A, Eq. WCA) at q^{n+1/2} through a cell list of cells at
// least the cut-off wide: count, scan (k_bin_scan on the cell arrays), fill, forces.
struct WcaParams {
  double eps, sigma, rc2;
  int nc[3];          // cells per axis
  double cell_inv[3]; // nc / L
  int lo[3], hi[3];   // neighbour cell offsets per axis (distinct cells only)
  int ncells;
  int* count;         // [ncells], zero between builds
  int* start;         // [ncells + 1]
  int* cursor;        // [ncells]
  int* list;          // [nb]
};
// fe = (with_trap ? fe : f) + F_wca; dt times the WCA total goes to the grid sum K0.
void blob_wca_forces(const BlobParams& p, BlobState s, const WcaParams& w, bool with_trap, cudaStream_t st);

// Elementwise blob updates of the fused step (one thread per blob component).
void blob_dp_from(const BlobParams& p, BlobState s, const double* jvt, cudaStream_t st);
void blob_inertial_from(const BlobParams& p, BlobState s, const double* jdvt, cudaStream_t st);
// jv = base + add (base may be null): J^{n+1/2} v^{n+1}; g: J L dv without 1/h^2.
// With step_dev (and hist_dev) the same launch also does the end-of-step bookkeeping of
// scalars_after_step (inertial: the viscous correction's source sum enters P^{n+1}).
void blob_finish_from(const BlobParams& p, BlobState s, const double* base, const double* add, const double* g,
                      bool inertial, cudaStream_t st, long long* step_dev = nullptr, int* hist_dev = nullptr);

// ---------------------------------------------------------------------------
// Stages launched once over every member of a batch (replica simulations of any grid;
// one precision per launch).  A device table holds each member's parameters and state;
// blob work finds its member through member_of[global blob index].
// ---------------------------------------------------------------------------
struct BlobMember {
  BlobParams p;
  BlobState s;
  const void* v;          // face velocities (R)
  void* work;             // work field (R): spread sources, dv~, dv
  const double* fvec;     // forces spread into the first solve (null: none)
  long long* step_dev;    // time level
  int* hist_dev;          // Adams-Bashforth history flag
  long long b0;           // first global blob index of the member
  int inertial;           // any excess mass: steps 4-8 run
  RowBins bins;           // row-block bins and accumulators of the fused x passes (batched stages)
};
enum BatchVec : int { BV_FORCE = 0, BV_CDP = 1, BV_SRC = 2 };
template <typename R> void batch_predict(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st);
// Batched stages with the blob work inside the group x passes: the row bins of every
// member at q^{n+1/2} (count, one scan block per member, fill; the accumulators zeroed),
// and steps 4, 6-8 and 9 from the accumulators the inverse x passes gathered into
// (bins.acc: J v~, J dv~, J dv, J L dv without 1/h^2, 3 nb each).
template <typename R>
void batch_bins(const BlobMember* m, const int* member_of, long long nbt, int nm, cudaStream_t st);
void batch_dp_from(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st);
void batch_inertial_from(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st);
void batch_finish_from(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st);
template <typename R>
void batch_spread(const BlobMember* m, const int* member_of, long long nbt, int which, cudaStream_t st);
template <typename R> void batch_dp(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st);
template <typename R> void batch_inertial(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st);
template <typename R> void batch_finish(const BlobMember* m, const int* member_of, long long nbt, cudaStream_t st);
// work[0 .. 3 ncell) = 0 for every member (ncell_max: the largest member's cells)
// work = 0 for every member of m; prefix16 (device, nm + 1 entries) holds the running
// sums of the members' work sizes in 16-byte words, total16 their sum.
void batch_zero_work(const BlobMember* m, const long long* prefix16, int nm, long long total16, cudaStream_t st);
void batch_scalars_before(const BlobMember* m, int nm, cudaStream_t st);
void batch_scalars_after(const BlobMember* m, int nm, cudaStream_t st);

// The right-hand side of every member (persistent blocks over all members' tile-planes).
template <typename R>
struct RhsMember {
  GridParams g;
  const R* v;
  R* adv;
  R* rhs;
  const long long* step_dev;
  const int* hist_dev;
  long long w0;           // first global tile-plane of the member
};
// members[0 .. nm) in order of w0; total = the last member's w0 + its tile-planes.
template <typename R>
void batch_rhs(const RhsMember<R>* members, int nm, long long total, bool noise, cudaStream_t st);
// Tile-planes (32 x 16 cells per tile) of a grid in the RHS kernel.
long long rhs_tile_planes(int nx, int ny, int nz);

// Scalar bookkeeping kernels.
void scalars_before_step(double* scal, double dt, double rho, double dvf, cudaStream_t st);
void scalars_after_step(double* scal, double dt, double rho, double dvf, bool inertial, long long* step_dev,
                        int* has_hist_dev, cudaStream_t st);

}  // namespace icm
