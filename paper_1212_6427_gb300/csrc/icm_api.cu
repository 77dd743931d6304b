// Host side of libicm: the C ABI declared in include/icm.h.
//
// Owns the device state of a simulation (face fields, Adams-Bashforth history,
// spectrum scratch, FFT tables, blob arrays, FP64 scalars) and enqueues one ICM
// step (arXiv:1212.6427, Sec. III.C, steps 1-9) as a fixed sequence of kernels on
// the simulation's stream.  The sequence is captured once into a CUDA graph; the
// time level lives in device memory, so the same graph replays every step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/icm.h"
#include "icm_internal.h"

using namespace icm;

namespace {

thread_local std::string g_err = "no error";

icm_alloc_fn g_alloc = nullptr;
icm_free_fn g_free = nullptr;
void* g_actx = nullptr;

icm_status fail(icm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define ICM_CK(call)                                                                                 \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(ICM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

bool side_ok(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

std::vector<int> factor_radices(int n) {
  std::vector<int> r;
  int m = n;
  while (m % 16 == 0) { r.push_back(16); m /= 16; }
  if (m % 8 == 0) { r.push_back(8); m /= 8; }
  if (m % 4 == 0) { r.push_back(4); m /= 4; }
  if (m % 2 == 0) { r.push_back(2); m /= 2; }
  while (m % 3 == 0) { r.push_back(3); m /= 3; }
  return r;
}

double kernel_sum_sq(int kernel) { return kernel == 3 ? 0.5 : 0.375; }

}  // namespace

int icm::record_error(int st, const char* msg) {
  g_err = msg;
  return st;
}

struct icm_sim {
  int nx = 0, ny = 0, nz = 0;
  long long ncell = 0;
  double h = 1, rho = 1, eta = 1, kT = 0, dt = 1;
  int kernel = 4, prec = 32, flags = 0, slip = 0;
  uint64_t seed = 0;
  bool advection = true;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // execution plan (icm_plan) and where it came from
  icm_plan plan = {1, 1, 16, 1, 0};
  int plan_src = 0;   // 0 default, 1 from the process-wide table, 2 set or tuned on this simulation
  // second stream of the step graph: the blob-side prologue runs beside the RHS
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  icm_alloc_fn alloc = nullptr;
  icm_free_fn release = nullptr;
  void* actx = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
  long long bytes = 0;

  // grid state (precision R = float or double)
  void* v = nullptr;     // face velocities
  void* adv = nullptr;   // A^{n-1}, overwritten by A^n
  void* work = nullptr;  // right-hand side / spread sources / dv~ / dv
  void* spec = nullptr;  // spectrum scratch
  // FFT plans and symbol tables
  AxisPlan px, py, pz;
  void *dx = nullptr, *ddx = nullptr, *dy = nullptr, *ddy = nullptr, *dz = nullptr, *ddz = nullptr;
  // the other split of the z side (plan z_split), where there is one
  bool has_zalt = false;
  AxisPlan pz_alt;
  void *dz_alt = nullptr, *ddz_alt = nullptr;
  int kx = 0, kxp = 0;
  alignas(64) unsigned char zmap[128];   // TMA descriptor of spec for the z pass
  bool has_zmap = false;
  // blobs
  long long nb = 0, cap = 0;
  double* blob = nullptr;
  double *q = nullptr, *qh = nullptr, *u = nullptr, *me = nullptr, *f = nullptr, *g = nullptr, *w0 = nullptr,
         *w1 = nullptr, *jvt = nullptr, *du = nullptr, *dp = nullptr, *cdp = nullptr, *src = nullptr, *fe = nullptr;
  double trap_k = 0.0, trap_c[3] = {0.0, 0.0, 0.0};   // harmonic trap (Sec. III.D test)
  double wca_eps = 0.0, wca_sigma = 1.0;              // WCA pair potential (Sec. IV.A)
  int wca_nc[3] = {1, 1, 1};
  int* wca_idx = nullptr;                             // cell count, start, cursor
  int* cell_list = nullptr;                           // [cap], in the blob allocation
  std::vector<double> me_host, f_host;
  bool any_me = false, any_force = false;
  // row-block bins of the blob work fused into the x passes (register FFT sides)
  bool fused = false;
  int nrowblk = 0;
  int* bin_idx = nullptr;     // count [nrowblk], start [nrowblk + 1], cursor [nrowblk]
  void* bin_blob = nullptr;   // list [kBinsPerBlob cap] ints, geometry [cap], accumulators [12 cap]
  int* bin_list = nullptr;
  void* geo = nullptr;
  double* acc = nullptr;
  // scalars
  double* scal = nullptr;
  long long* step_dev = nullptr;
  int* hist_dev = nullptr;
  int* err_dev = nullptr;
  double* partial = nullptr;
  static constexpr int kPartials = 1024;
  // page-locked host staging of the per-step host I/O: forces [3 cap], positions [3 cap],
  // velocities [3 cap], scalars [8] (the total force, then what icm_read_state reads);
  // the forces' slot is rewritten only once the copy out of it (ev_hforce) has passed
  double* hstage = nullptr;
  long long hstage_cap = -1;
  cudaEvent_t ev_hforce = nullptr;
  bool hforce_pending = false;
  // queued reads (icm_read_begin): two staging slots after the synchronous read's, used
  // in turn; read_head is the oldest pending, read_pending how many (0-2)
  static constexpr int kReadSlots = 2;
  cudaEvent_t ev_read[kReadSlots] = {nullptr, nullptr};
  int read_head = 0, read_pending = 0;
  // host <-> device copies of the per-step I/O run on their own streams beside the steps
  // (one up, one down, so that an upload never queues behind a download that waits for a
  // step): forces go up into dfstage and are copied into f on the simulation's stream; a
  // queued read gathers the blob state into a device slot of dsnap and copies that down
  cudaStream_t copy = nullptr, copy_up = nullptr;
  cudaEvent_t ev_fup = nullptr, ev_fcons = nullptr, ev_snap[kReadSlots] = {nullptr, nullptr};
  double* dfstage = nullptr;
  double* dsnap = nullptr;
  long long dstage_cap = -1;
  // graph of one step
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
  long long version = 0;     // bumped whenever the step sequence changes (batch graphs recapture)

  size_t rsize() const { return prec == 32 ? sizeof(float) : sizeof(double); }
};

namespace {

// Per blob slot: the bin list (kBinsPerBlob ints), the stencil record and 4 (n,3)
// FP64 accumulators.
constexpr size_t kGeoBytes = kStencilBytes;
constexpr int kAccPerBlob = 12;
size_t bin_list_bytes(long long cap) { return ((size_t)kBinsPerBlob * 4 * cap + 255) / 256 * 256; }
size_t bin_blob_bytes(long long cap) { return bin_list_bytes(cap) + (kGeoBytes + 8 * kAccPerBlob) * cap; }

void* dalloc(icm_sim* s, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  if (s->alloc) {
    p = s->alloc(s->actx, bytes, (void*)s->stream);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    s->allocs.push_back({p, bytes});
    s->bytes += (long long)bytes;
  }
  return p;
}

void dfree(icm_sim* s, void* p) {
  if (!p) return;
  for (size_t i = 0; i < s->allocs.size(); ++i) {
    if (s->allocs[i].first == p) {
      s->bytes -= (long long)s->allocs[i].second;
      s->allocs.erase(s->allocs.begin() + i);
      break;
    }
  }
  if (s->release)
    s->release(s->actx, p, (void*)s->stream);
  else
    cudaFree(p);
}

// Scoped temporary device buffer for the operator entry points.
struct Tmp {
  icm_sim* s;
  void* p;
  Tmp(icm_sim* s_, size_t bytes) : s(s_), p(dalloc(s_, bytes)) {}
  ~Tmp() {
    if (p) {
      cudaStreamSynchronize(s->stream);
      dfree(s, p);
    }
  }
};

template <typename R>
FftCtx<R> fft_ctx(const icm_sim* s) {
  FftCtx<R> f;
  f.nx = s->nx; f.ny = s->ny; f.nz = s->nz;
  f.kx = s->kx; f.kxp = s->kxp;
  f.ncell = s->ncell;
  f.px = s->px; f.py = s->py; f.pz = s->pz;
  f.dx = (const cplx_t<R>*)s->dx; f.ddx = (const R*)s->ddx;
  f.dy = (const cplx_t<R>*)s->dy; f.ddy = (const R*)s->ddy;
  f.dz = (const cplx_t<R>*)s->dz; f.ddz = (const R*)s->ddz;
  f.spec = (cplx_t<R>*)s->spec;
  f.zmap = s->has_zmap && s->plan.tma_z ? s->zmap : nullptr;
  f.err = s->err_dev;
  f.zalt = 0;
  if (s->plan.z_split && s->has_zalt) {
    f.zalt = 1;
    f.pz = s->pz_alt;
    f.dz = (const cplx_t<R>*)s->dz_alt;
    f.ddz = (const R*)s->ddz_alt;
  }
  return f;
}

GridParams grid_params(const icm_sim* s) {
  GridParams g;
  g.nx = s->nx; g.ny = s->ny; g.nz = s->nz;
  g.ncell = s->ncell;
  g.h = s->h; g.rho = s->rho; g.eta = s->eta; g.kT = s->kT; g.dt = s->dt;
  g.key0 = (uint32_t)(s->seed & 0xffffffffu);
  g.key1 = (uint32_t)(s->seed >> 32);
  g.rk = philox_round_keys(g.key0, g.key1);
  g.advection = s->advection ? 1 : 0;
  g.kz = s->plan.rhs_kz;
  return g;
}

double blob_volume(const icm_sim* s) {
  const double q = kernel_sum_sq(s->kernel);
  return s->h * s->h * s->h / (q * q * q);
}

BlobParams blob_params(const icm_sim* s) {
  BlobParams p;
  p.nx = s->nx; p.ny = s->ny; p.nz = s->nz;
  p.ncell = s->ncell;
  p.h = s->h; p.rho = s->rho; p.eta = s->eta; p.dt = s->dt;
  p.kernel = s->kernel;
  p.slip = s->slip;
  p.mtf = 1.5 * s->rho * blob_volume(s);
  p.inv_h = 1.0 / s->h;
  const int n[3] = {s->nx, s->ny, s->nz};
  for (int a = 0; a < 3; ++a) {
    p.box[a] = n[a] * s->h;
    p.inv_box[a] = 1.0 / p.box[a];
    p.trap_c[a] = s->trap_c[a];
  }
  p.trap_k = s->trap_k;
  p.kT = s->kT;
  p.err = s->err_dev;
  return p;
}

BlobState blob_state(const icm_sim* s) {
  BlobState b;
  b.nb = s->nb;
  b.q = s->q; b.qh = s->qh; b.u = s->u; b.me = s->me; b.f = s->f; b.fe = s->fe; b.g = s->g;
  b.w0 = s->w0; b.w1 = s->w1; b.jvt = s->jvt; b.du = s->du; b.dp = s->dp; b.cdp = s->cdp; b.src = s->src;
  b.scal = s->scal;
  b.err = s->err_dev;
  return b;
}

WcaParams wca_params(const icm_sim* s) {
  WcaParams w;
  w.eps = s->wca_eps;
  w.sigma = s->wca_sigma;
  const double rc = std::pow(2.0, 1.0 / 6.0) * s->wca_sigma;
  w.rc2 = rc * rc;
  const int n[3] = {s->nx, s->ny, s->nz};
  w.ncells = 1;
  for (int a = 0; a < 3; ++a) {
    w.nc[a] = s->wca_nc[a];
    w.cell_inv[a] = w.nc[a] / (n[a] * s->h);
    w.lo[a] = w.nc[a] >= 3 ? -1 : 0;
    w.hi[a] = w.nc[a] >= 2 ? 1 : 0;
    w.ncells *= w.nc[a];
  }
  w.count = s->wca_idx;
  w.start = s->wca_idx ? s->wca_idx + w.ncells : nullptr;
  w.cursor = s->wca_idx ? s->wca_idx + 2 * w.ncells + 1 : nullptr;
  w.list = s->cell_list;
  return w;
}

// Build one axis plan: radices, twiddles (long double), digit-reversed order, and
// the symbol d = (exp(i theta) - 1)/h, |d|^2 = 4 sin^2(theta/2)/h^2 by storage position
// (x: by natural wavenumber, only nx/2+1 of them).
icm_status build_axis(icm_sim* s, int n, bool natural, int count, AxisPlan& P, void*& dtab, void*& ddtab,
                      bool z_alt = false) {
  int r1 = 0, r2 = 0;
  const bool two = z_alt ? fft_split_z_alt(n, r1, r2) : fft_split(n, r1, r2);
  const std::vector<int> rad = two ? std::vector<int>{r1, r2} : factor_radices(n);
  P.n = n;
  P.nstages = (int)rad.size();
  for (size_t i = 0; i < rad.size(); ++i) P.radix[i] = rad[i];
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<int> pof(n), fop(n);
  for (int k = 0; k < n; ++k) {
    int pos = 0, M = n, rem = k;
    for (int r : rad) {
      pos += (M / r) * (rem % r);
      rem /= r;
      M /= r;
    }
    pof[k] = pos;
    fop[pos] = k;
  }
  const size_t rs = s->rsize();
  std::vector<unsigned char> tw(2 * rs * n), dt(2 * rs * count), dd(rs * count);
  auto put = [&](std::vector<unsigned char>& buf, size_t idx, long double val) {
    if (rs == 4) {
      float x = (float)val;
      memcpy(&buf[idx * 4], &x, 4);
    } else {
      double x = (double)val;
      memcpy(&buf[idx * 8], &x, 8);
    }
  };
  for (int m = 0; m < n; ++m) {
    const long double th = 2.0L * pi * (long double)m / (long double)n;
    put(tw, 2 * m, cosl(th));
    put(tw, 2 * m + 1, -sinl(th));
  }
  for (int i = 0; i < count; ++i) {
    const int k = natural ? i : fop[i];
    const long double th = 2.0L * pi * (long double)k / (long double)n;
    const long double h = s->h;
    put(dt, 2 * i, (cosl(th) - 1.0L) / h);
    put(dt, 2 * i + 1, sinl(th) / h);
    const long double sn = sinl(0.5L * th);
    put(dd, i, 4.0L * sn * sn / (h * h));
  }
  void* dtw = dalloc(s, tw.size());
  void* dpof = dalloc(s, sizeof(int) * n);
  dtab = dalloc(s, dt.size());
  ddtab = dalloc(s, dd.size());
  if (!dtw || !dpof || !dtab || !ddtab) return fail(ICM_ENOMEM, "device allocation of FFT tables failed");
  ICM_CK(cudaMemcpyAsync(dtw, tw.data(), tw.size(), cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaMemcpyAsync(dpof, pof.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaMemcpyAsync(dtab, dt.data(), dt.size(), cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaMemcpyAsync(ddtab, dd.data(), dd.size(), cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  P.tw = dtw;
  P.pos_of_freq = (const int*)dpof;
  return ICM_OK;
}

bool finite_all(const double* a, long long n) {
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

void invalidate_graph(icm_sim* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->graph_ok = false;
  s->version++;
}

// Per-launch CUDA events of an instrumented (eager) step: stage name, algorithmic
// bytes of one launch, accumulated milliseconds.
struct Prof {
  struct Entry {
    std::string name;
    double bytes = 0, ms = 0;
    cudaEvent_t a = nullptr, b = nullptr;
  };
  std::vector<Entry> e;
  size_t idx = 0;
  void begin(cudaStream_t st, const char* name, double bytes) {
    if (idx == e.size()) {
      Entry x;
      x.name = name;
      x.bytes = bytes;
      cudaEventCreate(&x.a);
      cudaEventCreate(&x.b);
      e.push_back(x);
    }
    cudaEventRecord(e[idx].a, st);
  }
  void end(cudaStream_t st) { cudaEventRecord(e[idx++].b, st); }
  void collect() {
    for (auto& x : e) {
      float t = 0;
      cudaEventElapsedTime(&t, x.a, x.b);
      x.ms += t;
    }
    idx = 0;
  }
  ~Prof() {
    for (auto& x : e) {
      cudaEventDestroy(x.a);
      cudaEventDestroy(x.b);
    }
  }
};

#define ICM_STAGE(name, bytes, ...)            \
  do {                                         \
    if (prof) prof->begin(st, name, (bytes));  \
    __VA_ARGS__;                               \
    if (prof) prof->end(st);                   \
  } while (0)

// Segments 1-3 of a step whose three solves run as group launches over several
// simulations (the separate blob path of enqueue_step between the solves).
template <typename R>
void enqueue_segment(icm_sim* s, int segment, int last) {
  cudaStream_t st = s->stream;
  const BlobParams bp = blob_params(s);
  const BlobState bs = blob_state(s);
  R* v = (R*)s->v;
  R* work = (R*)s->work;
  const double dvf = s->h * s->h * s->h;
  const size_t fbytes = 3 * (size_t)s->ncell * sizeof(R);
  if (segment == 1 && s->any_me) {
    // step 4, and the spread of step 5
    blob_momentum_change<R>(bp, bs, v, st);
    cudaMemsetAsync(work, 0, fbytes, st);
    blob_spread<R>(bp, s->nb, s->qh, s->cdp, work, st);
  } else if (segment == 2) {
    // steps 6 and 8 (blob side), and the spread of step 6
    blob_inertial<R>(bp, bs, work, st);
    cudaMemsetAsync(work, 0, fbytes, st);
    blob_spread<R>(bp, s->nb, s->qh, s->src, work, st);
  }
  if (segment == last) {
    // step 9
    if (s->any_me)
      blob_finish<R>(bp, bs, v, work, true, st);
    else
      blob_finish<R>(bp, bs, v, nullptr, false, st);
    scalars_after_step(s->scal, s->dt, s->rho, dvf, s->any_me, s->step_dev, s->hist_dev, st);
  }
}

// The row-block bins of a simulation's fused x passes (register x sides with blobs).
RowBins row_bins(const icm_sim* s) {
  RowBins bins;
  bins.count = s->bin_idx;
  bins.start = s->bin_idx ? s->bin_idx + s->nrowblk : nullptr;
  bins.cursor = s->bin_idx ? s->bin_idx + 2 * s->nrowblk + 1 : nullptr;
  bins.list = s->bin_list;
  bins.geo = s->geo;
  bins.acc = s->acc;
  bins.nacc = kAccPerBlob;
  bins.nblocks = s->nrowblk;
  bins.capacity = (long long)kBinsPerBlob * s->cap;
  return bins;
}

// The nine steps of Sec. III.C for one time level, enqueued on s->stream.  With a
// segment index (batched group solves) only the blob and stencil work between two
// solves is enqueued: segment 0 ends before the first solve, segments 1 and 2 after
// the first and second, segment 3 after the third; the caller runs the solves.
template <typename R>
void enqueue_step(icm_sim* s, Prof* prof, int segment = -1) {
  cudaStream_t st = s->stream;
  const FftCtx<R> fc = fft_ctx<R>(s);
  const GridParams gp = grid_params(s);
  const BlobParams bp = blob_params(s);
  const BlobState bs = blob_state(s);
  R* v = (R*)s->v;
  R* adv = (R*)s->adv;
  R* work = (R*)s->work;
  const double dvf = s->h * s->h * s->h;
  const double k0scale = 1.0 / (s->rho * dvf);
  const size_t fbytes = 3 * (size_t)s->ncell * sizeof(R);
  // algorithmic bytes per launch
  const double F = (double)fbytes;
  const double S = 3.0 * s->ny * s->nz * s->kx * 2.0 * sizeof(R);
  const double w3 = (double)s->kernel * s->kernel * s->kernel;
  const double w3l = (double)(s->kernel + 2) * (s->kernel + 2) * (s->kernel + 2);
  const double nb = (double)s->nb;
  const double gath = nb * 3.0 * w3 * sizeof(R);
  // forward x and y passes fused on clusters (a plan choice on grids that allow it)
  const bool xy = s->plan.fused_xy && fft_has_xy_passes(s->prec, s->nx, s->ny);
  auto solve = [&](const char* tag, const R* src, R* dst, R* dst2, int mode, double a, double b, const double* k0) {
    std::string t(tag);
    if (xy) {
      ICM_STAGE((t + ".xy_fwd").c_str(), F + S, fft_xy_forward<R>(fc, src, nullptr, st));
    } else {
      ICM_STAGE((t + ".x_fwd").c_str(), F + S, fft_x_forward<R>(fc, src, st));
      ICM_STAGE((t + ".y_fwd").c_str(), 2 * S, fft_y<R>(fc, false, st));
    }
    ICM_STAGE((t + ".z_sym").c_str(), 2 * S, fft_z_symbol<R>(fc, a, b, k0, k0 ? k0scale : 0.0, st));
    ICM_STAGE((t + ".y_inv").c_str(), 2 * S, fft_y<R>(fc, true, st));
    ICM_STAGE((t + ".x_inv").c_str(), S + (mode == OUT_STORE ? F : 3 * F), fft_x_inverse<R>(fc, dst, dst2, mode, st));
  };

  // forces at q^{n+1/2}: the constant ones, or with the trap those the predictor writes
  const bool wca = s->wca_eps > 0.0 && s->nb > 1 && s->wca_idx != nullptr;
  const double* fvec =
      s->nb == 0 ? nullptr : ((s->trap_k != 0.0 || wca) ? s->fe : (s->any_force ? s->f : nullptr));
  // thermal drift (Appendix B.2) at q^{n+1/2}, added to the right-hand side of the first solve
  const bool drift = (s->flags & ICM_FLAG_THERMAL_DRIFT) && s->kT > 0.0 && s->nb > 0;
  const bool fused = s->fused && s->plan.fused_blobs && s->nb > 0 && segment < 0;
  const RowBins bins = row_bins(s);
  const double geob = (double)(12 * sizeof(int) + 36 * sizeof(R));   // stencil record per blob

  // The blob-side prologue (scalars, predictor, pair forces, bins) reads only v and the
  // blob state: in the step graph it runs on a second stream beside the RHS and joins
  // before the first solve.  Instrumented steps keep one stream.
  const bool grouped = segment >= 0;
  const bool fork = prof == nullptr && s->plan.fork && !grouped;
  cudaStream_t sb = fork ? s->aux : st;
  if (fork) {
    cudaEventRecord(s->ev_fork, st);
    cudaStreamWaitEvent(sb, s->ev_fork, 0);
  }
  const int last = s->any_me ? 3 : 1;
  if (segment > 0) {
    enqueue_segment<R>(s, segment, last);
    return;
  }
  ICM_STAGE("scalars", 0, scalars_before_step(s->scal, s->dt, s->rho, dvf, sb));
  // step 1: midpoint predictor (Eq. particle_pred)
  ICM_STAGE("predict", 2 * gath + nb * 72, blob_predict<R>(bp, bs, v, sb));
  // pair forces at q^{n+1/2} (four kernels: cell count, scan, fill, forces)
  if (wca) ICM_STAGE("wca", nb * 96, blob_wca_forces(bp, bs, wca_params(s), s->trap_k != 0.0, sb));
  if (fused)
    ICM_STAGE("bins", nb * (24.0 + 2 * geob + 8.0 * kAccPerBlob), build_row_bins<R>(bp, s->nb, s->qh, bins, sb));
  if (fork) cudaEventRecord(s->ev_join, sb);
  // step 2: unperturbed fluid solve (Eq. provisional_step-1)
  ICM_STAGE("rhs", 4 * F, explicit_rhs<R>(gp, v, adv, work, s->step_dev, s->hist_dev, st));
  if (fork) cudaStreamWaitEvent(st, s->ev_join, 0);
  if (drift) ICM_STAGE("drift", 2 * gath + nb * 32, blob_spread_drift<R>(bp, bs, work, st));
  if (fused) {
    // The blob work of steps 2-9 runs inside the x passes of the three solves: the
    // spreads in the forward pass of the solve they feed, the interpolations in the
    // inverse pass of the solve whose output they read (Sec. III.C).
    double* acc1 = s->acc;                 // J v~
    double* acc2 = s->acc + 3 * s->nb;     // J dv~
    double* acc3 = s->acc + 6 * s->nb;     // J dv
    double* acc3l = s->acc + 9 * s->nb;    // J L dv (without 1/h^2)
    const double blobio = nb * (geob + 24.0);
    RowBlobs rb;
    rb.start = bins.start;
    rb.list = s->bin_list;
    rb.geo = s->geo;
    rb.p = bp;
    rb.vec = nullptr;
    rb.acc = nullptr;
    rb.acc_lap = nullptr;
    // forces spread in the first forward x pass
    auto passes = [&](const char* tag, const R* src, const double* vec, double a, double b, const double* k0,
                      R* dst, int mode, double* acc, double* acc_lap) {
      std::string t(tag);
      RowBlobs r = rb;
      r.vec = vec;
      r.acc = acc;
      r.acc_lap = acc_lap;
      if (xy) {
        ICM_STAGE((t + ".xy_fwd").c_str(), (src ? F : 0.0) + S + (vec ? blobio : 0.0),
                  fft_xy_forward<R>(fc, src, vec ? &r : nullptr, st));
      } else {
        if (vec)
          ICM_STAGE((t + ".x_fwd").c_str(), (src ? F : 0.0) + S + blobio, fft_x_forward_blobs<R>(fc, src, r, st));
        else
          ICM_STAGE((t + ".x_fwd").c_str(), F + S, fft_x_forward<R>(fc, src, st));
        ICM_STAGE((t + ".y_fwd").c_str(), 2 * S, fft_y<R>(fc, false, st));
      }
      ICM_STAGE((t + ".z_sym").c_str(), 2 * S, fft_z_symbol<R>(fc, a, b, k0, k0 ? k0scale : 0.0, st));
      ICM_STAGE((t + ".y_inv").c_str(), 2 * S, fft_y<R>(fc, true, st));
      const double out = mode == OUT_STORE ? F : (mode == OUT_ADD ? 2 * F : 0.0);
      ICM_STAGE((t + ".x_inv").c_str(), S + out + blobio, fft_x_inverse_blobs<R>(fc, dst, mode, r, st));
    };
    passes("rt1", work, fvec, s->rho / s->dt, 0.5 * s->eta, s->scal + SC_K0, v, OUT_STORE, acc1, nullptr);
    if (s->any_me) {
      // step 4: slip correction and momentum change (Eq. delta_u_nph_visc)
      ICM_STAGE("dp", nb * 264, blob_dp_from(bp, bs, acc1, st));
      // step 5: dv~ = m~_f / (rho (m~_f + m_e)) P S dp; only J dv~ is kept
      passes("rt2", nullptr, s->cdp, 1.0, 0.0, nullptr, v, OUT_NONE, acc2, nullptr);
      // steps 6 and 8 (blob side): source dp - m_e J dv~, u^{n+1}
      ICM_STAGE("inertial", nb * 168, blob_inertial_from(bp, bs, acc2, st));
      // step 6: (rho - dt/2 eta L) dv + dt grad dpi = S (dp - m_e J dv~); step 7: v = v~ + dv
      passes("rt3", nullptr, s->src, s->rho, 0.5 * s->dt * s->eta, s->scal + SC_SUMSRC, v, OUT_ADD, acc3, acc3l);
      // step 9 and the lagged slip term: J v^{n+1} = J v~ + J dv; with the end-of-step
      // scalars (the bookkeeping of scalars_after_step) in the same launch
      ICM_STAGE("finish", nb * 216, blob_finish_from(bp, bs, s->jvt, acc3, acc3l, true, st, s->step_dev, s->hist_dev));
    } else {
      ICM_STAGE("finish", nb * 144,
                blob_finish_from(bp, bs, nullptr, acc1, nullptr, false, st, s->step_dev, s->hist_dev));
    }
    return;
  }
  if (fvec) ICM_STAGE("spread", 2 * gath + nb * 48, blob_spread<R>(bp, s->nb, s->qh, fvec, work, st));
  if (grouped) return;
  solve("rt1", work, v, nullptr, OUT_STORE, s->rho / s->dt, 0.5 * s->eta, s->scal + SC_K0);
  if (s->any_me) {
    // step 4: slip correction and momentum change (Eq. delta_u_nph_visc)
    ICM_STAGE("dp", gath + nb * 136, blob_momentum_change<R>(bp, bs, v, st));
    // step 5: dv~ = m~_f / (rho (m~_f + m_e)) P S dp
    ICM_STAGE("zero", F, cudaMemsetAsync(work, 0, fbytes, st));
    ICM_STAGE("spread", 2 * gath + nb * 48, blob_spread<R>(bp, s->nb, s->qh, s->cdp, work, st));
    solve("rt2", work, work, nullptr, OUT_STORE, 1.0, 0.0, nullptr);
    // steps 6 and 8 (blob side): J dv~, source dp - m_e J dv~, u^{n+1}
    ICM_STAGE("inertial", gath + nb * 160, blob_inertial<R>(bp, bs, work, st));
    // step 6: (rho - dt/2 eta L) dv + dt grad dpi = S (dp - m_e J dv~); step 7: v = v~ + dv
    ICM_STAGE("zero", F, cudaMemsetAsync(work, 0, fbytes, st));
    ICM_STAGE("spread", 2 * gath + nb * 48, blob_spread<R>(bp, s->nb, s->qh, s->src, work, st));
    solve("rt3", work, v, work, OUT_ADD_AND_STORE2, s->rho, 0.5 * s->dt * s->eta, s->scal + SC_SUMSRC);
    // step 9 and the lagged slip term
    ICM_STAGE("finish", gath + nb * 3.0 * w3l * sizeof(R) + nb * 144, blob_finish<R>(bp, bs, v, work, true, st));
  } else {
    ICM_STAGE("finish", gath + nb * 144, blob_finish<R>(bp, bs, v, nullptr, false, st));
  }
  ICM_STAGE("scalars", 0, scalars_after_step(s->scal, s->dt, s->rho, dvf, s->any_me, s->step_dev, s->hist_dev, st));
}
#undef ICM_STAGE

// Process-wide table of tuned plans (icm_autotune), keyed by what the speed of a step
// depends on.
std::mutex g_plan_mu;
std::map<std::string, icm_plan> g_plans;

std::string plan_key(const icm_sim* s) {
  int bucket = 0;
  while ((1ll << bucket) < s->nb + 1) ++bucket;
  char buf[160];
  snprintf(buf, sizeof(buf), "%d,%d,%d,%d,%d,%d,%d,%d", s->nx, s->ny, s->nz, s->prec, s->kernel, s->flags, bucket,
           s->any_me ? 1 : 0);
  return buf;
}

// The plan of a simulation nobody tuned: everything on (the 32 x 8 z split on FP32 z
// sides of 256).  The RHS blocks are persistent
// when every block of a full GPU (two per SM) gets at least 8 tile-planes of 32 x 16
// cells, which the single-simulation sweeps found fastest from 128^3 up; on smaller
// grids they march 8 z planes on short z sides, else 16.
icm_plan default_plan(const icm_sim* s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    nsm = 1;
  const long long tile_planes = (long long)((s->nx + 31) / 32) * ((s->ny + 15) / 16) * s->nz;
  const int kz = tile_planes >= 16LL * std::max(nsm, 1) ? 0 : (s->nz <= 48 ? 8 : 16);
  // the 32 x 8 z split measured 5% faster than 16 x 16 in the FP32 tensor-map z pass at 256
  const int zs = s->prec == 32 && s->nz == 256 ? 1 : 0;
  return icm_plan{1, 1, kz, 1, 0, zs};
}

// Before a capture: simulations without a plan of their own take the tuned plan of
// their key, if there is one.
void resolve_plan(icm_sim* s) {
  if (s->plan_src == 2) return;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find(plan_key(s));
  if (it != g_plans.end()) {
    s->plan = it->second;
    s->plan_src = 1;
  } else if (s->plan_src == 1) {
    s->plan = default_plan(s);
    s->plan_src = 0;
  }
}

icm_status capture_graph(icm_sim* s) {
  invalidate_graph(s);
  resolve_plan(s);
  cudaGraph_t graph = nullptr;
  ICM_CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  if (s->prec == 32)
    enqueue_step<float>(s, nullptr);
  else
    enqueue_step<double>(s, nullptr);
  const cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ICM_ECUDA, "graph capture of the step failed: %s", cudaGetErrorString(e));
  }
  const cudaError_t e2 = cudaGraphInstantiate(&s->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return fail(ICM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e2));
  s->graph_ok = true;
  return ICM_OK;
}

icm_status grow_blobs(icm_sim* s, long long need) {
  if (need <= s->cap) return ICM_OK;
  long long cap = s->cap > 0 ? s->cap : 64;
  while (cap < need) cap *= 2;
  const long long per = 13 * 3 + 2;  // 13 vector arrays, masses, the WCA cell list (ints)
  double* nbuf = (double*)dalloc(s, sizeof(double) * per * cap);
  if (!nbuf) return fail(ICM_ENOMEM, "device allocation of %lld blob slots failed", cap);
  ICM_CK(cudaMemsetAsync(nbuf, 0, sizeof(double) * per * cap, s->stream));
  double* arrs[13];
  for (int i = 0; i < 13; ++i) arrs[i] = nbuf + (size_t)i * 3 * cap;
  double* me = nbuf + (size_t)39 * cap;
  if (s->nb > 0) {
    double* old[13] = {s->q, s->qh, s->u, s->f, s->g, s->w0, s->w1, s->jvt, s->du, s->dp, s->cdp, s->src, s->fe};
    for (int i = 0; i < 13; ++i)
      ICM_CK(cudaMemcpyAsync(arrs[i], old[i], sizeof(double) * 3 * s->nb, cudaMemcpyDeviceToDevice, s->stream));
    ICM_CK(cudaMemcpyAsync(me, s->me, sizeof(double) * s->nb, cudaMemcpyDeviceToDevice, s->stream));
  }
  void* nbin = nullptr;
  if (s->fused) {
    nbin = dalloc(s, bin_blob_bytes(cap));
    if (!nbin) {
      ICM_CK(cudaStreamSynchronize(s->stream));
      dfree(s, nbuf);
      return fail(ICM_ENOMEM, "device allocation of the bins of %lld blob slots failed", cap);
    }
  }
  ICM_CK(cudaStreamSynchronize(s->stream));
  if (s->blob) dfree(s, s->blob);
  s->blob = nbuf;
  if (s->fused) {
    if (s->bin_blob) dfree(s, s->bin_blob);
    s->bin_blob = nbin;
    s->bin_list = (int*)nbin;
    s->geo = (unsigned char*)nbin + bin_list_bytes(cap);
    s->acc = (double*)((unsigned char*)s->geo + kGeoBytes * cap);
  }
  s->cap = cap;
  s->q = arrs[0]; s->qh = arrs[1]; s->u = arrs[2]; s->f = arrs[3]; s->g = arrs[4]; s->w0 = arrs[5];
  s->w1 = arrs[6]; s->jvt = arrs[7]; s->du = arrs[8]; s->dp = arrs[9]; s->cdp = arrs[10]; s->src = arrs[11];
  s->fe = arrs[12];
  s->cell_list = reinterpret_cast<int*>(nbuf + (size_t)40 * cap);
  s->me = me;
  return ICM_OK;
}

void wrap_host(double* p, long long n, const icm_sim* s) {
  const double L[3] = {s->nx * s->h, s->ny * s->h, s->nz * s->h};
  for (long long i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double x = p[3 * i + a];
      x -= L[a] * std::floor(x / L[a]);
      if (x >= L[a]) x -= L[a];
      if (x < 0) x += L[a];
      p[3 * i + a] = x;
    }
}

// host double[3N] -> device field of precision R (via a temporary double buffer)
icm_status upload_field(icm_sim* s, const double* host, void* dst) {
  const long long n = 3 * s->ncell;
  if (s->prec == 64) {
    ICM_CK(cudaMemcpyAsync(dst, host, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
    return ICM_OK;
  }
  Tmp t(s, sizeof(double) * n);
  if (!t.p) return fail(ICM_ENOMEM, "staging allocation failed");
  ICM_CK(cudaMemcpyAsync(t.p, host, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
  convert_from_double<float>((const double*)t.p, (float*)dst, n, s->stream);
  ICM_CK(cudaGetLastError());
  return ICM_OK;
}

icm_status download_field(icm_sim* s, const void* src, double* host) {
  const long long n = 3 * s->ncell;
  if (s->prec == 64) {
    ICM_CK(cudaMemcpyAsync(host, src, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    ICM_CK(cudaStreamSynchronize(s->stream));
    return ICM_OK;
  }
  Tmp t(s, sizeof(double) * n);
  if (!t.p) return fail(ICM_ENOMEM, "staging allocation failed");
  convert_to_double<float>((const float*)src, (double*)t.p, n, s->stream);
  ICM_CK(cudaGetLastError());
  ICM_CK(cudaMemcpyAsync(host, t.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  return ICM_OK;
}

icm_status recompute_pbar(icm_sim* s) {
  if (s->prec == 32)
    field_sums<float>((const float*)s->v, s->ncell, s->scal + SC_PBAR, s->partial, icm_sim::kPartials, s->stream);
  else
    field_sums<double>((const double*)s->v, s->ncell, s->scal + SC_PBAR, s->partial, icm_sim::kPartials, s->stream);
  ICM_CK(cudaGetLastError());
  double sums[3];
  ICM_CK(cudaMemcpyAsync(sums, s->scal + SC_PBAR, sizeof(sums), cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  const double m = s->rho * s->h * s->h * s->h;
  for (int a = 0; a < 3; ++a) sums[a] *= m;
  ICM_CK(cudaMemcpyAsync(s->scal + SC_PBAR, sums, sizeof(sums), cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  return ICM_OK;
}

// The status of device error bits err (already read back); clears them on the device.
icm_status device_error_status(icm_sim* s, int err) {
  if (err) {
    ICM_CK(cudaMemsetAsync(s->err_dev, 0, sizeof(int), s->stream));
    ICM_CK(cudaStreamSynchronize(s->stream));
    if (err & DEV_ERR_TIMEOUT) return fail(ICM_ETIMEOUT, "a bounded device-side wait gave up");
    if (err & DEV_ERR_INDEX) return fail(ICM_EINDEX, "a device-side index check failed (checked build)");
    if (err & DEV_ERR_NONFINITE) return fail(ICM_ENONFINITE, "a non-finite blob position or velocity appeared");
    return fail(ICM_ECFL, "a blob moved more than one cell in a step (|u| dt / h > 1)");
  }
  return ICM_OK;
}

icm_status check_device_errors(icm_sim* s) {
  int err = 0;
  ICM_CK(cudaMemcpyAsync(&err, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  return device_error_status(s, err);
}

// The host staging buffer, sized for the current blob capacity.
// The device side of the copy stream's I/O, sized for the current blob capacity: the
// forces' landing buffer [3 cap] and two read slots [6 cap + 8] each; the stream and its
// events on first use.
icm_status ensure_dstage(icm_sim* s) {
  if (!s->copy) {
    if (cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy_up, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      if (s->copy) cudaStreamDestroy(s->copy);
      s->copy = nullptr;
      s->copy_up = nullptr;
      return fail(ICM_ECUDA, "creation of the copy streams failed");
    }
    ICM_CK(cudaEventCreateWithFlags(&s->ev_fup, cudaEventDisableTiming));
    ICM_CK(cudaEventCreateWithFlags(&s->ev_fcons, cudaEventDisableTiming));
    for (auto& e : s->ev_snap) ICM_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (s->dfstage && s->dstage_cap == s->cap) return ICM_OK;
  ICM_CK(cudaStreamSynchronize(s->stream));
  ICM_CK(cudaStreamSynchronize(s->copy));
  ICM_CK(cudaStreamSynchronize(s->copy_up));
  if (s->dfstage) dfree(s, s->dfstage);
  s->dfstage = nullptr;
  s->dsnap = nullptr;
  const size_t slot = 6 * (size_t)s->cap + 8;
  double* p = (double*)dalloc(s, sizeof(double) * (3 * (size_t)s->cap + 2 * slot));
  if (!p) return fail(ICM_ENOMEM, "no device memory for the copy stream's buffers");
  s->dfstage = p;
  s->dsnap = p + 3 * (size_t)s->cap;
  s->dstage_cap = s->cap;
  return ICM_OK;
}

// Layout (doubles): forces [3 cap]; then three read slots (the synchronous read's and the
// two of icm_read_begin), each positions [3 cap], velocities [3 cap], scalars [8]
// (momentum [3], step, error bits).
constexpr size_t kReadScalars = 8;
size_t read_slot_doubles(long long cap) { return 6 * (size_t)cap + kReadScalars; }
double* read_slot(icm_sim* s, int slot) { return s->hstage + 3 * (size_t)s->cap + slot * read_slot_doubles(s->cap); }

icm_status ensure_hstage(icm_sim* s) {
  if (s->hstage && s->hstage_cap == s->cap) return ICM_OK;
  ICM_CK(cudaStreamSynchronize(s->stream));
  if (s->hstage) cudaFreeHost(s->hstage);
  s->hstage = nullptr;
  s->hforce_pending = false;
  if (cudaMallocHost(&s->hstage, sizeof(double) * (3 * (size_t)s->cap + 3 * read_slot_doubles(s->cap))) !=
      cudaSuccess) {
    s->hstage = nullptr;
    cudaGetLastError();
    return fail(ICM_ENOMEM, "no page-locked host memory for the staging buffer");
  }
  s->hstage_cap = s->cap;
  if (!s->ev_hforce) ICM_CK(cudaEventCreateWithFlags(&s->ev_hforce, cudaEventDisableTiming));
  return ICM_OK;
}

}  // namespace

namespace {
template <typename R>
void enqueue_coupling(icm_sim* s, long long n, const double* qdev, const double* unit, double a, double b,
                      double* outdev) {
  const BlobParams bp = blob_params(s);
  const FftCtx<R> fc = fft_ctx<R>(s);
  R* work = (R*)s->work;
  const size_t fbytes = 3 * (size_t)s->ncell * sizeof(R);
  for (long long p = 0; p < n; ++p)
    for (int c = 0; c < 3; ++c) {
      cudaMemsetAsync(work, 0, fbytes, s->stream);
      blob_spread<R>(bp, 1, qdev + 3 * (n + p), unit + 3 * c, work, s->stream);
      spectral_solve<R>(fc, work, work, nullptr, OUT_STORE, a, b, nullptr, 0.0, s->stream);
      blob_interp<R>(bp, 1, qdev + 3 * p, work, false, outdev + 9 * p + 3 * c, s->stream);   // column c
    }
}
}  // namespace

// A device copy of everything a step changes (fields, blob arrays, scalars, counters),
// for the autotuner's trial steps.
struct StateCopy {
  icm_sim* s;
  size_t fbytes, bbytes;
  Tmp v, adv, blob, sc;
  explicit StateCopy(icm_sim* s_)
      : s(s_),
        fbytes(3 * (size_t)s_->ncell * s_->rsize()),
        bbytes(s_->blob ? sizeof(double) * (13 * 3 + 2) * (size_t)s_->cap : 0),
        v(s_, fbytes),
        adv(s_, fbytes),
        blob(s_, bbytes),
        sc(s_, sizeof(double) * SC_COUNT + 64) {}
  bool ok() const { return v.p && adv.p && blob.p && sc.p; }
  icm_status copy(bool save) {
    auto cp = [&](void* dev, void* keep, size_t n) -> cudaError_t {
      return n ? cudaMemcpyAsync(save ? keep : dev, save ? dev : keep, n, cudaMemcpyDeviceToDevice, s->stream)
               : cudaSuccess;
    };
    char* k = (char*)sc.p;
    ICM_CK(cp(s->v, v.p, fbytes));
    ICM_CK(cp(s->adv, adv.p, fbytes));
    ICM_CK(cp(s->blob, blob.p, bbytes));
    ICM_CK(cp(s->scal, k, sizeof(double) * SC_COUNT));
    ICM_CK(cp(s->step_dev, k + sizeof(double) * SC_COUNT, sizeof(long long)));
    ICM_CK(cp(s->hist_dev, k + sizeof(double) * SC_COUNT + 8, sizeof(int)));
    ICM_CK(cudaStreamSynchronize(s->stream));
    return ICM_OK;
  }
  icm_status save() { return copy(true); }
  icm_status restore() { return copy(false); }
};

extern "C" {

icm_status icm_set_default_allocator(icm_alloc_fn alloc, icm_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return fail(ICM_EINVAL, "allocator needs both alloc and free");
  g_alloc = alloc;
  g_free = release;
  g_actx = ctx;
  return ICM_OK;
}

const char* icm_last_error(void) { return g_err.c_str(); }

icm_status icm_create(const int32_t grid[3], double h, double rho, double eta, double kT, double dt, int32_t kernel,
                      uint64_t seed, int32_t precision, int32_t flags, void* cuda_stream, icm_sim** out) {
  if (!grid || !out) return fail(ICM_EINVAL, "grid and out must not be NULL");
  *out = nullptr;
  if (kernel != 3 && kernel != 4) return fail(ICM_EINVAL, "kernel must be 3 or 4, got %d", kernel);
  for (int a = 0; a < 3; ++a) {
    if (!side_ok(grid[a]) || grid[a] < 2 * kernel || grid[a] > kMaxSide)
      return fail(ICM_EINVAL, "grid side %d must be 2^a 3^b in [%d, %d]", grid[a], 2 * kernel, kMaxSide);
  }
  const double vals[5] = {h, rho, eta, kT, dt};
  for (double x : vals)
    if (!std::isfinite(x)) return fail(ICM_EINVAL, "non-finite parameter");
  if (h <= 0 || rho <= 0 || eta <= 0 || dt <= 0) return fail(ICM_EINVAL, "h, rho, eta and dt must be > 0");
  if (kT < 0) return fail(ICM_EINVAL, "kT must be >= 0");
  if (precision != 32 && precision != 64) return fail(ICM_EINVAL, "precision must be 32 or 64");
  if (flags & ~(ICM_FLAG_NO_ADVECTION | ICM_FLAG_SLIP_ZERO | ICM_FLAG_SLIP_FULL | ICM_FLAG_THERMAL_DRIFT))
    return fail(ICM_EINVAL, "unknown flag bits 0x%x", flags);
  if ((flags & ICM_FLAG_SLIP_ZERO) && (flags & ICM_FLAG_SLIP_FULL))
    return fail(ICM_EINVAL, "choose one slip correction");

  icm_sim* s = new icm_sim();
  s->nx = grid[0]; s->ny = grid[1]; s->nz = grid[2];
  s->ncell = (long long)s->nx * s->ny * s->nz;
  s->h = h; s->rho = rho; s->eta = eta; s->kT = kT; s->dt = dt;
  s->kernel = kernel; s->seed = seed; s->prec = precision; s->flags = flags;
  s->plan = default_plan(s);
  s->advection = !(flags & ICM_FLAG_NO_ADVECTION);
  s->slip = (flags & ICM_FLAG_SLIP_ZERO) ? 1 : ((flags & ICM_FLAG_SLIP_FULL) ? 2 : 0);
  s->alloc = g_alloc; s->release = g_free; s->actx = g_actx;
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return fail(ICM_ECUDA, "cudaStreamCreate failed");
    }
    s->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    icm_destroy(s);
    return fail(ICM_ECUDA, "creation of the auxiliary stream failed");
  }
  fft_prepare();
  grid_prepare();
  s->kx = s->nx / 2 + 1;
  s->kxp = (s->kx + 15) / 16 * 16;
  const size_t rs = s->rsize();
  const size_t fbytes = 3 * (size_t)s->ncell * rs;
  s->v = dalloc(s, fbytes);
  s->adv = dalloc(s, fbytes);
  s->work = dalloc(s, fbytes);
  s->spec = dalloc(s, 3 * (size_t)s->nz * s->ny * s->kxp * 2 * rs);
  s->scal = (double*)dalloc(s, sizeof(double) * SC_COUNT);
  s->step_dev = (long long*)dalloc(s, 256);
  s->hist_dev = (int*)dalloc(s, 256);
  s->err_dev = (int*)dalloc(s, 256);
  s->partial = (double*)dalloc(s, sizeof(double) * 3 * icm_sim::kPartials);
  if (!s->v || !s->adv || !s->work || !s->spec || !s->scal || !s->step_dev || !s->hist_dev || !s->err_dev ||
      !s->partial) {
    icm_destroy(s);
    return fail(ICM_ENOMEM, "device allocation of %.1f MB of grid state failed", (4.0 * fbytes) / 1e6);
  }
  icm_status st = ICM_OK;
  if ((st = build_axis(s, s->nx, true, s->kx, s->px, s->dx, s->ddx)) != ICM_OK ||
      (st = build_axis(s, s->ny, false, s->ny, s->py, s->dy, s->ddy)) != ICM_OK ||
      (st = build_axis(s, s->nz, false, s->nz, s->pz, s->dz, s->ddz)) != ICM_OK) {
    const std::string msg = g_err;
    icm_destroy(s);
    return fail(st, "%s", msg.c_str());
  }
  {
    int r1 = 0, r2 = 0;
    s->has_zalt = fft_split_z_alt(s->nz, r1, r2);
  }
  if (s->has_zalt && (st = build_axis(s, s->nz, false, s->nz, s->pz_alt, s->dz_alt, s->ddz_alt, true)) != ICM_OK) {
    const std::string msg = g_err;
    icm_destroy(s);
    return fail(st, "%s", msg.c_str());
  }
  s->has_zmap = make_zmap(s->zmap, s->spec, s->prec, s->kx, s->kxp, s->ny, s->nz);
  s->fused = fft_has_blob_passes(s->nx);
  if (s->fused) {
    s->nrowblk = (int)((s->ny * (long long)s->nz + 31) / 32);
    s->bin_idx = (int*)dalloc(s, sizeof(int) * (3 * (size_t)s->nrowblk + 1));
    if (!s->bin_idx) {
      icm_destroy(s);
      return fail(ICM_ENOMEM, "device allocation of the row-block bins failed");
    }
    cudaMemsetAsync(s->bin_idx, 0, sizeof(int) * (3 * (size_t)s->nrowblk + 1), s->stream);
  }
  cudaMemsetAsync(s->v, 0, fbytes, s->stream);
  cudaMemsetAsync(s->adv, 0, fbytes, s->stream);
  cudaMemsetAsync(s->work, 0, fbytes, s->stream);
  cudaMemsetAsync(s->scal, 0, sizeof(double) * SC_COUNT, s->stream);
  cudaMemsetAsync(s->step_dev, 0, 256, s->stream);
  cudaMemsetAsync(s->hist_dev, 0, 256, s->stream);
  cudaMemsetAsync(s->err_dev, 0, 256, s->stream);
  const cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    icm_destroy(s);
    return fail(ICM_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
  }
  *out = s;
  return ICM_OK;
}

void icm_destroy(icm_sim* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->copy) cudaStreamSynchronize(s->copy);
  if (s->copy_up) cudaStreamSynchronize(s->copy_up);
  if (s->aux) cudaStreamSynchronize(s->aux);
  invalidate_graph(s);
  while (!s->allocs.empty()) dfree(s, s->allocs.back().first);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  if (s->aux) cudaStreamDestroy(s->aux);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->ev_hforce) cudaEventDestroy(s->ev_hforce);
  for (cudaEvent_t e : s->ev_read)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : s->ev_snap)
    if (e) cudaEventDestroy(e);
  if (s->ev_fup) cudaEventDestroy(s->ev_fup);
  if (s->ev_fcons) cudaEventDestroy(s->ev_fcons);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->copy_up) cudaStreamDestroy(s->copy_up);
  if (s->hstage) cudaFreeHost(s->hstage);
  delete s;
}

icm_status icm_add_blobs(icm_sim* s, int64_t n, const double* pos, const double* vel, const double* excess_mass) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (n < 0) return fail(ICM_EINVAL, "n must be >= 0");
  if (n == 0) return ICM_OK;
  // a queued read returns the blobs that existed when it was queued
  if (s->read_pending > 0) return fail(ICM_EBUSY, "reads are pending (icm_read_finish them first)");
  if (!pos || !excess_mass) return fail(ICM_EINVAL, "pos and excess_mass are required");
  if (!finite_all(pos, 3 * n) || !finite_all(excess_mass, n) || (vel && !finite_all(vel, 3 * n)))
    return fail(ICM_EINVAL, "non-finite blob input");
  const double mtf = 1.5 * s->rho * blob_volume(s);
  for (int64_t i = 0; i < n; ++i)
    if (!(excess_mass[i] > -mtf)) return fail(ICM_EINVAL, "excess mass %g <= -m~_f = %g", excess_mass[i], -mtf);
  if (vel)
    for (int64_t i = 0; i < 3 * n; ++i)
      if (std::fabs(vel[i]) * s->dt > s->h) return fail(ICM_ECFL, "blob velocity %g gives |u| dt / h > 1", vel[i]);
  icm_status st = grow_blobs(s, s->nb + n);
  if (st != ICM_OK) return st;
  std::vector<double> p(pos, pos + 3 * n);
  wrap_host(p.data(), n, s);
  ICM_CK(cudaMemcpyAsync(s->q + 3 * s->nb, p.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaMemcpyAsync(s->qh + 3 * s->nb, p.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
  if (vel)
    ICM_CK(cudaMemcpyAsync(s->u + 3 * s->nb, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
  else
    ICM_CK(cudaMemsetAsync(s->u + 3 * s->nb, 0, sizeof(double) * 3 * n, s->stream));
  ICM_CK(cudaMemsetAsync(s->f + 3 * s->nb, 0, sizeof(double) * 3 * n, s->stream));
  ICM_CK(cudaMemsetAsync(s->g + 3 * s->nb, 0, sizeof(double) * 3 * n, s->stream));
  ICM_CK(cudaMemcpyAsync(s->me + s->nb, excess_mass, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  s->me_host.insert(s->me_host.end(), excess_mass, excess_mass + n);
  s->f_host.resize(3 * (s->nb + n), 0.0);
  s->nb += n;
  bool any = false;
  for (double m : s->me_host) any |= (m != 0.0);
  s->any_me = any;
  invalidate_graph(s);
  return ICM_OK;
}

icm_status icm_set_blob_forces(icm_sim* s, const double* force) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (s->nb == 0) return ICM_OK;
  if (!force) return fail(ICM_EINVAL, "force must not be NULL");
  icm_status st = ensure_hstage(s);
  if (st != ICM_OK) return st;
  if ((st = ensure_dstage(s)) != ICM_OK) return st;
  // the previous copy out of the staging slot must have passed before it is rewritten
  if (s->hforce_pending) ICM_CK(cudaEventSynchronize(s->ev_hforce));
  s->hforce_pending = false;
  // one pass: finiteness and the copy into the staging slot
  double* fs = s->hstage;
  const long long n3 = 3 * s->nb;
  bool any = false, finite = true;
  for (long long i = 0; i < n3; ++i) {
    const double x = force[i];
    finite &= std::isfinite(x);
    any |= x != 0.0;
    fs[i] = x;
  }
  if (!finite) return fail(ICM_EINVAL, "non-finite force");
  // up on the upload stream (beside the steps still queued), once the previous forces
  // have left the landing buffer; then into f on the simulation's stream, behind its steps
  ICM_CK(cudaStreamWaitEvent(s->copy_up, s->ev_fcons, 0));
  ICM_CK(cudaMemcpyAsync(s->dfstage, fs, sizeof(double) * n3, cudaMemcpyHostToDevice, s->copy_up));
  ICM_CK(cudaEventRecord(s->ev_hforce, s->copy_up));
  ICM_CK(cudaEventRecord(s->ev_fup, s->copy_up));
  s->hforce_pending = true;
  ICM_CK(cudaStreamWaitEvent(s->stream, s->ev_fup, 0));
  ICM_CK(cudaMemcpyAsync(s->f, s->dfstage, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s->stream));
  ICM_CK(cudaEventRecord(s->ev_fcons, s->stream));
  // FP64 compensated total force for the momentum bookkeeping
  rows_sum3(s->f, nullptr, s->nb, nullptr, s->scal + SC_SUMF, s->partial, icm_sim::kPartials, s->stream);
  ICM_CK(cudaGetLastError());
  if (any != s->any_force) {
    s->any_force = any;
    invalidate_graph(s);
  }
  // the caller's buffer has been copied when this returns
  return ICM_OK;
}

icm_status icm_set_blob_trap(icm_sim* s, double k, const double center[3]) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (!center) return fail(ICM_EINVAL, "center must not be NULL");
  if (!std::isfinite(k) || k < 0) return fail(ICM_EINVAL, "trap constant must be finite and >= 0");
  if (!finite_all(center, 3)) return fail(ICM_EINVAL, "non-finite trap center");
  s->trap_k = k;
  for (int a = 0; a < 3; ++a) s->trap_c[a] = center[a];
  invalidate_graph(s);
  return ICM_OK;
}

icm_status icm_set_blob_wca(icm_sim* s, double epsilon, double sigma) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (!std::isfinite(epsilon) || !std::isfinite(sigma) || epsilon < 0 || !(sigma > 0))
    return fail(ICM_EINVAL, "WCA needs epsilon >= 0 and sigma > 0, finite");
  const double rc = std::pow(2.0, 1.0 / 6.0) * sigma;
  const int n[3] = {s->nx, s->ny, s->nz};
  int nc[3];
  for (int a = 0; a < 3; ++a) {
    const double L = n[a] * s->h;
    if (epsilon > 0 && L < 2.0 * rc)
      return fail(ICM_EINVAL, "box side %g is shorter than twice the WCA cut-off %g", L, rc);
    nc[a] = std::max(1, std::min(64, (int)(L / rc)));
  }
  ICM_CK(cudaStreamSynchronize(s->stream));
  if (s->wca_idx) {
    dfree(s, s->wca_idx);
    s->wca_idx = nullptr;
  }
  s->wca_eps = epsilon;
  s->wca_sigma = sigma;
  if (epsilon > 0) {
    const size_t ncells = (size_t)nc[0] * nc[1] * nc[2];
    s->wca_idx = (int*)dalloc(s, sizeof(int) * (3 * ncells + 1));
    if (!s->wca_idx) {
      s->wca_eps = 0.0;
      return fail(ICM_ENOMEM, "device allocation of the WCA cell list failed");
    }
    ICM_CK(cudaMemsetAsync(s->wca_idx, 0, sizeof(int) * (3 * ncells + 1), s->stream));
    for (int a = 0; a < 3; ++a) s->wca_nc[a] = nc[a];
  }
  invalidate_graph(s);
  return ICM_OK;
}

icm_status icm_step(icm_sim* s, int64_t nsteps) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (nsteps < 0) return fail(ICM_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return ICM_OK;
  if (!s->graph_ok) {
    icm_status st = capture_graph(s);
    if (st != ICM_OK) return st;
  }
  for (int64_t i = 0; i < nsteps; ++i) ICM_CK(cudaGraphLaunch(s->gexec, s->stream));
  return ICM_OK;
}

icm_status icm_get_plan(const icm_sim* s, icm_plan* out) {
  if (!s || !out) return fail(ICM_EINVAL, "NULL argument");
  *out = s->plan;
  return ICM_OK;
}

icm_status icm_set_plan(icm_sim* s, const icm_plan* plan) {
  if (!s || !plan) return fail(ICM_EINVAL, "NULL argument");
  if (plan->rhs_kz != 0 && (plan->rhs_kz < 4 || plan->rhs_kz > 64))
    return fail(ICM_EINVAL, "rhs_kz must be 0 (persistent) or in 4..64");
  s->plan = icm_plan{plan->fused_blobs ? 1 : 0, plan->tma_z ? 1 : 0, plan->rhs_kz, plan->fork ? 1 : 0,
                     plan->fused_xy ? 1 : 0, plan->z_split ? 1 : 0};
  s->plan_src = 2;
  invalidate_graph(s);
  return ICM_OK;
}

icm_status icm_autotune(icm_sim* s, int32_t nsteps, icm_plan* chosen, double* ms_per_step) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (nsteps < 1) return fail(ICM_EINVAL, "nsteps must be >= 1");
  ICM_CK(cudaStreamSynchronize(s->stream));
  ICM_CK(cudaStreamSynchronize(s->aux));
  icm_status st = check_device_errors(s);
  if (st != ICM_OK) return st;
  StateCopy keep(s);
  if (!keep.ok()) return fail(ICM_ENOMEM, "no device memory for the autotuner's state copy");
  if ((st = keep.save()) != ICM_OK) return st;
  auto copy_state = [&](bool) -> icm_status { return keep.restore(); };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ICM_CK(cudaEventCreate(&e0));
  ICM_CK(cudaEventCreate(&e1));
  auto trial = [&](const icm_plan& p, double& ms) -> icm_status {
    s->plan = p;
    s->plan_src = 2;
    icm_status r = capture_graph(s);
    if (r != ICM_OK) return r;
    ICM_CK(cudaGraphLaunch(s->gexec, s->stream));   // warm-up
    ICM_CK(cudaEventRecord(e0, s->stream));
    for (int i = 0; i < nsteps; ++i) ICM_CK(cudaGraphLaunch(s->gexec, s->stream));
    ICM_CK(cudaEventRecord(e1, s->stream));
    ICM_CK(cudaStreamSynchronize(s->stream));
    float t = 0.0f;
    ICM_CK(cudaEventElapsedTime(&t, e0, e1));
    ms = t / nsteps;
    r = check_device_errors(s);
    const icm_status rs = copy_state(false);
    return r != ICM_OK ? r : rs;
  };
  icm_plan best = s->plan;
  double best_ms = 0.0;
  st = trial(best, best_ms);
  // one choice at a time, the others held at the best so far
  std::vector<std::pair<int icm_plan::*, std::vector<int>>> knobs;
  if (s->fused) knobs.push_back({&icm_plan::fused_blobs, {1, 0}});
  if (s->has_zmap) knobs.push_back({&icm_plan::tma_z, {1, 0}});
  knobs.push_back({&icm_plan::rhs_kz, {0, 8, 16, 32}});
  knobs.push_back({&icm_plan::fork, {1, 0}});
  if (fft_has_xy_passes(s->prec, s->nx, s->ny)) knobs.push_back({&icm_plan::fused_xy, {0, 1}});
  if (s->has_zalt) knobs.push_back({&icm_plan::z_split, {0, 1}});
  for (size_t k = 0; st == ICM_OK && k < knobs.size(); ++k)
    for (int val : knobs[k].second) {
      if (best.*(knobs[k].first) == val) continue;
      icm_plan p = best;
      p.*(knobs[k].first) = val;
      double ms = 0.0;
      if ((st = trial(p, ms)) != ICM_OK) break;
      if (ms < best_ms) {
        best = p;
        best_ms = ms;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ICM_OK) return st;
  s->plan = best;
  s->plan_src = 2;
  invalidate_graph(s);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[plan_key(s)] = best;
  }
  if (chosen) *chosen = best;
  if (ms_per_step) *ms_per_step = best_ms;
  return ICM_OK;
}

icm_status icm_sync(icm_sim* s) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  ICM_CK(cudaStreamSynchronize(s->stream));
  return check_device_errors(s);
}

icm_status icm_debug_wait_timeout(icm_sim* s, int64_t limit_ns) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (limit_ns < 1 || limit_ns > 2000000000ll) return fail(ICM_EINVAL, "limit_ns must be in [1, 2e9]");
  debug_wait_timeout(s->err_dev, (long long)limit_ns, s->stream);
  ICM_CK(cudaGetLastError());
  return ICM_OK;
}

icm_status icm_read_state(icm_sim* s, double* pos, double* vel, double* fluid_v, double momentum[3], int64_t* step) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  icm_status st = ensure_hstage(s);
  if (st != ICM_OK) return st;
  // every read goes into the page-locked staging buffer behind the queued work; one wait
  double* ps = read_slot(s, 0);
  double* us = ps + 3 * s->cap;
  double* sc = us + 3 * s->cap;   // total momentum [3], step, error bits
  const size_t bb = sizeof(double) * 3 * s->nb;
  if (pos && s->nb) ICM_CK(cudaMemcpyAsync(ps, s->q, bb, cudaMemcpyDeviceToHost, s->stream));
  if (vel && s->nb) ICM_CK(cudaMemcpyAsync(us, s->u, bb, cudaMemcpyDeviceToHost, s->stream));
  if (momentum) {
    // P = (FP64 fluid bookkeeping) + sum_i m_e,i u_i, compensated, on the device
    rows_sum3(s->u, s->me, s->nb, s->scal + SC_PBAR, s->scal + SC_PTOT, s->partial, icm_sim::kPartials, s->stream);
    ICM_CK(cudaGetLastError());
    ICM_CK(cudaMemcpyAsync(sc, s->scal + SC_PTOT, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  }
  ICM_CK(cudaMemcpyAsync(sc + 3, s->step_dev, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaMemcpyAsync(sc + 4, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  int err = 0;
  long long stp = 0;
  memcpy(&err, sc + 4, sizeof(int));
  memcpy(&stp, sc + 3, sizeof(long long));
  const icm_status dev = device_error_status(s, err);
  if (fluid_v) {
    st = download_field(s, s->v, fluid_v);
    if (st != ICM_OK) return st;
  }
  if (pos && s->nb) memcpy(pos, ps, bb);
  if (vel && s->nb) memcpy(vel, us, bb);
  if (momentum) memcpy(momentum, sc, 3 * sizeof(double));
  if (step) *step = stp;
  return dev;
}

// Queue the blob-state reads of icm_read_state (without the fluid) into the next free
// slot behind the queued work, and an event after them; no wait.
icm_status icm_read_begin(icm_sim* s) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (s->read_pending >= icm_sim::kReadSlots) return fail(ICM_EBUSY, "two reads are pending already");
  icm_status st = ensure_hstage(s);
  if (st != ICM_OK) return st;
  if ((st = ensure_dstage(s)) != ICM_OK) return st;
  const int slot = (s->read_head + s->read_pending) % icm_sim::kReadSlots;
  if (!s->ev_read[slot]) ICM_CK(cudaEventCreateWithFlags(&s->ev_read[slot], cudaEventDisableTiming));
  // on the simulation's stream: the momentum sum and one gather of the state into the
  // slot's device block; on the copy stream: that block down to the slot's staging area,
  // beside the steps queued after this call (the slot was last read by a finished read)
  double* dslot = s->dsnap + slot * (6 * (size_t)s->cap + 8);
  rows_sum3(s->u, s->me, s->nb, s->scal + SC_PBAR, s->scal + SC_PTOT, s->partial, icm_sim::kPartials, s->stream);
  blob_snapshot(s->q, s->u, s->nb, s->scal + SC_PTOT, s->step_dev, s->err_dev, dslot, s->stream);
  ICM_CK(cudaGetLastError());
  ICM_CK(cudaEventRecord(s->ev_snap[slot], s->stream));
  ICM_CK(cudaStreamWaitEvent(s->copy, s->ev_snap[slot], 0));
  ICM_CK(cudaMemcpyAsync(read_slot(s, 1 + slot), dslot, sizeof(double) * (6 * (size_t)s->nb + 5),
                         cudaMemcpyDeviceToHost, s->copy));
  ICM_CK(cudaEventRecord(s->ev_read[slot], s->copy));
  ++s->read_pending;
  return ICM_OK;
}

// Wait for the oldest queued read and copy it out.
icm_status icm_read_finish(icm_sim* s, double* pos, double* vel, double momentum[3], int64_t* step) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (s->read_pending == 0) return fail(ICM_EINVAL, "no read is pending (icm_read_begin)");
  const int slot = s->read_head;
  ICM_CK(cudaEventSynchronize(s->ev_read[slot]));
  s->read_head = (s->read_head + 1) % icm_sim::kReadSlots;
  --s->read_pending;
  // the slot holds positions [3 nb], velocities [3 nb], momentum [3], step, error bits
  const double* ps = read_slot(s, 1 + slot);
  const double* us = ps + 3 * s->nb;
  const double* sc = us + 3 * s->nb;
  long long errl = 0, stp = 0;
  memcpy(&errl, sc + 4, sizeof(long long));
  memcpy(&stp, sc + 3, sizeof(long long));
  const int err = (int)errl;
  const size_t bb = sizeof(double) * 3 * s->nb;
  if (pos && s->nb) memcpy(pos, ps, bb);
  if (vel && s->nb) memcpy(vel, us, bb);
  if (momentum) memcpy(momentum, sc, 3 * sizeof(double));
  if (step) *step = stp;
  return device_error_status(s, err);
}

icm_status icm_write_state(icm_sim* s, const double* pos, const double* vel, const double* fluid_v,
                           const double* adv_prev, const double* slip_g, int64_t step) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  if (!fluid_v || (s->nb > 0 && (!pos || !vel))) return fail(ICM_EINVAL, "pos, vel and fluid_v are required");
  if (step < 0) return fail(ICM_EINVAL, "step must be >= 0");
  const long long n3 = 3 * s->ncell;
  if (!finite_all(fluid_v, n3) || (adv_prev && !finite_all(adv_prev, n3)) ||
      (s->nb && (!finite_all(pos, 3 * s->nb) || !finite_all(vel, 3 * s->nb))) ||
      (slip_g && !finite_all(slip_g, 3 * s->nb)))
    return fail(ICM_EINVAL, "non-finite state");
  icm_status st = upload_field(s, fluid_v, s->v);
  if (st != ICM_OK) return st;
  if (adv_prev) {
    if ((st = upload_field(s, adv_prev, s->adv)) != ICM_OK) return st;
  }
  const int hist = adv_prev ? 1 : 0;
  ICM_CK(cudaMemcpyAsync(s->hist_dev, &hist, sizeof(int), cudaMemcpyHostToDevice, s->stream));
  const long long stp = step;
  ICM_CK(cudaMemcpyAsync(s->step_dev, &stp, sizeof(long long), cudaMemcpyHostToDevice, s->stream));
  if (s->nb) {
    std::vector<double> p(pos, pos + 3 * s->nb);
    wrap_host(p.data(), s->nb, s);
    ICM_CK(cudaMemcpyAsync(s->q, p.data(), sizeof(double) * 3 * s->nb, cudaMemcpyHostToDevice, s->stream));
    ICM_CK(cudaMemcpyAsync(s->u, vel, sizeof(double) * 3 * s->nb, cudaMemcpyHostToDevice, s->stream));
    if (slip_g)
      ICM_CK(cudaMemcpyAsync(s->g, slip_g, sizeof(double) * 3 * s->nb, cudaMemcpyHostToDevice, s->stream));
    else
      ICM_CK(cudaMemsetAsync(s->g, 0, sizeof(double) * 3 * s->nb, s->stream));
  }
  ICM_CK(cudaMemsetAsync(s->err_dev, 0, sizeof(int), s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  return recompute_pbar(s);
}

icm_status icm_read_aux(icm_sim* s, double* adv_prev, double* slip_g, int32_t* has_history) {
  if (!s) return fail(ICM_EINVAL, "NULL simulation");
  ICM_CK(cudaStreamSynchronize(s->stream));
  if (adv_prev) {
    const icm_status st = download_field(s, s->adv, adv_prev);
    if (st != ICM_OK) return st;
  }
  if (slip_g && s->nb)
    ICM_CK(cudaMemcpyAsync(slip_g, s->g, sizeof(double) * 3 * s->nb, cudaMemcpyDeviceToHost, s->stream));
  int hist = 0;
  ICM_CK(cudaMemcpyAsync(&hist, s->hist_dev, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  if (has_history) *has_history = hist;
  return ICM_OK;
}

icm_status icm_profile_steps(icm_sim* s, int64_t nsteps, int32_t max_stages, int32_t* nstages, char* names,
                             double* ms, double* bytes) {
  if (!s || nsteps < 1 || max_stages < 1 || !nstages || !names || !ms || !bytes)
    return fail(ICM_EINVAL, "bad arguments");
  ICM_CK(cudaStreamSynchronize(s->stream));
  Prof prof;
  for (int64_t i = 0; i < nsteps; ++i) {
    if (s->prec == 32)
      enqueue_step<float>(s, &prof);
    else
      enqueue_step<double>(s, &prof);
    ICM_CK(cudaGetLastError());
    ICM_CK(cudaStreamSynchronize(s->stream));
    prof.collect();
  }
  const int n = (int)std::min<size_t>(prof.e.size(), (size_t)max_stages);
  for (int i = 0; i < n; ++i) {
    memset(names + 32 * i, 0, 32);
    strncpy(names + 32 * i, prof.e[i].name.c_str(), 31);
    ms[i] = prof.e[i].ms;
    bytes[i] = prof.e[i].bytes;
  }
  *nstages = n;
  return check_device_errors(s);
}

icm_status icm_peak_fma(int32_t precision, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s) return fail(ICM_EINVAL, "flops_per_s must not be NULL");
  if (precision != 32 && precision != 64) return fail(ICM_EINVAL, "precision must be 32 or 64");
  // about 40 ms of FMA work at each precision's rate on a GB300
  const int iters = precision == 64 ? 2048 : 65536;
  const double r = fma_rate(precision, iters, 8, (cudaStream_t)cuda_stream, nullptr);
  if (!(r > 0.0)) return fail(ICM_ECUDA, "the FMA-chain kernel failed");
  *flops_per_s = r;
  return ICM_OK;
}

icm_status icm_kernel_volume(int32_t kernel, double h, double* volume) {
  if (volume == nullptr) return fail(ICM_EINVAL, "volume must not be NULL");
  if (kernel != 3 && kernel != 4) return fail(ICM_EINVAL, "kernel must be 3 or 4");
  if (!(h > 0.0) || !std::isfinite(h)) return fail(ICM_EINVAL, "h must be finite and > 0");
  const double q = kernel_sum_sq(kernel);
  *volume = h * h * h / (q * q * q);
  return ICM_OK;
}

int64_t icm_num_blobs(const icm_sim* s) { return s ? s->nb : -1; }
int64_t icm_device_bytes(const icm_sim* s) { return s ? s->bytes : -1; }

// ---------------------------------------------------------------------------
// Operator-level entry points
// ---------------------------------------------------------------------------

icm_status icm_op_interpolate(icm_sim* s, int64_t nb, const double* pos, const double* fluid_v, double* out) {
  if (!s || nb < 0 || (nb > 0 && (!pos || !fluid_v || !out))) return fail(ICM_EINVAL, "bad arguments");
  if (nb == 0) return ICM_OK;
  std::vector<double> p(pos, pos + 3 * nb);
  wrap_host(p.data(), nb, s);
  Tmp dq(s, sizeof(double) * 3 * nb), dout(s, sizeof(double) * 3 * nb);
  if (!dq.p || !dout.p) return fail(ICM_ENOMEM, "allocation failed");
  icm_status st = upload_field(s, fluid_v, s->work);
  if (st != ICM_OK) return st;
  ICM_CK(cudaMemcpyAsync(dq.p, p.data(), sizeof(double) * 3 * nb, cudaMemcpyHostToDevice, s->stream));
  const BlobParams bp = blob_params(s);
  if (s->prec == 32)
    blob_interp<float>(bp, nb, (const double*)dq.p, (const float*)s->work, false, (double*)dout.p, s->stream);
  else
    blob_interp<double>(bp, nb, (const double*)dq.p, (const double*)s->work, false, (double*)dout.p, s->stream);
  ICM_CK(cudaGetLastError());
  ICM_CK(cudaMemcpyAsync(out, dout.p, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  return ICM_OK;
}

icm_status icm_op_interpolate_laplacian(icm_sim* s, int64_t nb, const double* pos, const double* fluid_v,
                                        double* out) {
  if (!s || nb < 0 || (nb > 0 && (!pos || !fluid_v || !out))) return fail(ICM_EINVAL, "bad arguments");
  if (nb == 0) return ICM_OK;
  std::vector<double> p(pos, pos + 3 * nb);
  wrap_host(p.data(), nb, s);
  Tmp dq(s, sizeof(double) * 3 * nb), dout(s, sizeof(double) * 3 * nb);
  if (!dq.p || !dout.p) return fail(ICM_ENOMEM, "allocation failed");
  icm_status st = upload_field(s, fluid_v, s->work);
  if (st != ICM_OK) return st;
  ICM_CK(cudaMemcpyAsync(dq.p, p.data(), sizeof(double) * 3 * nb, cudaMemcpyHostToDevice, s->stream));
  const BlobParams bp = blob_params(s);
  if (s->prec == 32)
    blob_interp<float>(bp, nb, (const double*)dq.p, (const float*)s->work, true, (double*)dout.p, s->stream);
  else
    blob_interp<double>(bp, nb, (const double*)dq.p, (const double*)s->work, true, (double*)dout.p, s->stream);
  ICM_CK(cudaGetLastError());
  ICM_CK(cudaMemcpyAsync(out, dout.p, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  return ICM_OK;
}

icm_status icm_op_spread(icm_sim* s, int64_t nb, const double* pos, const double* force, double* out) {
  if (!s || nb < 0 || !out || (nb > 0 && (!pos || !force))) return fail(ICM_EINVAL, "bad arguments");
  std::vector<double> p(pos ? pos : (const double*)nullptr, pos ? pos + 3 * nb : (const double*)nullptr);
  wrap_host(p.data(), nb, s);
  Tmp dq(s, sizeof(double) * 3 * (nb + 1)), df(s, sizeof(double) * 3 * (nb + 1));
  if (!dq.p || !df.p) return fail(ICM_ENOMEM, "allocation failed");
  ICM_CK(cudaMemsetAsync(s->work, 0, 3 * (size_t)s->ncell * s->rsize(), s->stream));
  if (nb > 0) {
    ICM_CK(cudaMemcpyAsync(dq.p, p.data(), sizeof(double) * 3 * nb, cudaMemcpyHostToDevice, s->stream));
    ICM_CK(cudaMemcpyAsync(df.p, force, sizeof(double) * 3 * nb, cudaMemcpyHostToDevice, s->stream));
    const BlobParams bp = blob_params(s);
    if (s->prec == 32)
      blob_spread<float>(bp, nb, (const double*)dq.p, (const double*)df.p, (float*)s->work, s->stream);
    else
      blob_spread<double>(bp, nb, (const double*)dq.p, (const double*)df.p, (double*)s->work, s->stream);
    ICM_CK(cudaGetLastError());
  }
  return download_field(s, s->work, out);
}

icm_status icm_op_spectral_solve(icm_sim* s, double a, double b, const double* rhs, double* out) {
  if (!s || !rhs || !out) return fail(ICM_EINVAL, "bad arguments");
  if (!(a >= 0) || !(b >= 0) || !(a + b > 0) || !std::isfinite(a) || !std::isfinite(b))
    return fail(ICM_EINVAL, "need a >= 0, b >= 0, a + b > 0");
  icm_status st = upload_field(s, rhs, s->work);
  if (st != ICM_OK) return st;
  if (s->prec == 32)
    spectral_solve<float>(fft_ctx<float>(s), (const float*)s->work, (float*)s->work, nullptr, OUT_STORE, a, b, nullptr,
                          0.0, s->stream);
  else
    spectral_solve<double>(fft_ctx<double>(s), (const double*)s->work, (double*)s->work, nullptr, OUT_STORE, a, b,
                           nullptr, 0.0, s->stream);
  ICM_CK(cudaGetLastError());
  return download_field(s, s->work, out);
}

icm_status icm_op_coupling(icm_sim* s, int64_t n, const double* qi, const double* qj, double a, double b,
                           double* out) {
  if (!s || n < 0 || (n > 0 && (!qi || !qj || !out))) return fail(ICM_EINVAL, "bad arguments");
  if (!(a >= 0) || !(b >= 0) || !(a + b > 0) || !std::isfinite(a) || !std::isfinite(b))
    return fail(ICM_EINVAL, "need a >= 0, b >= 0, a + b > 0");
  if (n == 0) return ICM_OK;
  if (!finite_all(qi, 3 * n) || !finite_all(qj, 3 * n)) return fail(ICM_EINVAL, "non-finite position");
  std::vector<double> q(6 * (size_t)n);
  memcpy(q.data(), qi, sizeof(double) * 3 * n);
  memcpy(q.data() + 3 * n, qj, sizeof(double) * 3 * n);
  wrap_host(q.data(), 2 * n, s);
  const double unit[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  Tmp tq(s, sizeof(double) * q.size()), tu(s, sizeof(unit)), to(s, sizeof(double) * 9 * n);
  if (!tq.p || !tu.p || !to.p) return fail(ICM_ENOMEM, "allocation failed");
  ICM_CK(cudaMemcpyAsync(tq.p, q.data(), sizeof(double) * q.size(), cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaMemcpyAsync(tu.p, unit, sizeof(unit), cudaMemcpyHostToDevice, s->stream));
  if (s->prec == 32)
    enqueue_coupling<float>(s, n, (const double*)tq.p, (const double*)tu.p, a, b, (double*)to.p);
  else
    enqueue_coupling<double>(s, n, (const double*)tq.p, (const double*)tu.p, a, b, (double*)to.p);
  ICM_CK(cudaGetLastError());
  std::vector<double> colmajor(9 * (size_t)n);
  ICM_CK(cudaMemcpyAsync(colmajor.data(), to.p, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  for (long long p = 0; p < n; ++p)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) out[9 * p + 3 * r + c] = colmajor[9 * p + 3 * c + r];
  return ICM_OK;
}

icm_status icm_op_explicit_rhs(icm_sim* s, const double* fluid_v, const double* adv_prev, int64_t step,
                               double* out_rhs, double* out_adv) {
  if (!s || !fluid_v || !out_rhs || step < 0) return fail(ICM_EINVAL, "bad arguments");
  const size_t fb = 3 * (size_t)s->ncell * s->rsize();
  Tmp tv(s, fb), ta(s, fb), tc(s, 256);
  if (!tv.p || !ta.p || !tc.p) return fail(ICM_ENOMEM, "allocation failed");
  icm_status st = upload_field(s, fluid_v, tv.p);
  if (st != ICM_OK) return st;
  if (adv_prev) {
    if ((st = upload_field(s, adv_prev, ta.p)) != ICM_OK) return st;
  } else {
    ICM_CK(cudaMemsetAsync(ta.p, 0, fb, s->stream));
  }
  long long hdr[2] = {step, adv_prev ? 1 : 0};
  int hist = adv_prev ? 1 : 0;
  ICM_CK(cudaMemcpyAsync(tc.p, &hdr[0], sizeof(long long), cudaMemcpyHostToDevice, s->stream));
  ICM_CK(cudaMemcpyAsync((char*)tc.p + 64, &hist, sizeof(int), cudaMemcpyHostToDevice, s->stream));
  const GridParams gp = grid_params(s);
  if (s->prec == 32)
    explicit_rhs<float>(gp, (const float*)tv.p, (float*)ta.p, (float*)s->work, (const long long*)tc.p,
                        (const int*)((char*)tc.p + 64), s->stream);
  else
    explicit_rhs<double>(gp, (const double*)tv.p, (double*)ta.p, (double*)s->work, (const long long*)tc.p,
                         (const int*)((char*)tc.p + 64), s->stream);
  ICM_CK(cudaGetLastError());
  if ((st = download_field(s, s->work, out_rhs)) != ICM_OK) return st;
  if (out_adv) return download_field(s, ta.p, out_adv);
  return ICM_OK;
}

icm_status icm_op_stress_normals(icm_sim* s, int64_t step, double* out) {
  if (!s || !out || step < 0) return fail(ICM_EINVAL, "bad arguments");
  const size_t n6 = 6 * (size_t)s->ncell;
  Tmp t(s, n6 * s->rsize()), td(s, n6 * sizeof(double));
  if (!t.p || !td.p) return fail(ICM_ENOMEM, "allocation failed");
  const GridParams gp = grid_params(s);
  if (s->prec == 32) {
    stress_normals<float>(gp, step, (float*)t.p, s->stream);
    convert_to_double<float>((const float*)t.p, (double*)td.p, (long long)n6, s->stream);
  } else {
    stress_normals<double>(gp, step, (double*)td.p, s->stream);
  }
  ICM_CK(cudaGetLastError());
  ICM_CK(cudaMemcpyAsync(out, td.p, n6 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  ICM_CK(cudaStreamSynchronize(s->stream));
  return ICM_OK;
}

icm_status icm_op_philox(int64_t n, uint32_t ctr0, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3, uint32_t key0,
                         uint32_t key1, uint32_t* out) {
  if (n < 0 || (n > 0 && !out)) return fail(ICM_EINVAL, "bad arguments");
  if (n == 0) return ICM_OK;
  uint32_t* d = nullptr;
  ICM_CK(cudaMalloc(&d, sizeof(uint32_t) * 4 * n));
  philox_words(n, ctr0, ctr1, ctr2, ctr3, key0, key1, d, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(ICM_ECUDA, "philox kernel: %s", cudaGetErrorString(e));
  return ICM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched replicas: the steps of every member simulation captured into one graph
// as independent branches (fork on the batch stream, one chain per member stream,
// join back), so one graph launch advances all of them and the GPU runs the
// members' kernels side by side.
// ---------------------------------------------------------------------------
// With group solves on, members of the same grid (precision, sides and cell width,
// hence the same FFT tables and symbols) run each of the three solves of a step as
// one set of five launches over all of them, on a stream of the group: the members'
// stencil and blob work runs on their own streams between the solves.  This divides
// the number of FFT launches per step by the group size, for batches of many small
// grids whose launches are too short to fill the GPU.
struct icm_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<icm_sim*> sims;
  std::vector<long long> versions;
  std::vector<cudaEvent_t> events;  // fork, joins, ..., done (last)
  cudaGraphExec_t gexec = nullptr;
  bool ok = false;
  int grouped = 0;                     // 0 members apart, 1 group solves, 2 group solves + batched stages,
                                       // 3 the same with the blob work inside the group x passes
  long long kernels = -1;              // kernel nodes of the captured step graph
  std::vector<cudaStream_t> gstreams;  // one per group of the last capture
  void* reps = nullptr;                // device tables of the group solves
  void* stage_tables = nullptr;        // device member tables of the batched stages
  std::vector<void*> group_specs;      // spectra of the groups with the tensor-map z pass
};

namespace {

void batch_clear_graph(icm_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->ok = false;
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  b->events.clear();
  if (b->reps) cudaFree(b->reps);
  b->reps = nullptr;
  if (b->stage_tables) cudaFree(b->stage_tables);
  b->stage_tables = nullptr;
  for (void* p : b->group_specs) cudaFree(p);
  b->group_specs.clear();
}

// Whether every member can run in a batch of batched stages: one precision, register
// FFT passes along every axis (group solves), no pair forces and no thermal drift (the
// stages that have no batched form).
bool stages_possible(const icm_batch* b) {
  if (b->sims.empty()) return false;
  for (const icm_sim* s : b->sims) {
    if (s->prec != b->sims[0]->prec || !fft_has_group_passes(s->nx, s->ny, s->nz)) return false;
    if ((s->wca_eps > 0.0 && s->nb > 1) || ((s->flags & ICM_FLAG_THERMAL_DRIFT) && s->kT > 0.0 && s->nb > 0))
      return false;
  }
  return true;
}

struct alignas(64) ZMap {
  unsigned char bytes[128];
};

struct SolveGroup {
  std::vector<icm_sim*> members;  // every member: the first solve
  std::vector<icm_sim*> inertial; // members with excess mass: the second and third
  size_t table[3] = {0, 0, 0};    // offsets (in RepFft entries) of the three tables
  // batched stages: one buffer with every member's spectrum (member i in slot i) and the
  // tensor map of the z pass over all of them; null where the group has none
  unsigned char* spec = nullptr;
  size_t spec_bytes = 0;
  ZMap zmap;
};

bool same_grid(const icm_sim* a, const icm_sim* b) {
  return a->prec == b->prec && a->nx == b->nx && a->ny == b->ny && a->nz == b->nz && a->h == b->h;
}

RepFft rep_entry(const icm_sim* s, int rt) {
  RepFft r;
  const double dvf = s->h * s->h * s->h;
  const double k0mul = 1.0 / (s->rho * dvf) / (double)s->ncell;
  r.src = s->work;
  r.spec = s->spec;
  r.slot = -1;
  r.rb = nullptr;
  r.dst2 = nullptr;
  if (rt == 0) {        // (rho/dt - eta/2 L) v~ = rhs, projected
    r.dst = s->v;
    r.k0sum = s->scal + SC_K0;
    r.a = s->rho / s->dt;
    r.b = 0.5 * s->eta;
    r.k0mul = k0mul;
  } else if (rt == 1) { // P S dp
    r.dst = s->work;
    r.k0sum = nullptr;
    r.a = 1.0;
    r.b = 0.0;
    r.k0mul = 0.0;
  } else {              // (rho - dt/2 eta L) dv = S src, projected; v += dv
    r.dst = s->v;
    r.dst2 = s->work;
    r.k0sum = s->scal + SC_SUMSRC;
    r.a = s->rho;
    r.b = 0.5 * s->dt * s->eta;
    r.k0mul = k0mul;
  }
  return r;
}

// Solve rt (0-2) of a group.  With the blob work in its x passes (blobs): the spread of
// the table's vectors in the forward pass and the gathers in the inverse pass, which
// stores v~ (rt 0), nothing (rt 1) or adds dv to v (rt 2).  Without: the spread sources
// are in the work fields and the inverse pass stores v~, dv~ or v += dv and dv.
template <typename R>
void group_solve(const SolveGroup& g, const RepFft* reps, int rt, bool blobs, cudaStream_t st) {
  const std::vector<icm_sim*>& m = rt == 0 ? g.members : g.inertial;
  const int mode = blobs ? (rt == 0 ? OUT_STORE : (rt == 1 ? OUT_NONE : OUT_ADD))
                         : (rt == 2 ? OUT_ADD_AND_STORE2 : OUT_STORE);
  spectral_solve_group<R>(fft_ctx<R>(m[0]), reps + g.table[rt], (int)m.size(), mode, st,
                          g.spec ? g.zmap.bytes : nullptr, blobs);
}

// The step of every member as batched stages: each stage of the per-member sequence
// (scalars, predictor, right-hand side, spreads, momentum change, inertial update,
// finish) is one launch over all members, found through device member tables; the
// three solves are group solves, one set of launches per grid, the groups side by side
// on their own streams.  Members with excess mass take part in the second and third
// solves and the stages between them.
template <typename R>
icm_status batch_capture_stages(icm_batch* b) {
  const size_t n = b->sims.size();
  // groups: members on the same grid (a group may hold one member)
  std::vector<SolveGroup> groups;
  for (icm_sim* s : b->sims) {
    size_t gi = 0;
    while (gi < groups.size() && !same_grid(groups[gi].members[0], s)) ++gi;
    if (gi == groups.size()) groups.emplace_back();
    groups[gi].members.push_back(s);
    if (s->any_me) groups[gi].inertial.push_back(s);
  }
  // Groups on a z side of the tensor-map z pass (with the plan's choice of it) put their
  // members' spectra side by side in one buffer, so that one tensor map covers every
  // member and the persistent z pass walks all of their tiles; the members' own spectra
  // stay unused while the batch runs.  Below z side 96 the one-block-per-tile z pass
  // keeps more blocks per SM and ran faster over a group; without room for the buffer
  // the group keeps it too.
  for (SolveGroup& g : groups) {
    const icm_sim* s0 = g.members[0];
    if (!s0->plan.tma_z || !s0->has_zmap || s0->nz < 96) continue;
    g.spec_bytes = 3 * (size_t)s0->nz * s0->ny * s0->kxp * 2 * s0->rsize();
    void* buf = nullptr;
    if (cudaMalloc(&buf, g.spec_bytes * g.members.size()) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (!make_zmap(g.zmap.bytes, buf, s0->prec, s0->kx, s0->kxp, s0->ny, s0->nz, 3 * (int)g.members.size())) {
      cudaFree(buf);
      continue;
    }
    b->group_specs.push_back(buf);
    g.spec = (unsigned char*)buf;
  }
  // grouped = 3: the blob work of the solves inside the group x passes, as in a single
  // simulation's fused step, when every member can (register x side with row bins, and
  // blobs); otherwise separate spread and gather launches.
  bool blobs = b->grouped == 3;
  for (const icm_sim* s : b->sims) blobs = blobs && s->fused && s->nb > 0;
  std::vector<RepFft> reps_host;
  std::vector<RowBlobs> rbs_host;   // parallel to reps_host (blobs)
  for (SolveGroup& g : groups)
    for (int rt = 0; rt < 3; ++rt) {
      g.table[rt] = reps_host.size();
      for (icm_sim* m : rt == 0 ? g.members : g.inertial) {
        RepFft r = rep_entry(m, rt);
        r.rb = nullptr;
        if (g.spec) {
          const int slot = (int)(std::find(g.members.begin(), g.members.end(), m) - g.members.begin());
          r.spec = g.spec + (size_t)slot * g.spec_bytes;
          r.slot = slot;
        }
        if (blobs) {
          const RowBins bn = row_bins(m);
          RowBlobs w;
          w.start = bn.start;
          w.list = bn.list;
          w.geo = bn.geo;
          w.p = blob_params(m);
          const long long nb = m->nb;
          if (rt == 0) {          // forces spread; J v~ gathered
            w.vec = m->trap_k != 0.0 ? m->fe : (m->any_force ? m->f : nullptr);
            w.acc = m->acc;
            w.acc_lap = nullptr;
          } else if (rt == 1) {   // the weighted momentum change spread; J dv~ gathered
            r.src = nullptr;
            w.vec = m->cdp;
            w.acc = m->acc + 3 * nb;
            w.acc_lap = nullptr;
          } else {                // the source of the viscous correction spread; J dv, J L dv
            r.src = nullptr;
            r.dst2 = nullptr;
            w.vec = m->src;
            w.acc = m->acc + 6 * nb;
            w.acc_lap = m->acc + 9 * nb;
          }
          rbs_host.push_back(w);
        }
        reps_host.push_back(r);
      }
    }
  // member tables: all members and the inertial ones (blob stages), and the RHS table
  // (members with noise first, then those without)
  std::vector<BlobMember> all, inert;
  std::vector<int> mof_all, mof_in;
  std::vector<long long> zero_prefix{0};   // running 16-byte words of the inertial members' work
  for (icm_sim* s : b->sims) {
    BlobMember m;
    m.p = blob_params(s);
    m.s = blob_state(s);
    m.v = s->v;
    m.work = s->work;
    m.fvec = s->nb == 0 ? nullptr : (s->trap_k != 0.0 ? s->fe : (s->any_force ? s->f : nullptr));
    m.step_dev = s->step_dev;
    m.hist_dev = s->hist_dev;
    m.inertial = s->any_me ? 1 : 0;
    m.bins = row_bins(s);
    m.b0 = (long long)mof_all.size();
    for (long long i = 0; i < s->nb; ++i) mof_all.push_back((int)all.size());
    all.push_back(m);
    if (s->any_me) {
      m.b0 = (long long)mof_in.size();
      for (long long i = 0; i < s->nb; ++i) mof_in.push_back((int)inert.size());
      inert.push_back(m);
      zero_prefix.push_back(zero_prefix.back() + 3 * s->ncell * (long long)sizeof(R) / 16);
    }
  }
  std::vector<RhsMember<R>> rhs_noise, rhs_quiet;
  long long tot_noise = 0, tot_quiet = 0;
  for (icm_sim* s : b->sims) {
    RhsMember<R> r;
    r.g = grid_params(s);
    r.g.kz = 0;
    r.v = (const R*)s->v;
    r.adv = (R*)s->adv;
    r.rhs = (R*)s->work;
    r.step_dev = s->step_dev;
    r.hist_dev = s->hist_dev;
    long long& tot = s->kT > 0.0 ? tot_noise : tot_quiet;
    r.w0 = tot;
    tot += rhs_tile_planes(s->nx, s->ny, s->nz);
    (s->kT > 0.0 ? rhs_noise : rhs_quiet).push_back(r);
  }
  bool any_force = false;
  for (const BlobMember& m : all) any_force |= m.fvec != nullptr;
  // one device allocation for every table, each part 256-byte aligned
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_all = 0, o_in = o_all + al(all.size() * sizeof(BlobMember));
  const size_t o_mall = o_in + al(inert.size() * sizeof(BlobMember));
  const size_t o_min = o_mall + al(mof_all.size() * sizeof(int));
  const size_t o_rn = o_min + al(mof_in.size() * sizeof(int));
  const size_t o_rq = o_rn + al(rhs_noise.size() * sizeof(RhsMember<R>));
  const size_t o_reps = o_rq + al(rhs_quiet.size() * sizeof(RhsMember<R>));
  const size_t o_rbs = o_reps + al(reps_host.size() * sizeof(RepFft));
  const size_t o_zp = o_rbs + al(rbs_host.size() * sizeof(RowBlobs));
  const size_t total_bytes = o_zp + al(zero_prefix.size() * sizeof(long long)) + 256;
  ICM_CK(cudaMalloc(&b->stage_tables, total_bytes));
  unsigned char* base = (unsigned char*)b->stage_tables;
  for (size_t i = 0; i < rbs_host.size(); ++i) reps_host[i].rb = (const RowBlobs*)(base + o_rbs) + i;
  auto put = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpy(base + off, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  ICM_CK(put(o_all, all.data(), all.size() * sizeof(BlobMember)));
  ICM_CK(put(o_in, inert.data(), inert.size() * sizeof(BlobMember)));
  ICM_CK(put(o_mall, mof_all.data(), mof_all.size() * sizeof(int)));
  ICM_CK(put(o_min, mof_in.data(), mof_in.size() * sizeof(int)));
  ICM_CK(put(o_rn, rhs_noise.data(), rhs_noise.size() * sizeof(RhsMember<R>)));
  ICM_CK(put(o_rq, rhs_quiet.data(), rhs_quiet.size() * sizeof(RhsMember<R>)));
  ICM_CK(put(o_reps, reps_host.data(), reps_host.size() * sizeof(RepFft)));
  ICM_CK(put(o_rbs, rbs_host.data(), rbs_host.size() * sizeof(RowBlobs)));
  ICM_CK(put(o_zp, zero_prefix.data(), zero_prefix.size() * sizeof(long long)));
  const long long* d_zp = (const long long*)(base + o_zp);
  const BlobMember* d_all = (const BlobMember*)(base + o_all);
  const BlobMember* d_in = (const BlobMember*)(base + o_in);
  const int* d_mall = (const int*)(base + o_mall);
  const int* d_min = (const int*)(base + o_min);
  const RhsMember<R>* d_rn = (const RhsMember<R>*)(base + o_rn);
  const RhsMember<R>* d_rq = (const RhsMember<R>*)(base + o_rq);
  const RepFft* d_reps = (const RepFft*)(base + o_reps);
  while (b->gstreams.size() < groups.size()) {
    cudaStream_t gs = nullptr;
    ICM_CK(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    b->gstreams.push_back(gs);
  }
  // events (created before the capture): into and out of every group solve, and the
  // one icm_batch_step records after its launches
  const size_t need = 2 * groups.size() * 3 + 1;
  b->events.resize(need, nullptr);
  for (auto& ev : b->events) ICM_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  size_t next_event = 0;
  auto event = [&]() -> cudaEvent_t { return next_event < need ? b->events[next_event++] : nullptr; };
  const long long nb_all = (long long)mof_all.size(), nb_in = (long long)mof_in.size();
  const int n_all = (int)all.size(), n_in = (int)inert.size();
  cudaStream_t st = b->stream;
  auto solves = [&](int rt) {
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      const std::vector<icm_sim*>& m = rt == 0 ? groups[gi].members : groups[gi].inertial;
      cudaStream_t gs = b->gstreams[gi];
      cudaEvent_t in = event(), out = event();
      if (m.empty()) continue;
      cudaEventRecord(in, st);
      cudaStreamWaitEvent(gs, in, 0);
      group_solve<R>(groups[gi], d_reps, rt, blobs, gs);
      cudaEventRecord(out, gs);
      cudaStreamWaitEvent(st, out, 0);
    }
  };
  cudaGraph_t graph = nullptr;
  ICM_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  batch_scalars_before(d_all, n_all, st);
  batch_predict<R>(d_all, d_mall, nb_all, st);
  if (blobs) batch_bins<R>(d_all, d_mall, nb_all, n_all, st);
  batch_rhs<R>(d_rn, (int)rhs_noise.size(), tot_noise, true, st);
  batch_rhs<R>(d_rq, (int)rhs_quiet.size(), tot_quiet, false, st);
  if (any_force && !blobs) batch_spread<R>(d_all, d_mall, nb_all, BV_FORCE, st);
  solves(0);
  if (n_in > 0) {
    if (blobs) {
      batch_dp_from(d_in, d_min, nb_in, st);
    } else {
      batch_dp<R>(d_in, d_min, nb_in, st);
      batch_zero_work(d_in, d_zp, n_in, zero_prefix.back(), st);
      batch_spread<R>(d_in, d_min, nb_in, BV_CDP, st);
    }
  }
  solves(1);
  if (n_in > 0) {
    if (blobs) {
      batch_inertial_from(d_in, d_min, nb_in, st);
    } else {
      batch_inertial<R>(d_in, d_min, nb_in, st);
      batch_zero_work(d_in, d_zp, n_in, zero_prefix.back(), st);
      batch_spread<R>(d_in, d_min, nb_in, BV_SRC, st);
    }
  }
  solves(2);
  if (blobs)
    batch_finish_from(d_all, d_mall, nb_all, st);
  else
    batch_finish<R>(d_all, d_mall, nb_all, st);
  batch_scalars_after(d_all, n_all, st);
  event();   // recorded after the launches of icm_batch_step
  const cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ICM_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
  }
  (void)n;
  size_t nn = 0;
  b->kernels = 0;
  if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->kernels;
      }
  }
  const cudaError_t e2 = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return fail(ICM_ECUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e2));
  b->versions.clear();
  for (icm_sim* s : b->sims) b->versions.push_back(s->version);
  b->ok = true;
  return ICM_OK;
}

icm_status batch_capture(icm_batch* b) {
  batch_clear_graph(b);
  if (b->grouped >= 2 && stages_possible(b))
    return b->sims[0]->prec == 32 ? batch_capture_stages<float>(b) : batch_capture_stages<double>(b);
  const size_t n = b->sims.size();
  // groups of two or more members on a grid with register FFT passes
  std::vector<SolveGroup> groups;
  std::vector<int> group_of(n, -1);
  if (b->grouped) {
    std::vector<int> leader(n, -1);   // first member on the same grid
    for (size_t i = 0; i < n; ++i) {
      const icm_sim* s = b->sims[i];
      if (!fft_has_group_passes(s->nx, s->ny, s->nz)) continue;
      leader[i] = (int)i;
      for (size_t j = 0; j < i; ++j)
        if (leader[j] == (int)j && same_grid(b->sims[j], s)) {
          leader[i] = (int)j;
          break;
        }
    }
    std::map<int, int> gid;
    for (size_t i = 0; i < n; ++i) {
      if (leader[i] < 0 || std::count(leader.begin(), leader.end(), leader[i]) < 2) continue;
      auto it = gid.find(leader[i]);
      if (it == gid.end()) {
        it = gid.emplace(leader[i], (int)groups.size()).first;
        groups.emplace_back();
      }
      group_of[i] = it->second;
      groups[it->second].members.push_back(b->sims[i]);
      if (b->sims[i]->any_me) groups[it->second].inertial.push_back(b->sims[i]);
    }
  }
  if (!groups.empty()) {
    std::vector<RepFft> host;
    for (SolveGroup& g : groups)
      for (int rt = 0; rt < 3; ++rt) {
        g.table[rt] = host.size();
        for (icm_sim* m : rt == 0 ? g.members : g.inertial) host.push_back(rep_entry(m, rt));
      }
    ICM_CK(cudaMalloc(&b->reps, host.size() * sizeof(RepFft)));
    ICM_CK(cudaMemcpy(b->reps, host.data(), host.size() * sizeof(RepFft), cudaMemcpyHostToDevice));
    while (b->gstreams.size() < groups.size()) {
      cudaStream_t gs = nullptr;
      ICM_CK(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
      b->gstreams.push_back(gs);
    }
  }
  const RepFft* reps = (const RepFft*)b->reps;
  // events, created before the capture: fork, the edges into and out of every group
  // solve, the joins, and last the one icm_batch_step records after its launches
  size_t need = 1 + n + groups.size() + 1;
  for (const SolveGroup& g : groups) need += g.members.size() + 1 + 2 * (g.inertial.size() + (g.inertial.empty() ? 0 : 1));
  b->events.resize(need, nullptr);
  for (auto& ev : b->events) ICM_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  size_t next_event = 0;
  auto event = [&]() -> cudaEvent_t { return next_event < need ? b->events[next_event++] : nullptr; };
  auto edge = [&](cudaStream_t from, cudaStream_t to) {
    cudaEvent_t e = event();
    cudaEventRecord(e, from);
    cudaStreamWaitEvent(to, e, 0);
  };
  cudaGraph_t graph = nullptr;
  ICM_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaEvent_t fork = event();
  cudaEventRecord(fork, b->stream);
  for (size_t i = 0; i < n; ++i) {
    icm_sim* s = b->sims[i];
    cudaStreamWaitEvent(s->stream, fork, 0);
    const int seg = group_of[i] >= 0 ? 0 : -1;
    if (s->prec == 32)
      enqueue_step<float>(s, nullptr, seg);
    else
      enqueue_step<double>(s, nullptr, seg);
  }
  for (int rt = 0; rt < 3; ++rt) {
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      const SolveGroup& g = groups[gi];
      const std::vector<icm_sim*>& m = rt == 0 ? g.members : g.inertial;
      if (m.empty()) continue;
      cudaStream_t gs = b->gstreams[gi];
      for (icm_sim* s : m) edge(s->stream, gs);
      if (m[0]->prec == 32)
        group_solve<float>(g, reps, rt, false, gs);
      else
        group_solve<double>(g, reps, rt, false, gs);
      cudaEvent_t done = event();
      cudaEventRecord(done, gs);
      for (icm_sim* s : m) {
        cudaStreamWaitEvent(s->stream, done, 0);
        if (s->prec == 32)
          enqueue_step<float>(s, nullptr, rt + 1);
        else
          enqueue_step<double>(s, nullptr, rt + 1);
      }
    }
  }
  for (size_t i = 0; i < n; ++i) edge(b->sims[i]->stream, b->stream);
  for (size_t gi = 0; gi < groups.size(); ++gi) edge(b->gstreams[gi], b->stream);
  event();   // recorded after the launches of icm_batch_step
  const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ICM_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
  }
  if (next_event != need) {
    cudaGraphDestroy(graph);
    return fail(ICM_ECUDA, "batch capture used %zu of %zu events", next_event, need);
  }
  size_t nn = 0;
  b->kernels = 0;
  if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->kernels;
      }
  }
  const cudaError_t e2 = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return fail(ICM_ECUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e2));
  b->versions.clear();
  for (icm_sim* s : b->sims) b->versions.push_back(s->version);
  b->ok = true;
  return ICM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Serving: jobs queue on the host and are admitted first come first served while
// their device footprint fits the HBM budget and a slot is free.  Each active job
// replays its own step graph on its own stream, so the jobs' kernels overlap on the
// device; a pump enqueues a few steps per active job without waiting, and a job is
// retired (results read, memory freed) once the event recorded after its last step
// has completed.  Nothing blocks except reading a finished job's results.
// ---------------------------------------------------------------------------
struct icm_server {
  struct Job {
    int64_t id = 0;
    int32_t grid[3];
    double h, rho, eta, kT, dt;
    int32_t kernel, precision, flags;
    uint64_t seed;
    std::vector<double> pos, vel, me, force;
    int64_t nsteps = 0, enqueued = 0;
    int32_t state = 0;  // 0 waiting, 1 active, 2 done, 3 failed
    icm_sim* sim = nullptr;
    cudaEvent_t done = nullptr;
    int64_t bytes = 0;
    std::chrono::steady_clock::time_point t_submit, t_done;
    std::vector<double> out_pos, out_vel;
    double out_mom[3] = {0, 0, 0};
  };
  int64_t budget = 0, used = 0;
  int32_t max_active = 0;
  int64_t next_id = 1;
  std::deque<Job*> waiting;
  std::vector<Job*> active;
  std::map<int64_t, Job*> jobs;
};

extern "C" {

int64_t icm_estimate_device_bytes(const int32_t grid[3], int32_t precision, int64_t nblobs) {
  if (!grid || grid[0] < 1 || grid[1] < 1 || grid[2] < 1 || (precision != 32 && precision != 64) || nblobs < 0)
    return -1;
  const int64_t rs = precision == 32 ? 4 : 8;
  const int64_t ncell = (int64_t)grid[0] * grid[1] * grid[2];
  const int64_t kxp = (grid[0] / 2 + 1 + 15) / 16 * 16;
  int64_t cap = 64;
  while (cap < nblobs) cap *= 2;
  const int64_t fields = 3 * (3 * ncell * rs);
  const int64_t spec = 3 * (int64_t)grid[2] * grid[1] * kxp * 2 * rs;
  const int64_t tables = 3 * (int64_t)kMaxSide * (3 * 2 * rs + 4) + 16 * 256;
  const int64_t blobs = nblobs > 0 ? 41 * cap * 8 + (int64_t)bin_blob_bytes(cap) : 0;
  const int64_t bins = 4 * (3 * ((int64_t)grid[1] * grid[2] / 32 + 1) + 1);
  return fields + spec + tables + blobs + bins + 8 * 3 * 1024 + 4096;
}

icm_status icm_batch_create(void* cuda_stream, icm_batch** out) {
  if (!out) return fail(ICM_EINVAL, "out must not be NULL");
  icm_batch* b = new icm_batch();
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(ICM_ECUDA, "cudaStreamCreate failed");
    }
    b->own_stream = true;
  }
  *out = b;
  return ICM_OK;
}

icm_status icm_batch_set(icm_batch* b, int32_t n, icm_sim* const* sims) {
  if (!b || n < 0 || (n > 0 && !sims)) return fail(ICM_EINVAL, "bad arguments");
  std::vector<icm_sim*> v(sims, sims + n);
  for (size_t i = 0; i < v.size(); ++i) {
    if (!v[i]) return fail(ICM_EINVAL, "NULL simulation in batch");
    for (size_t j = 0; j < i; ++j)
      if (v[j] == v[i]) return fail(ICM_EINVAL, "a simulation appears twice in the batch");
  }
  if (b->stream) cudaStreamSynchronize(b->stream);
  b->sims = v;
  batch_clear_graph(b);
  return ICM_OK;
}

icm_status icm_batch_step(icm_batch* b, int64_t nsteps) {
  if (!b || nsteps < 0) return fail(ICM_EINVAL, "bad arguments");
  if (nsteps == 0 || b->sims.empty()) return ICM_OK;
  bool stale = !b->ok;
  for (size_t i = 0; !stale && i < b->sims.size(); ++i) stale = b->versions[i] != b->sims[i]->version;
  if (stale) {
    for (icm_sim* m : b->sims) {
      const icm_plan before = m->plan;
      resolve_plan(m);
      if (memcmp(&before, &m->plan, sizeof(icm_plan)) != 0) invalidate_graph(m);
    }
    // work already queued on the members' own streams must precede the batch
    for (icm_sim* s : b->sims) cudaStreamSynchronize(s->stream);
    const icm_status st = batch_capture(b);
    if (st != ICM_OK) return st;
  }
  for (int64_t i = 0; i < nsteps; ++i) ICM_CK(cudaGraphLaunch(b->gexec, b->stream));
  // later work on a member's own stream waits for the batch
  cudaEvent_t done = b->events.back();
  ICM_CK(cudaEventRecord(done, b->stream));
  for (icm_sim* s : b->sims) ICM_CK(cudaStreamWaitEvent(s->stream, done, 0));
  return ICM_OK;
}

icm_status icm_batch_set_grouped(icm_batch* b, int32_t grouped) {
  if (!b || grouped < 0 || grouped > 3) return fail(ICM_EINVAL, "bad arguments");
  if (b->grouped != grouped) {
    if (b->stream) ICM_CK(cudaStreamSynchronize(b->stream));
    b->grouped = grouped;
    batch_clear_graph(b);
  }
  return ICM_OK;
}

int32_t icm_batch_get_grouped(const icm_batch* b) { return b ? b->grouped : -1; }

int64_t icm_batch_kernels_per_step(const icm_batch* b) { return b && b->ok ? b->kernels : -1; }

icm_status icm_batch_autotune(icm_batch* b, int32_t nsteps) {
  if (!b || nsteps < 1) return fail(ICM_EINVAL, "bad arguments");
  if (b->sims.empty()) return ICM_OK;
  if (b->stream) ICM_CK(cudaStreamSynchronize(b->stream));
  // the members' states, restored after every trial
  std::vector<std::unique_ptr<StateCopy>> keep;
  for (icm_sim* m : b->sims) {
    ICM_CK(cudaStreamSynchronize(m->stream));
    keep.emplace_back(new StateCopy(m));
    if (!keep.back()->ok()) return fail(ICM_ENOMEM, "no device memory for the autotuner's state copy");
    const icm_status st = keep.back()->save();
    if (st != ICM_OK) return st;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ICM_CK(cudaEventCreate(&e0));
  ICM_CK(cudaEventCreate(&e1));
  // one plan for every member (what matters is how the members share the GPU)
  auto trial = [&](const icm_plan& p, int grouped, double& ms) -> icm_status {
    if (b->grouped != grouped) {
      b->grouped = grouped;
      batch_clear_graph(b);
    }
    for (icm_sim* m : b->sims) {
      m->plan = p;
      m->plan_src = 2;
      invalidate_graph(m);
    }
    icm_status r = icm_batch_step(b, 1);   // capture and warm-up
    if (r != ICM_OK) return r;
    ICM_CK(cudaEventRecord(e0, b->stream));
    if ((r = icm_batch_step(b, nsteps)) != ICM_OK) return r;
    ICM_CK(cudaEventRecord(e1, b->stream));
    ICM_CK(cudaStreamSynchronize(b->stream));
    float t = 0.0f;
    ICM_CK(cudaEventElapsedTime(&t, e0, e1));
    ms = t / nsteps;
    for (size_t i = 0; i < b->sims.size(); ++i) {
      ICM_CK(cudaStreamSynchronize(b->sims[i]->stream));
      if ((r = check_device_errors(b->sims[i])) != ICM_OK) return r;
      if ((r = keep[i]->restore()) != ICM_OK) return r;
    }
    return ICM_OK;
  };
  icm_plan best = icm_plan{1, 1, 16, 1, 0, 0};
  int best_grouped = 0;
  double best_ms = 0.0;
  icm_status st = trial(best, best_grouped, best_ms);
  const std::vector<std::pair<int icm_plan::*, std::vector<int>>> knobs = {
      {&icm_plan::fused_blobs, {1, 0}}, {&icm_plan::tma_z, {1, 0}}, {&icm_plan::rhs_kz, {0, 4, 8, 16, 32}},
      {&icm_plan::fork, {1, 0}}, {&icm_plan::fused_xy, {0, 1}}, {&icm_plan::z_split, {0, 1}}};
  for (size_t k = 0; st == ICM_OK && k < knobs.size(); ++k)
    for (int val : knobs[k].second) {
      if (best.*(knobs[k].first) == val) continue;
      icm_plan p = best;
      p.*(knobs[k].first) = val;
      double ms = 0.0;
      if ((st = trial(p, best_grouped, ms)) != ICM_OK) break;
      if (ms < best_ms) {
        best = p;
        best_ms = ms;
      }
    }
  // group solves (the members' own plans then matter only for the RHS z march)
  if (st == ICM_OK) {
    icm_plan p = best;
    p.fused_blobs = 0;
    p.tma_z = 0;
    p.fork = 0;
    double ms = 0.0;
    st = trial(p, 1, ms);
    if (st == ICM_OK && ms < best_ms) {
      best = p;
      best_grouped = 1;
      best_ms = ms;
      // the RHS march again: in grouped steps every member's RHS precedes the first
      // group solve, so its latency counts where before it overlapped other members
      for (int kz : {0, 4, 8, 16, 32}) {
        if (kz == best.rhs_kz || st != ICM_OK) continue;
        icm_plan q = best;
        q.rhs_kz = kz;
        double mq = 0.0;
        if ((st = trial(q, 1, mq)) == ICM_OK && mq < best_ms) {
          best = q;
          best_ms = mq;
        }
      }
    }
  }
  // batched stages: every per-member stage one launch over all members, the blob work
  // in separate launches (2) or inside the group x passes (3), with and without the
  // tensor-map z pass (the members' other plan choices do not enter: the stages have
  // their own launch shapes)
  if (stages_possible(b))
    for (int g : {2, 3})
      for (int tz : {1, 0}) {
        if (st != ICM_OK) break;
        icm_plan p = best;
        p.tma_z = tz;
        double ms = 0.0;
        st = trial(p, g, ms);
        if (st == ICM_OK && ms < best_ms) {
          best = p;
          best_grouped = g;
          best_ms = ms;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ICM_OK) return st;
  for (icm_sim* m : b->sims) {
    m->plan = best;
    m->plan_src = 2;
    invalidate_graph(m);
  }
  b->grouped = best_grouped;
  batch_clear_graph(b);
  return ICM_OK;
}

icm_status icm_batch_sync(icm_batch* b) {
  if (!b) return fail(ICM_EINVAL, "NULL batch");
  ICM_CK(cudaStreamSynchronize(b->stream));
  icm_status worst = ICM_OK;
  for (icm_sim* s : b->sims) {
    const icm_status st = check_device_errors(s);
    if (st != ICM_OK) worst = st;
  }
  return worst;
}

void icm_batch_destroy(icm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_clear_graph(b);
  for (cudaStream_t gs : b->gstreams) cudaStreamDestroy(gs);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

icm_status icm_server_create(int64_t hbm_budget_bytes, int32_t max_active, icm_server** out) {
  if (!out || hbm_budget_bytes <= 0 || max_active < 1) return fail(ICM_EINVAL, "bad arguments");
  icm_server* sv = new icm_server();
  sv->budget = hbm_budget_bytes;
  sv->max_active = max_active;
  *out = sv;
  return ICM_OK;
}

icm_status icm_server_submit(icm_server* sv, const icm_job_desc* d, int64_t* job_id) {
  if (!sv || !d || !job_id) return fail(ICM_EINVAL, "bad arguments");
  if (d->nsteps < 1 || d->nblobs < 0 || (d->nblobs > 0 && (!d->pos || !d->excess_mass)))
    return fail(ICM_EINVAL, "a job needs nsteps >= 1 and, with blobs, positions and masses");
  const int64_t est = icm_estimate_device_bytes(d->grid, d->precision, d->nblobs);
  if (est < 0) return fail(ICM_EINVAL, "invalid grid or precision");
  if (est > sv->budget) return fail(ICM_ENOMEM, "the job needs %lld bytes, more than the whole budget", (long long)est);
  auto* j = new icm_server::Job();
  j->id = sv->next_id++;
  memcpy(j->grid, d->grid, sizeof(j->grid));
  j->h = d->h; j->rho = d->rho; j->eta = d->eta; j->kT = d->kT; j->dt = d->dt;
  j->kernel = d->kernel; j->precision = d->precision; j->flags = d->flags; j->seed = d->seed;
  const int64_t n = d->nblobs;
  j->pos.assign(d->pos, d->pos + 3 * n);
  if (d->vel) j->vel.assign(d->vel, d->vel + 3 * n);
  j->me.assign(d->excess_mass, d->excess_mass + n);
  if (d->force) j->force.assign(d->force, d->force + 3 * n);
  j->nsteps = d->nsteps;
  j->bytes = est;
  j->t_submit = std::chrono::steady_clock::now();
  sv->waiting.push_back(j);
  sv->jobs[j->id] = j;
  *job_id = j->id;
  return ICM_OK;
}

icm_status icm_server_pump(icm_server* sv, int32_t steps_per_pump, int32_t* n_active, int32_t* n_waiting,
                           int32_t* n_finished) {
  if (!sv || steps_per_pump < 1) return fail(ICM_EINVAL, "bad arguments");
  int32_t finished = 0;
  // 1. retire jobs whose last step has completed on the device
  std::vector<icm_server::Job*> still;
  for (auto* j : sv->active) {
    if (j->enqueued < j->nsteps || cudaEventQuery(j->done) != cudaSuccess) {
      still.push_back(j);
      continue;
    }
    const int64_t nb = (int64_t)j->me.size();
    j->out_pos.resize(3 * nb);
    j->out_vel.resize(3 * nb);
    const icm_status rs = icm_read_state(j->sim, nb ? j->out_pos.data() : nullptr, nb ? j->out_vel.data() : nullptr,
                                         nullptr, j->out_mom, nullptr);
    j->state = rs == ICM_OK ? 2 : 3;
    j->t_done = std::chrono::steady_clock::now();
    sv->used -= j->bytes;
    cudaEventDestroy(j->done);
    j->done = nullptr;
    icm_destroy(j->sim);
    j->sim = nullptr;
    ++finished;
  }
  sv->active.swap(still);
  // 2. admission, first come first served, while the footprint fits
  while (!sv->waiting.empty() && (int32_t)sv->active.size() < sv->max_active) {
    icm_server::Job* j = sv->waiting.front();
    if (sv->used + j->bytes > sv->budget) break;
    icm_sim* s = nullptr;
    icm_status st = icm_create(j->grid, j->h, j->rho, j->eta, j->kT, j->dt, j->kernel, j->seed, j->precision, j->flags,
                               nullptr, &s);
    const int64_t nb = (int64_t)j->me.size();
    if (st == ICM_OK && nb > 0)
      st = icm_add_blobs(s, nb, j->pos.data(), j->vel.empty() ? nullptr : j->vel.data(), j->me.data());
    if (st == ICM_OK && nb > 0 && !j->force.empty()) st = icm_set_blob_forces(s, j->force.data());
    if (st == ICM_ENOMEM) {
      // out of device memory now: the job stays first in line for the next pump
      if (s) icm_destroy(s);
      break;
    }
    if (st == ICM_OK && cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming) != cudaSuccess) st = ICM_ECUDA;
    sv->waiting.pop_front();
    if (st != ICM_OK) {
      if (s) icm_destroy(s);
      j->state = 3;
      j->t_done = std::chrono::steady_clock::now();
      ++finished;
      continue;
    }
    j->sim = s;
    j->bytes = icm_device_bytes(s);
    sv->used += j->bytes;
    j->state = 1;
    sv->active.push_back(j);
  }
  // 3. enqueue the next steps of every active job on its own stream (no waiting)
  for (auto* j : sv->active) {
    const int64_t k = std::min<int64_t>(steps_per_pump, j->nsteps - j->enqueued);
    if (k <= 0) continue;
    const icm_status st = icm_step(j->sim, k);
    if (st != ICM_OK) return st;
    j->enqueued += k;
    if (j->enqueued == j->nsteps) ICM_CK(cudaEventRecord(j->done, j->sim->stream));
  }
  if (n_active) *n_active = (int32_t)sv->active.size();
  if (n_waiting) *n_waiting = (int32_t)sv->waiting.size();
  if (n_finished) *n_finished = finished;
  return ICM_OK;
}

icm_status icm_server_result(icm_server* sv, int64_t job_id, int32_t* state, double* pos, double* vel,
                             double momentum[3], double* latency_s) {
  if (!sv) return fail(ICM_EINVAL, "NULL server");
  auto it = sv->jobs.find(job_id);
  if (it == sv->jobs.end()) return fail(ICM_EINVAL, "unknown job id %lld", (long long)job_id);
  icm_server::Job* j = it->second;
  if (state) *state = j->state;
  if (j->state >= 2) {
    const size_t n = j->out_pos.size();
    if (pos && n) memcpy(pos, j->out_pos.data(), sizeof(double) * n);
    if (vel && n) memcpy(vel, j->out_vel.data(), sizeof(double) * n);
    if (momentum) memcpy(momentum, j->out_mom, sizeof(j->out_mom));
    if (latency_s) latency_s[0] = std::chrono::duration<double>(j->t_done - j->t_submit).count();
  }
  return ICM_OK;
}

icm_status icm_server_cancel(icm_server* sv, int64_t job_id) {
  if (!sv) return fail(ICM_EINVAL, "NULL server");
  auto it = sv->jobs.find(job_id);
  if (it == sv->jobs.end()) return fail(ICM_EINVAL, "unknown job id %lld", (long long)job_id);
  icm_server::Job* j = it->second;
  if (j->state == 0) {
    for (auto w = sv->waiting.begin(); w != sv->waiting.end(); ++w)
      if (*w == j) {
        sv->waiting.erase(w);
        break;
      }
  } else if (j->state == 1) {
    // the steps already enqueued for this job (one pump's worth at most) run out on its
    // own stream before its memory goes back to the budget; other jobs are not waited for
    const cudaError_t e = cudaStreamSynchronize(j->sim->stream);
    for (auto a = sv->active.begin(); a != sv->active.end(); ++a)
      if (*a == j) {
        sv->active.erase(a);
        break;
      }
    sv->used -= j->bytes;
    if (j->done) cudaEventDestroy(j->done);
    j->done = nullptr;
    icm_destroy(j->sim);
    j->sim = nullptr;
    if (e != cudaSuccess) {
      j->state = 3;
      j->t_done = std::chrono::steady_clock::now();
      return fail(ICM_ECUDA, "%s", cudaGetErrorString(e));
    }
  } else {
    return ICM_OK;   // already done, failed or cancelled
  }
  j->state = 4;
  j->t_done = std::chrono::steady_clock::now();
  return ICM_OK;
}

int64_t icm_server_bytes_in_use(const icm_server* sv) { return sv ? sv->used : -1; }

void icm_server_destroy(icm_server* sv) {
  if (!sv) return;
  for (auto& kv : sv->jobs) {
    if (kv.second->sim) icm_destroy(kv.second->sim);
    if (kv.second->done) cudaEventDestroy(kv.second->done);
    delete kv.second;
  }
  delete sv;
}

}  // extern "C"
