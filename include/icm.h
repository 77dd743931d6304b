/*
 * icm.h -- C ABI of the GB300 (sm_103a) library for one time step of the
 * incompressible Inertial Coupling Method (ICM):
 *
 *   F. Balboa Usabiaga, R. Delgado-Buscalioni, B. E. Griffith, A. Donev,
 *   "Inertial coupling method for particles in an incompressible fluctuating
 *   fluid", arXiv:1212.6427.
 *
 * Blob particles (positions q, velocities u, excess masses m_e, external forces F)
 * are coupled by a no-slip constraint to a periodic, incompressible, thermally
 * fluctuating fluid discretised on a staggered (MAC) grid.  One call of
 * icm_step advances the nine-step scheme of Sec. III.C ("Summary of Algorithm")
 * once per step entirely on the GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: Nx x Ny x Nz cells of side h, periodic in every direction.  Cell
 *    (i,j,k) is centred at ((i+1/2)h, (j+1/2)h, (k+1/2)h).  Component v_x of a
 *    face field sits at (ih, (j+1/2)h, (k+1/2)h), v_y and v_z likewise.
 *  - A "face field" on the host is a double array of 3*Nx*Ny*Nz values, the three
 *    components one after the other, each with flat index i + Nx*(j + Ny*k).
 *  - Blob arrays on the host are double, row-major: pos[n][3], vel[n][3],
 *    force[n][3], excess_mass[n].
 *  - All pointers named in a signature are HOST pointers unless the name ends
 *    in _dev.  The caller owns every host buffer; the library copies what it
 *    needs before returning and never keeps a host pointer.  The library owns all
 *    device memory of a simulation (allocated through the allocator set with
 *    icm_set_default_allocator, else cudaMalloc) and frees it in icm_destroy.
 *  - Every call is issued on the simulation's CUDA stream.  Calls that return
 *    host data synchronise that stream; icm_step only enqueues work.
 *  - Every function returns an icm_status; on failure icm_last_error() gives a
 *    one-line reason.  A failed call leaves the simulation as it was, except
 *    ICM_ECUDA, after which the simulation should be destroyed.
 *  - Not thread safe per simulation: one host thread at a time per icm_sim.
 */
#ifndef ICM_H_
#define ICM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct icm_sim icm_sim;   /* opaque */

typedef enum {
  ICM_OK = 0,
  ICM_EINVAL = -1,       /* invalid argument (value, size, NULL where required)      */
  ICM_ENOMEM = -2,       /* device allocation failed or over the memory budget       */
  ICM_ECUDA = -3,        /* a CUDA call failed (message in icm_last_error)            */
  ICM_ECFL = -4,         /* a blob moved more than one cell in a step: |u| dt / h > 1  */
  ICM_ENONFINITE = -5,   /* a NaN or Inf appeared in the blob state                   */
  ICM_ETIMEOUT = -6,     /* a bounded device-side wait gave up                        */
  ICM_EBUSY = -7,        /* the request cannot be taken now (e.g. batch slots full)   */
  ICM_EINDEX = -8        /* a device-side index check failed (the checked build only,
                            libicm_checked.so, compiled with -DICM_INDEX_CHECKS=1)     */
} icm_status;

/* Flags of icm_create. */
#define ICM_FLAG_NO_ADVECTION 0x1   /* drop the advective flux (Sec. II.B: no measurable effect) */
#define ICM_FLAG_SLIP_VISC    0x0   /* slip correction Eq. delta_u_nph_visc (paper's default)   */
#define ICM_FLAG_SLIP_ZERO    0x2   /* delta u = 0: first-order variant (Sec. III.C)            */
#define ICM_FLAG_SLIP_FULL    0x4   /* Eq. delta_u_nph: viscous + centring correction           */
#define ICM_FLAG_THERMAL_DRIFT 0x8  /* add the thermal drift kT m~_f/m~ d(delta_a)/dq at q^{n+1/2}
                                       to the first solve (Appendix B.2, Eq. thermal_drift,
                                       kernel-derivative form); no effect at kT = 0       */

/* Allocator used for the device memory of simulations created afterwards.
 * alloc(ctx, bytes, stream) returns a device pointer aligned to >= 256 bytes or
 * NULL; free(ctx, ptr, stream) releases it.  Passing NULL for both restores
 * cudaMalloc/cudaFree.  Process-wide; not thread safe against icm_create. */
typedef void* (*icm_alloc_fn)(void* ctx, size_t bytes, void* cuda_stream);
typedef void (*icm_free_fn)(void* ctx, void* ptr, void* cuda_stream);
icm_status icm_set_default_allocator(icm_alloc_fn alloc, icm_free_fn release, void* ctx);

/* Create a simulation (Sec. III: MAC grid, Peskin kernel, parameters of the
 * fluid equation Eq. LLNS_incomp_v).
 *   grid[3]   : Nx, Ny, Nz.  Each side 2^a 3^b, at least 2*kernel and at most 512.
 *   h         : grid spacing (> 0).        rho : fluid density (> 0).
 *   eta       : shear viscosity (> 0).     kT  : temperature (>= 0; 0 = deterministic).
 *   dt        : time step (> 0).
 *   kernel    : 3 or 4 (Peskin 3-point or 4-point function, Sec. III.A.1).
 *   seed      : key of the Philox4x32-10 stream of the stochastic stress.
 *   precision : 32 (FP32 fields, FP64 blob state and momentum bookkeeping) or 64.
 *   flags     : ICM_FLAG_* above.
 *   cuda_stream : cudaStream_t to work on, or NULL for a stream the library creates.
 *   out       : receives the handle.
 * Errors: ICM_EINVAL for any value outside the ranges above or a non-finite
 * value; ICM_ENOMEM if the device state cannot be allocated. */
icm_status icm_create(const int32_t grid[3], double h, double rho, double eta, double kT,
                      double dt, int32_t kernel, uint64_t seed, int32_t precision,
                      int32_t flags, void* cuda_stream, icm_sim** out);

/* Release all device memory of the simulation (synchronises its stream). */
void icm_destroy(icm_sim* sim);

/* One-line description of the last error of this thread (never NULL). */
const char* icm_last_error(void);

/* Append n blobs (Sec. II.A: position q, velocity u, excess mass m_e = m - rho dV).
 *   pos  : n*3 positions; wrapped into [0, N h) per axis.
 *   vel  : n*3 velocities, or NULL for zero.
 *   excess_mass : n values, each > -m~_f = -(3/2) rho dV with dV = h^3/(sum phi^2)^3
 *                 (8 h^3 for the 3-point kernel), so that m~ = m_e + m~_f > 0
 *                 (Appendix A, Eq. rho_eff_inv_incomp).
 * New blobs get F = 0 and a zero lagged slip term (q^{-1/2} = q^0).
 * Errors: ICM_EINVAL (n < 0, NULL pos, non-finite input, excess mass out of range),
 * ICM_EBUSY (queued reads pending: icm_read_finish them first). */
icm_status icm_add_blobs(icm_sim* sim, int64_t n, const double* pos, const double* vel,
                         const double* excess_mass);

/* Set the external force of every blob (Sec. III.C step 1: F^{n+1/2}), held until
 * the next call: force[n_total*3].  The values are copied before the call returns
 * (the caller may reuse the buffer at once); the upload runs on an upload stream of the
 * simulation beside the steps already queued, and the copy into place and the FP64 total
 * force are queued on the simulation's stream, ordered before the next step.
 * Errors: ICM_EINVAL (NULL, non-finite), ICM_ENOMEM (device landing buffer). */
icm_status icm_set_blob_forces(icm_sim* sim, const double* force);

/* Add to every blob the force of the harmonic potential V(r) = k r^2 / 2 about
 * center[3] (the temporal accuracy test of Sec. III.D, Eq. E_dt_definition),
 * evaluated each step at q^{n+1/2}: F_i^{n+1/2} = F_i - k d_i, d_i = q_i^{n+1/2} - center
 * taken to the nearest periodic image.  k = 0 removes the trap.  The total momentum
 * bookkeeping includes the trap's impulse.  Errors: ICM_EINVAL (NULL center,
 * non-finite values, k < 0). */
icm_status icm_set_blob_trap(icm_sim* sim, double k, const double center[3]);

/* Add the forces of the purely repulsive truncated Lennard-Jones (WCA) pair potential
 * V(r) = 4 eps ((sigma/r)^12 - (sigma/r)^6) + eps for r < 2^(1/6) sigma, 0 beyond
 * (Sec. IV.A, Eq. WCA), between every pair of blobs (nearest periodic image), evaluated
 * each step at q^{n+1/2} through a cell list.  epsilon = 0 removes them.  Errors:
 * ICM_EINVAL (non-finite, epsilon < 0, sigma <= 0, a box side shorter than twice the
 * cut-off), ICM_ENOMEM. */
icm_status icm_set_blob_wca(icm_sim* sim, double epsilon, double sigma);

/* Execution plan: implementation choices that change the speed of a step but not its
 * result beyond rounding (no counterpart in the paper).  Defaults: every choice on
 * except fused_xy, rhs_kz as below. */
typedef struct icm_plan {
  int32_t fused_blobs; /* 1: spreading and interpolation inside the x FFT passes through row-block
                          bins (sides 32, 48, 64, 96, 128, 192, 256, 384, 512); 0: separate kernels */
  int32_t tma_z;       /* 1: persistent z pass fed by TMA (z sides <= 256 with register kernels);
                          0: one block per z tile                                                  */
  int32_t rhs_kz;      /* right-hand-side kernel: 4..64 z planes marched by each block, or 0 for
                          persistent blocks (as many as the SMs hold) marching even shares of
                          all tile-planes (default 0 when each of two blocks per SM gets at least
                          8 tile-planes of 32 x 16 cells, else 8 for Nz <= 48 and 16 otherwise)    */
  int32_t fork;        /* 1: the blob-side prologue runs on a second stream beside the RHS          */
  int32_t fused_xy;    /* 1: forward x and y FFT passes fused on thread-block clusters (FP32,
                          Nx = Ny in 32, 64, 128, 256); 0 (default): two passes                    */
  int32_t z_split;     /* 1: the z transform with its other two-stage split (Nz = 32: 4 x 8, 48:
                          12 x 4, 64: 16 x 4, 96: 8 x 12, 128: 8 x 16, 192: 12 x 16, 256: 32 x 8);
                          0 (default): the axis split (8 x 4, 16 x 3, 8 x 8, 16 x 6, 16 x 8,
                          16 x 12, 16 x 16)                                                        */
} icm_plan;

/* The plan the next step will use.  Errors: ICM_EINVAL (NULL). */
icm_status icm_get_plan(const icm_sim* sim, icm_plan* out);

/* Fix the plan (choices the simulation cannot use fall back to the alternative).
 * Errors: ICM_EINVAL (NULL, rhs_kz neither 0 nor in 4..64). */
icm_status icm_set_plan(icm_sim* sim, const icm_plan* plan);

/* Autotuner: time the candidate plans over nsteps steps each (one choice at a time,
 * the others held at the best so far) on a copy of the current state, keep the
 * fastest, restore the state, and record the plan in a process-wide table keyed by
 * grid, precision, kernel, flags, blob count (power-of-two bucket) and whether blobs
 * have excess mass, which simulations without a fixed plan use when they capture their
 * step.  chosen and ms_per_step (the chosen plan's time) may be NULL.  Synchronises.
 * Errors: ICM_EINVAL (nsteps < 1), ICM_ENOMEM (no room for the state copy), device
 * errors of the trial steps (the state is restored first). */
icm_status icm_autotune(icm_sim* sim, int32_t nsteps, icm_plan* chosen, double* ms_per_step);

/* Enqueue nsteps ICM steps (Sec. III.C steps 1-9) on the simulation's stream.
 * Asynchronous: errors detected on the device (ICM_ECFL, ICM_ENONFINITE) are
 * reported by the next icm_sync / icm_read_state.  Errors: ICM_EINVAL (nsteps<0). */
icm_status icm_step(icm_sim* sim, int64_t nsteps);

/* Wait for the simulation's stream; report device-side errors raised since the
 * last report (ICM_ECFL: some blob had |u| dt/h > 1, Sec. III.D; ICM_ENONFINITE;
 * ICM_ETIMEOUT: a bounded device-side wait for a tensor-memory copy gave up, after
 * which the step's results are undefined and the simulation must be destroyed). */
icm_status icm_sync(icm_sim* sim);

/* Failure-path check, no counterpart in the paper: enqueue on the simulation's stream
 * a one-thread kernel that waits, with the same bounded mbarrier wait the TMA z pass
 * uses, for a transaction that is never issued.  After limit_ns nanoseconds
 * (1 <= limit_ns <= 2e9) it raises the simulation's timeout bit, so the next icm_sync
 * returns ICM_ETIMEOUT, as a copy that never lands would.  Nothing faults, nothing
 * stays in flight and the context stays usable.  Errors: ICM_EINVAL, ICM_ECUDA. */
icm_status icm_debug_wait_timeout(icm_sim* sim, int64_t limit_ns);

/* Read the state at the current time level (synchronises).  Any pointer may be
 * NULL to skip that output.
 *   pos[n*3], vel[n*3] : blob positions (in [0, N h)) and velocities.
 *   fluid_v[3*N]       : face velocities, layout as in the header comment.
 *   momentum[3]        : total momentum P = rho dV_f sum_k v_k + sum_i m_e,i u_i
 *                        (Sec. II, after Eq. no_slip), from the FP64 bookkeeping; the
 *                        blob sum is an FP64 compensated sum on the device.
 *   step               : number of steps taken (time level n).
 * Everything is read into a page-locked staging buffer of the simulation with one
 * wait.  Device errors of earlier steps are returned after the outputs are filled. */
icm_status icm_read_state(icm_sim* sim, double* pos, double* vel, double* fluid_v,
                          double momentum[3], int64_t* step);

/* Queued reads, for loops that read every step: icm_read_begin gathers icm_read_state's
 * blob outputs (positions, velocities, total momentum, step; no fluid) into a device
 * slot behind the work queued so far, copies that slot down to one of two page-locked
 * staging slots on a download stream of the simulation, and returns at once; the caller
 * may queue more steps (and forces) while the copy is in flight.  icm_read_finish waits for the oldest queued read and copies it
 * out (any pointer may be NULL); it returns the device errors raised before that read,
 * as icm_read_state would have (reporting one clears the device's error bits, including
 * bits of steps queued after the read).  Blobs cannot be added while reads are pending.
 * Errors: icm_read_begin ICM_EBUSY when two reads are pending, ICM_ENOMEM (staging
 * buffers); icm_read_finish ICM_EINVAL when none is pending. */
icm_status icm_read_begin(icm_sim* sim);
icm_status icm_read_finish(icm_sim* sim, double* pos, double* vel, double momentum[3], int64_t* step);

/* Overwrite the full state (checkpoint restore).  pos, vel: n_total*3 (required);
 * fluid_v: 3*N (required); adv_prev: 3*N advective flux div(rho v v^T)^{n-1} of the
 * previous step (Eq. Adams_Bashforth), or NULL for "no history" (A^{n-1} := A^n);
 * slip_g: n_total*3 lagged term J^{n-1/2} L dv^{n-1/2} (Eq. delta_u_nph_visc), or
 * NULL for zero; step: time level n (the Philox counter).  The total fluid
 * momentum bookkeeping is recomputed from fluid_v in FP64. */
icm_status icm_write_state(icm_sim* sim, const double* pos, const double* vel,
                           const double* fluid_v, const double* adv_prev,
                           const double* slip_g, int64_t step);

/* Read the rest of the state needed to resume bit-for-bit: adv_prev (3*N, or NULL),
 * slip_g (n_total*3, or NULL), has_history (0 if no step was taken since the last
 * icm_write_state with adv_prev = NULL). */
icm_status icm_read_aux(icm_sim* sim, double* adv_prev, double* slip_g, int32_t* has_history);

/* Advance nsteps steps like icm_step, but with every kernel launched eagerly and
 * bracketed by CUDA events on the simulation's stream (for measurement; slower
 * than the graph).  For each launch of one step, in order (at most max_stages):
 * names[i*32 .. i*32+31] a NUL-terminated stage name ("rhs", "rt1.z_sym", ...),
 * ms[i] the milliseconds summed over the nsteps steps, bytes[i] the algorithmic
 * bytes one launch must move (reads + writes of its operands, no re-reads).
 * Synchronises.  Errors: ICM_EINVAL (NULL, nsteps < 1), device errors as icm_sync. */
icm_status icm_profile_steps(icm_sim* sim, int64_t nsteps, int32_t max_stages, int32_t* nstages, char* names,
                             double* ms, double* bytes);

/* Total momentum P = rho h^3 sum_k v_k of a face field that is already on the device,
 * for callers that must not allocate device memory.  The paper has no counterpart:
 * this is a service of the library.  It uses the compensated FP64 scheme of the fluid
 * part of icm_read_state's momentum with a different block partition (fixed chunks of
 * 8192 cells per block), so the two agree to FP64 rounding, not bit for bit (tested
 * to 1e-12 relative).  Callers that cannot allocate include
 * code running while a stream capture is open (cudaMalloc is refused there),
 * processes whose device memory is already reserved by a framework's pool, and
 * loops that must not take the device-wide synchronisation of cudaMalloc/cudaFree.
 *   fluid_v_dev : device pointer to 3*ncell values (float if precision == 32,
 *                 double if 64), the face-field layout of the header comment;
 *                 read only, owned by the caller.
 *   ncell       : Nx*Ny*Nz, 1 <= ncell <= 134217728 (512^3); larger is ICM_EINVAL.
 *   rho, h      : density and grid spacing (the factor rho h^3).
 *   cuda_stream : stream to run on (NULL = legacy default stream); synchronised.
 *                 It must not be capturing (ICM_EINVAL).  While any capture is open,
 *                 pass a non-blocking stream of your own, not NULL: the legacy
 *                 stream is refused (ICM_EINVAL) while a blocking stream captures.
 *                 The call ends with a copy to the host and a wait on this stream;
 *                 open other threads' captures in relaxed mode, since global-mode
 *                 captures may forbid that wait.
 *   momentum[3] : host output.
 * Allocates nothing: its scratch is a fixed array of 3*16384+8 doubles (~384 KB)
 * that the library declares in device memory, held by every GPU that loads the
 * library until the process exits.  The first call on each device looks up that
 * array's device address (once, with that device current); make that first call
 * before any stream capture.  That address is cached per device for the life of the
 * process: do not use the library across a cudaDeviceReset (or a reset of the primary
 * context), which would leave the cached address stale.  All calls share the array and each overwrites what
 * the previous one left there, so calls that overlap on the GPU (other streams or
 * threads at the same time) race and must be serialised by the caller.
 * Errors: ICM_EINVAL (NULL pointer, bad precision, ncell out of range), ICM_ECUDA. */
icm_status icm_fluid_momentum_static(const void* fluid_v_dev, int32_t precision, int64_t ncell, double rho,
                                     double h, void* cuda_stream, double momentum[3]);

/* The blob volume dV = (J S 1)^-1 = h^3 / (sum_k phi(k)^2)^3 of a Peskin kernel (Sec.
 * III.A.1, after Eq. JS_invariance): 8 h^3 for the 3-point kernel (as the paper states)
 * and (8/3)^3 h^3 for the 4-point kernel.  The rest mass m_f = rho dV and the
 * incompressible dragged mass m~_f = 3 rho dV / 2 (Appendix A) follow from it.
 *   kernel : 3 or 4;  h : grid spacing > 0;  volume : host output.
 * Errors: ICM_EINVAL (bad kernel, h <= 0 or not finite, NULL volume). */
icm_status icm_kernel_volume(int32_t kernel, double h, double* volume);

/* Measured FMA throughput of the current device (flop/s, an FMA counts 2) in FP32
 * (precision 32) or FP64 (64): eight independent FMA chains per thread in eight
 * 256-thread blocks per SM, timed with CUDA events on cuda_stream (NULL = legacy
 * stream) over a second launch after a first one; synchronises.  The denominator of
 * the FP64 path's arithmetic roofline; no counterpart in the paper.
 * Errors: ICM_EINVAL (bad precision, NULL output), ICM_ECUDA. */
icm_status icm_peak_fma(int32_t precision, void* cuda_stream, double* flops_per_s);

/* Number of blobs and bytes of device memory the simulation holds. */
int64_t icm_num_blobs(const icm_sim* sim);
int64_t icm_device_bytes(const icm_sim* sim);

/* ------------------------------------------------------------------------
 * Operator-level entry points.  Each runs one operator of the step on the GPU
 * with the simulation's grid, kernel and parameters, using its scratch buffers
 * (the simulation's state is not touched), and synchronises.  Inputs and
 * outputs are host arrays in the layouts above.
 * ------------------------------------------------------------------------ */

/* J (Sec. III.A.1): out[nb*3] = sum_k phi(q_i - r_k) v_k per component. */
icm_status icm_op_interpolate(icm_sim* sim, int64_t nb, const double* pos,
                              const double* fluid_v, double* out);

/* J L (the lagged slip term of Eq. delta_u_nph_visc): out = J (L v), L the
 * 7-point Laplacian of each component, evaluated as one gather. */
icm_status icm_op_interpolate_laplacian(icm_sim* sim, int64_t nb, const double* pos,
                                        const double* fluid_v, double* out);

/* S (Sec. III.A.1): out[3*N] = sum_i dV_f^-1 phi(q_i - r_k) F_i. */
icm_status icm_op_spread(icm_sim* sim, int64_t nb, const double* pos, const double* force,
                         double* out);

/* Helmholtz solve + projection by 3D FFT (Sec. III.D): solves
 * (a I - b L) x + G pi = rhs, D x = 0, i.e. x^ = P^ rhs^ / (a + b |d|^2) with P = I on
 * the mean.  (a, b) = (rho/dt, eta/2) is Eq. provisional_step-1, (1, 0) the
 * projection of step 5, (rho, dt eta/2) Eq. dv_eq_modified-1.  a = 0, b = eta is
 * the steady Stokes solve of the mobility of Sec. III.A.2; there the mean mode has no
 * solution and is set to zero.  a >= 0, b >= 0, a + b > 0; Errors: ICM_EINVAL. */
icm_status icm_op_spectral_solve(icm_sim* sim, double a, double b, const double* rhs,
                                 double* out);

/* Blob-grid coupling matrices of Sec. III.A.2: for each pair p, the 3x3 matrix
 *   out[9p + 3r + c] = e_r . J(qi_p) (a I - b L)^-1 P S(qj_p) e_c
 * (spread of a unit force e_c at qj_p, solve as icm_op_spectral_solve, interpolation
 * at qi_p), row-major.  (a, b) = (1, 0) gives J_i P S_j (translational invariance,
 * Fig. JPS); (0, eta) the Stokes mobility -J_i (eta L)^-1 P S_j.  qi, qj: n x 3
 * positions (host).  Uses the simulation's grid, kernel and scratch; synchronises.
 * Errors: ICM_EINVAL (NULL, n < 0, non-finite positions, a, b as above), ICM_ENOMEM. */
icm_status icm_op_coupling(icm_sim* sim, int64_t n, const double* qi, const double* qj, double a, double b,
                           double* out);

/* Dense explicit right-hand side of Eq. provisional_step-1 at time level `step`:
 * r = (rho/dt) v + (eta/2) L v + div Sigma^n - (3/2 A^n - 1/2 A^{n-1}), and A^n.
 * adv_prev may be NULL (no history).  out_adv may be NULL. */
icm_status icm_op_explicit_rhs(icm_sim* sim, const double* fluid_v, const double* adv_prev,
                               int64_t step, double* out_rhs, double* out_adv);

/* The 6 unit normals per cell of step `step` (Sec. III.B.2: W^n), ordered
 * (xx, yy, zz, xy, xz, yz), out[6*N] (component-major, cell i + Nx (j + Ny k)).
 * Philox4x32-10, key = the seed's two 32-bit halves, counter (cell, step, call, 0):
 * call 0 of a cell gives xx, yy (words 0-1) and zz, xy (words 2-3); call 1 at the
 * cell of plane k = 2m gives its xz, yz (words 0-1) and those of the cell above it,
 * plane 2m + 1 (words 2-3); unit normals by Box-Muller from u = (word + 1/2) 2^-32. */
icm_status icm_op_stress_normals(icm_sim* sim, int64_t step, double* out);

/* Raw Philox4x32-10 words: for i < n, counter (ctr0 + i, ctr1, ctr2, ctr3) and
 * key (key0, key1); out[4*n].  No simulation needed. */
icm_status icm_op_philox(int64_t n, uint32_t ctr0, uint32_t ctr1, uint32_t ctr2,
                         uint32_t ctr3, uint32_t key0, uint32_t key1, uint32_t* out);

/* ------------------------------------------------------------------------
 * Batched replicas.  A batch advances several independent simulations with one
 * CUDA graph launch per step: the step of every member (Sec. III.C) is captured as
 * an independent branch, so the GPU runs the members' kernels side by side.  The
 * paper runs one simulation at a time; this layer has no counterpart there.
 * ------------------------------------------------------------------------ */
typedef struct icm_batch icm_batch;

/* Create an empty batch working on cuda_stream (NULL: a stream of its own). */
icm_status icm_batch_create(void* cuda_stream, icm_batch** out);

/* Set the members (n distinct simulations; the caller keeps ownership and must
 * not destroy a member while it belongs to a batch).  Synchronises the batch. */
icm_status icm_batch_set(icm_batch* batch, int32_t n, icm_sim* const* sims);

/* Advance every member nsteps steps (one graph launch per step; recaptured when
 * membership or a member's step sequence changed).  Asynchronous; later work on a
 * member's own stream is ordered after these steps. */
icm_status icm_batch_step(icm_batch* batch, int64_t nsteps);

/* Group solves (grouped = 1; default 0): members on the same grid (precision,
 * sides and cell width h) run each of the three fluid solves of a step (Sec. III.C,
 * steps 2, 5 and 6) as one set of FFT launches over all of them, between which each
 * member's own stencil and blob kernels run on its stream; members take the separate
 * (unfused) blob path and the plain z pass.  A grid whose sides lack register FFT
 * passes, or that only one member has, runs its step as usual.  Results agree with
 * ungrouped steps to rounding.
 * Batched stages (grouped = 2): the group solves as above, and every other stage of the
 * step (scalar bookkeeping, predictor, right-hand side, spreads, momentum change,
 * inertial update, finish) as one launch over all members, whatever their grids and
 * blob counts, through device tables of the members; about a dozen launches plus the
 * group solves per step.  Needs one precision for all members, register FFT passes
 * along every axis of every grid, and no WCA pair forces or thermal drift; otherwise
 * the batch runs as with grouped = 1.  Groups on z sides from 96 whose plan takes the
 * tensor-map z pass put their members' spectra in one buffer of the batch (the members'
 * own spectra stay unused meanwhile).  The batch's device tables and these buffers come
 * from cudaMalloc, not from the members' allocator, and are freed at the next capture
 * or by icm_batch_destroy.  Batched stages with the blob work in the group
 * x passes (grouped = 3): as 2, but where every member has blobs and a register x side
 * the spreads and interpolations run inside the x passes of the group solves, as in a
 * single simulation's fused step (row bins of all members in three launches; no
 * separate spread, zeroing or interpolation launch); otherwise as 2.  Synchronises when
 * the setting changes.  Errors: ICM_EINVAL for grouped other than 0 to 3. */
icm_status icm_batch_set_grouped(icm_batch* batch, int32_t grouped);
/* The current setting (0 to 3), -1 for a NULL batch. */
int32_t icm_batch_get_grouped(const icm_batch* batch);
/* Kernel launches in one batch step of the captured graph (the graph is captured by
 * the first icm_batch_step after a change); -1 before a capture or for NULL. */
int64_t icm_batch_kernels_per_step(const icm_batch* batch);

/* Autotune the batch as a whole: candidate plans (one choice at a time, as
 * icm_autotune) are applied to every member and timed over nsteps batch steps,
 * then group solves and batched stages (icm_batch_set_grouped 1, 2, 3) with that plan;
 * every member's state is
 * restored after each trial and the fastest choice is fixed on the batch and all
 * members.  Synchronises.  Errors: as icm_autotune. */
icm_status icm_batch_autotune(icm_batch* batch, int32_t nsteps);

/* Wait for the batch; returns the first device-side error of any member. */
icm_status icm_batch_sync(icm_batch* batch);
void icm_batch_destroy(icm_batch* batch);

/* Device bytes a simulation of this grid, precision and blob count will hold
 * (-1 for invalid arguments); what the server admits jobs by. */
int64_t icm_estimate_device_bytes(const int32_t grid[3], int32_t precision, int64_t nblobs);

/* ------------------------------------------------------------------------
 * Serving.  Jobs (one simulation each, advanced a given number of steps) queue on
 * the host and are admitted first come first served while their device footprint
 * fits the HBM budget and an active slot is free.  Every active job replays its own
 * step graph on its own stream, so the jobs' kernels overlap on the GPU; a job
 * leaves with its final blob state once its last step has completed, freeing its
 * memory for the next.  No counterpart in the paper.
 * ------------------------------------------------------------------------ */
typedef struct icm_server icm_server;
typedef struct {
  int32_t grid[3];
  double h, rho, eta, kT, dt;
  int32_t kernel;
  uint64_t seed;
  int32_t precision, flags;
  int64_t nblobs;
  const double* pos;          /* nblobs*3 (copied at submit) */
  const double* vel;          /* nblobs*3 or NULL */
  const double* excess_mass;  /* nblobs */
  const double* force;        /* nblobs*3 or NULL (constant external force) */
  int64_t nsteps;             /* >= 1 */
} icm_job_desc;

icm_status icm_server_create(int64_t hbm_budget_bytes, int32_t max_active, icm_server** out);
/* Queue a job; its arrays are copied.  ICM_ENOMEM if it can never fit the budget. */
icm_status icm_server_submit(icm_server* server, const icm_job_desc* job, int64_t* job_id);
/* Retire jobs whose last step has completed, admit waiting jobs that fit, and
 * enqueue up to steps_per_pump more steps of every active job.  Does not wait for
 * the GPU (reading a finished job's results is the only synchronisation).  Any
 * output pointer may be NULL; n_finished counts jobs retired by this call. */
icm_status icm_server_pump(icm_server* server, int32_t steps_per_pump, int32_t* n_active, int32_t* n_waiting,
                           int32_t* n_finished);
/* state: 0 waiting, 1 active, 2 done, 3 failed, 4 cancelled.  When done: pos, vel
 * (nblobs*3), momentum[3] and latency_s (submit to completion, seconds), each may be
 * NULL.  A job the device has no memory for at admission (ICM_ENOMEM from the
 * allocator) stays first in line and is retried at the next pump. */
icm_status icm_server_result(icm_server* server, int64_t job_id, int32_t* state, double* pos, double* vel,
                             double momentum[3], double* latency_s);
/* Withdraw a job between pumps.  A waiting job leaves the queue; an active job's
 * already enqueued steps (at most one pump's worth) are waited for on its own stream,
 * then its simulation is destroyed and its bytes return to the budget.  Other jobs
 * are neither waited for nor changed.  Its state becomes 4 (cancelled); a job that
 * has already finished is left as it is.  Errors: ICM_EINVAL (unknown id), ICM_ECUDA. */
icm_status icm_server_cancel(icm_server* server, int64_t job_id);
int64_t icm_server_bytes_in_use(const icm_server* server);
void icm_server_destroy(icm_server* server);

#ifdef __cplusplus
}
#endif
#endif /* ICM_H_ */
