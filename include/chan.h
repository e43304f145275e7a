/*
 * chan.h — C ABI of a single-GPU (sm_103a) library that advances the
 * velocity–vorticity (v–omega_2) formulation of incompressible turbulent
 * channel flow by semi-implicit low-storage RK3 substeps, and writes the
 * filtered velocities and filtered stresses of the second-order-consistent
 * database of Vela-Martin et al., arXiv:1808.06461.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: channel half-height h = 1 (walls at y = -1 and y = +1), friction
 *   velocity u_tau = 1, so nu = 1 / Re_tau (Sec. 2.1).
 * Grid: Nx, Nz are the collocation points of the periodic directions
 *   (Sec. 2.1: N_1/2, N_3/2 Fourier modes, 3/2-rule dealiasing); Ny is the
 *   number of wall-normal points (odd, >= 9).  Nx, Nz must be even and of
 *   the form 2^a 3^b with 3Nx/2, 3Nz/2 in [6, 4608].
 * Fourier field layout ("spectral layout"): interleaved complex double
 *   (re, im), C order [Ny][Nz][Nx/2], i.e. element (j, jz, kx) at
 *   2 * ((j * Nz + jz) * (Nx/2) + kx).  kx = 0 .. Nx/2-1 (k_1 = 2 pi kx / Lx);
 *   jz in FFT order (k_3 = 2 pi kz / Lz, kz = jz for jz < Nz/2, jz - Nz
 *   otherwise).  The kz Nyquist row jz = Nz/2 is held at zero.  A kx > 0
 *   coefficient stands for itself and its complex conjugate at -kx; the
 *   kx = 0 column must be Hermitian in kz.  Physical fields are
 *   u(x, z) = sum u_k exp(+i (k_1 x + k_3 z)).
 * Profiles (U1, U3, statistics): double[Ny], index j of the mesh returned by
 *   chan_get_grid.
 * Ownership: a chan_t owns all the device memory it allocates; every
 *   pointer argument is caller-owned and only read or written during the
 *   call.  Host pointers may be pageable or pinned.
 * Streams: all device work of a handle runs in order on one CUDA stream
 *   (the library's own, or the caller's via chan_opts.stream).  Entry points
 *   that return host data synchronise that stream before returning;
 *   chan_step is asynchronous.
 * Errors: every int-returning call returns CHAN_OK (0) or a negative
 *   CHAN_E* code and records a message readable with chan_last_error.  No
 *   call aborts the process or traps the GPU.
 */
#ifndef CHAN_H
#define CHAN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHAN_OK        0
#define CHAN_EINVAL   -1   /* bad argument: sizes, dt <= 0, NULL handle, unknown kind   */
#define CHAN_ENOMEM   -2   /* device or host allocation failed                           */
#define CHAN_ECUDA    -3   /* a CUDA runtime call or kernel launch failed                */
#define CHAN_ENAN     -4   /* the state holds a non-finite value (checked on read-back)  */
#define CHAN_ESTATE   -5   /* call out of order (e.g. chan_step before chan_set_state)   */
#define CHAN_ETIMEOUT -6   /* a bounded device-side wait ran out (persistent batches)   */

#define CHAN_FILTER_SHARP 0   /* Eq. (fou_fil): G = 1 if |k1| < pi/l1c and |k3| < pi/l3c   */
#define CHAN_FILTER_BOX   1   /* top-hat of widths (D1, D3): G = sinc(k1 D1/2) sinc(k3 D3/2) */

#define CHAN_PREC_FP64  0     /* every step in FP64                                        */
#define CHAN_PREC_MIXED 1     /* FFTs and products in FP32; y-solves, mean flow, stats FP64 */
#define CHAN_PREC_F64X  2     /* FFTs, products and the substep's wall-normal sweeps in
                                 double-float (FP32 pairs, ~2^-47), Fourier fields stored
                                 as pairs; mean flow, stats FP64                           */
#define CHAN_PREC_MIXED_DF 3  /* FFTs and products in FP32; the substep's wall-normal
                                 sweeps in double-float with Fourier fields stored as
                                 pairs (as CHAN_PREC_F64X); mean flow, stats FP64           */

#define CHAN_NSTAT 20         /* rows of chan_stats' output, see chan_stats                */

typedef struct chan_s* chan_t;

typedef struct chan_opts {
  double re_tau;     /* friction Reynolds number; nu = 1/re_tau                      */
  double Lx, Lz;     /* periods of the box in x (streamwise) and z (spanwise)        */
  int Nx, Ny, Nz;    /* collocation points                                           */
  double dt;         /* time step of a full RK3 step (each substep uses dt)          */
  double eta_w;      /* wall Kolmogorov scale of the mesh (default 1.0)              */
  double grid_re;    /* Re_tau the mesh is clustered for (<= 0: re_tau)              */
  int precision;     /* CHAN_PREC_FP64, _MIXED, _F64X or _MIXED_DF                    */
  void* stream;      /* cudaStream_t to run on, or NULL for a library-owned stream   */
  const double* mesh;/* explicit wall-normal mesh double[Ny] (increasing from -1 to 1,
                        mirror symmetric), e.g. from chan_optimize_mesh; NULL: the
                        Kolmogorov-scaled formula                                      */
  int slab_planes;   /* planes per slab of the plane-local transform passes (0: all Ny
                        planes unless the twelve mixed-layout transform fields would
                        pass 8 GiB, then the fewest equal slabs below that).  Results
                        do not depend on it; only the transform buffers scale with it.
                        The filter pass runs in slabs of at most these planes whose six
                        products and nine outputs stay within 4 GiB                    */
  int lean_tables;   /* 1: keep the implicit-step LU factors and homogeneous solutions of
                        one RK3 substep only and recompute them at each substep (a third
                        of the table memory, more FP64 work); 2: as 1, and those tables
                        and the Poisson factors occupy no memory of their own: each
                        substep computes them into work fields that are dead from the
                        non-linear terms to the Poisson step (the filtered pressure then
                        allocates its own Poisson factors on its first call); in the
                        pair-stored precisions 2 acts as 1; -1: keep all three; 0: 1 when
                        the box would otherwise need more than 200 GB, and 2 when it would
                        still need more than 150 GB.  Results do not depend on it        */
  int y_tables;      /* where the wall-normal sweeps read their mode-independent tables:
                        1 in place from global memory, 2 staged in shared memory, 0 staged
                        unless that needs more than 16 KB per CTA (chan_autotune may
                        change it).  Results do not depend on it                        */
  int keep_rhs;      /* 1: keep the interior right-hand sides of the last Helmholtz solves
                        (two Fourier fields), from which the next substep's right-hand
                        side follows without the B product (Appendix A); -1: form B X
                        in every substep instead; 0: keep them unless the box would then
                        need more than 150 GB.  The two forms agree to rounding, not
                        bitwise                                                         */
} chan_opts;

/* Fill *o with defaults: eta_w = 1, grid_re = 0, FP64, library stream. */
void chan_opts_default(chan_opts* o);

/*
 * Create a channel on the current CUDA device (Sec. 2.1 / Appendix A set-up):
 * mesh, compact finite-difference operators (Appendix B), per-wavenumber
 * LU factors of the implicit RK3 Helmholtz and Poisson operators, their
 * homogeneous solutions and influence matrices.  No state yet: call
 * chan_set_state next.  *out receives the handle (NULL on failure).
 */
int chan_init(chan_t* out, double re_tau, double Lx, double Lz, int Nx, int Ny, int Nz, double dt);
int chan_init_ex(chan_t* out, const chan_opts* o);

/* Release everything the handle owns (a library interface; the paper has no
 * counterpart).  NULL is a no-op. */
void chan_free(chan_t h);

/* Message of the last error on this handle (or of the last failed init when h is NULL). */
const char* chan_last_error(chan_t h);

/* Number of complex coefficients of one Fourier field: Ny * Nz * (Nx/2). */
size_t chan_fourier_count(chan_t h);

/* Bytes of device memory the handle holds. */
size_t chan_device_bytes(chan_t h);

/*
 * Device bytes chan_init_ex requests for a box of this size and precision
 * (including the filter's transfer function); 0 for invalid sizes.  No GPU
 * needed.  For admission by HBM footprint; the allocator may round up.
 */
size_t chan_footprint_bytes(int Nx, int Ny, int Nz, int precision);

/*
 * Near-wall mesh optimisation of Appendix B.  Starting from the
 * mesh chan_init_ex would build for *o, moves the first 20 interior points at
 * each wall (mirrored), every moved cell kept within a factor of two of its
 * starting size, by steepest descent on
 *   L = |g - g_ana| + C |mu - mu_ref|,
 * g the discrete solution of (B - k* A) g = 0 with g(-1) = 1, g(+1) = 0 at the
 * box's most critical modified wavenumber k* = k1max^2 + k3max^2 + 6/(nu dt),
 * g_ana its sinh solution, mu the moved points and mu_ref their start (the
 * paper uses C ~ 1e-3).  Writes the mesh (double[Ny]) to y and |g - g_ana|
 * before and after.  Host only, no GPU.  Pass the mesh back in opts.mesh.
 */
int chan_optimize_mesh(const chan_opts* o, int iters, double C, double* y, double* err_before, double* err_after);

/*
 * Autotuner (no paper counterpart): times the z-pass with 1, 2, 4, 8 and 16
 * columns per CTA, the x-pass with 96, 128, 160, 192, 256, 288, 384 and 512 threads per CTA, and the
 * wall-normal sweeps with their mode-independent tables staged in shared
 * memory or read in place from global memory, on the current state; keeps
 * the fastest and caches the choice for every later handle of the same
 * (Nx, Ny, Nz, precision) in the process.  The choices only regroup or
 * relocate identical arithmetic, so results are bitwise unchanged.  Needs a
 * state; overwrites only scratch; synchronises.  chan_tuned_shape reports
 * the shapes in use (ytab_global: 1 when the sweeps read their tables in
 * place; by default they do when staging would need more than 16 KB per CTA).
 */
int chan_autotune(chan_t h);
int chan_tuned_shape(chan_t h, int* kb_z, int* xthreads, int* ytab_global);

/*
 * Replay whole RK3 steps (three substeps) from a CUDA graph captured on the
 * first use (enable = 1) instead of launching each kernel; chan_step falls
 * back to single launches at a step's ragged ends and while tracing is on.
 * Results are identical either way.  Off by default.
 */
int chan_set_graph(chan_t h, int enable);

/* Wall-normal mesh, double[Ny] (Sec. 2.1: spacing ~ local Kolmogorov scale). */
int chan_get_grid(chan_t h, double* y);

/*
 * Set the state from host arrays: the variables Appendix A advances, v = u_2
 * and omega_2 in spectral layout, and the mean profiles U1, U3 of Sec. 2.1
 * (zero at the walls).  Derives chi = Lap v (Appendix A, Eq. (chi2)) and
 * dv/dy on the device, clears the previous-substep non-linear terms, sets
 * the target mass flux to the flux of U1 and the RK3 substep counter to 0.
 * The (0,0) Fourier coefficients of v and omega_2 are ignored (held at 0).
 */
int chan_set_state(chan_t h, const double* v, const double* omega2, const double* U1, const double* U3);
/* Same with device pointers (same layouts). */
int chan_set_state_device(chan_t h, const void* v, const void* omega2, const void* U1, const void* U3);

/* Copy the current state (v, omega_2, U1, U3 of Appendix A and Sec. 2.1) out
 * (host; synchronises).  In the pair-stored modes the pairs are merged to FP64. */
int chan_get_state(chan_t h, double* v, double* omega2, double* U1, double* U3);
/* Device-to-device copy of the state into caller buffers (asynchronous). */
int chan_get_state_device(chan_t h, void* v, void* omega2, void* U1, void* U3);

/*
 * Checkpoint and restart (no paper counterpart; the paper restarts its runs from
 * stored full fields, Sec. 3).  A checkpoint holds everything the next substep
 * reads: v, omega_2, chi, dv/dy, the previous non-linear terms and implicit
 * right-hand sides, U_1, U_3 and their previous <H>, the flux target, the RK3
 * phase and time, in the handle's storage format, so a run restarted from it
 * continues bitwise as the original would (a state upload re-derives chi and
 * starts a fresh RK3 step instead).  chan_checkpoint_bytes gives the size;
 * _save copies it into the caller's host buffer (synchronises); _load checks that
 * the buffer was written by a handle of the same box, grid, time step and
 * precision (CHAN_EINVAL otherwise) and installs it.
 */
size_t chan_checkpoint_bytes(chan_t h);
int chan_checkpoint_save(chan_t h, void* buf);
int chan_checkpoint_load(chan_t h, const void* buf);

/*
 * Advance nsub RK3 substeps (Appendix A, Eqs. (chi1), (chi2), (psi); order of
 * operations of Appendix C): u_1, u_3 and their y-derivatives from
 * (v, omega_2); vorticity; dealiased H = u x omega; N_chi and N_omega2
 * (Eq. (hghv)); implicit Helmholtz steps for omega_2 and chi; Poisson for
 * v with the influence-matrix wall correction; mean profiles with the
 * constant-flux pressure gradient.  Asynchronous on the handle's stream.
 */
int chan_step(chan_t h, int nsub);

/*
 * Filtered velocities ubar_i = G u_i and stresses
 * tau_ij = G P(u_i u_j) - P(ubar_i ubar_j) of the current state (Sec. 3.1),
 * P the dealiased projection on the stored modes.  kind is CHAN_FILTER_*;
 * (p1, p3) are l_1c^+, l_3c^+ for SHARP (the paper uses 120, 60) or the
 * box widths Delta_x^+, Delta_z^+ for BOX.  ubar receives 3 fields and tau
 * 6 fields (order 11, 22, 33, 12, 13, 23), spectral layout, field-major;
 * either may be NULL (the result is still kept for chan_stats).  Does not
 * advance time.  Synchronises when a host pointer is given.
 */
int chan_filter_stresses(chan_t h, int kind, double p1, double p3, double* ubar, double* tau);

/*
 * Filtered enstrophy filt(omega_i omega_i) = G P(omega_i omega_i) of the
 * current state, the tenth variable of the paper's database (Sec. 3.1);
 * kind and (p1, p3) as for chan_filter_stresses.  ens receives one field,
 * spectral layout, host.  Does not advance time; synchronises.
 */
int chan_filtered_enstrophy(chan_t h, int kind, double p1, double p3, double* ens);

/*
 * The low-storage database record of the current state (Sec. 3.1, Table 2):
 * with the sharp cut-off filter (l_1c^+ = p1, l_3c^+ = p3) the ten stored
 * variables ubar_1..3, filt(u_i u_j) (11, 22, 33, 12, 13, 23) and
 * filt(omega_i omega_i), on the retained modes only: kx = 0..M1-1 and
 * kz = 0..K3 followed by -K3..-1 (M3 = 2 K3 + 1).  rec receives
 * [10][Ny][M3][M1] interleaved complex doubles (host); *m1, *m3 receive M1,
 * M3.  Call with rec = NULL to query the sizes only.  The device keeps a
 * buffer of that size after the first call.  Does not advance time.
 */
int chan_database_record(chan_t h, double p1, double p3, double* rec, int* m1, int* m3);

/*
 * Filtered pressure of the current state from the filtered stresses,
 * Sec. 3.1 Eq. (2): d_kk pbar = -d_ij filt(u_i u_j) per Fourier mode, with
 * the wall condition d pbar/dy = nu chibar (the filtered wall-normal momentum
 * balance at a wall) and the mean mode P = -filt(u_2 u_2).  kind, (p1, p3) as
 * for chan_filter_stresses.  p receives one field, spectral layout, host.
 * The first call builds per-wavenumber tables (2 Ny doubles per class) kept
 * on the device.  Does not advance time; synchronises.
 */
int chan_filtered_pressure(chan_t h, int kind, double p1, double p3, double* p);

/*
 * Two-dimensional energy spectra of the current state (Sec. 3.3):
 * E_i(k1, y, k3) = w |u_i(k1, y, k3)|^2 with w = 2 for kx > 0 (the
 * conjugate mode) and 1 for kx = 0; the mean (0,0) mode is excluded, so the
 * sum over modes at a height is the variance of u_i'.  E receives
 * [3][Ny][Nz][Nx/2] doubles (host).  Synchronises.
 */
int chan_spectra(chan_t h, double* E);

/*
 * Plane statistics of the current state (Sec. 3.3), double[CHAN_NSTAT][Ny]:
 * rows 0-1 U1, U3; rows 2-7 <u_i u_j> (11,22,33,12,13,23, Parseval over
 * all stored modes, means included); rows 8-13 <ubar_i ubar_j> and rows
 * 14-19 <tau_ij> of the last chan_filter_stresses (zero if none).  utau =
 * sqrt(nu |dU1/dy|) averaged over both walls, ubulk = flux/2, f = mean
 * pressure gradient of the last substep.  Any output pointer may be NULL.
 * Synchronises.
 */
int chan_stats(chan_t h, double* out, double* utau, double* ubulk, double* f);

/*
 * Dealiased Fourier coefficients of H = u x omega of the current state
 * (3 fields, spectral layout, field-major, host), without advancing time.
 * A diagnostic of the non-linear pass (Appendix A, Eq. (hghv) input).
 */
int chan_nonlinear(chan_t h, double* H);

/*
 * Per-kernel timing (tracing; the paper has no counterpart).  enable = 1
 * resets the counters and brackets every subsequent kernel launch of the
 * handle with CUDA events on its stream; enable = 0 stops recording.
 * chan_profile_read synchronises and writes, for each kernel id
 * k < CHAN_NKERNELS, the summed device time in ms and the launch count
 * since the last reset (launches are counted even when timing is off).
 * chan_kernel_name(k) names kernel k (NULL when out of range).
 */
#define CHAN_NKERNELS 18
int chan_profile(chan_t h, int enable);
int chan_profile_read(chan_t h, double* ms, long long* launches);
const char* chan_kernel_name(int k);

/*
 * Non-linear terms of the v and omega_2 equations of the current state,
 * Appendix A Eq. (hghv): N_chi = -d/dy(i k1 H1 + i k3 H3) - k^2 H2 and
 * N_omega2 = i k3 H1 - i k1 H3 (the D1 derivative is the compact scheme).
 * N receives 2 fields (N_chi, N_omega2), spectral layout, host.  Does not
 * advance time; synchronises.
 */
int chan_rhs_terms(chan_t h, double* N);

/*
 * chan_rhs_terms_noalloc — the same N_chi, N_omega2 as chan_rhs_terms, but
 * from caller device buffers and without allocating any device memory
 * (the paper has no counterpart; this is a library interface).  For callers
 * that cannot call cudaMalloc where they evaluate the terms: code running
 * inside a memory pool it does not own, a latency-bound loop that cannot
 * afford an allocation's implicit synchronisation, or a caller that has
 * reserved all device memory for its own arena.
 *   H: device, 3 fields (H1, H2, H3) in spectral layout, field-major.
 *   N: device, 2 fields (N_chi, N_omega2) written in the same layout.
 *   Both are plain FP64 complex (interleaved re, im doubles) in every
 *   precision mode, also for handles whose own fields are stored as FP32
 *   pairs (CHAN_PREC_F64X, CHAN_PREC_MIXED_DF); the arithmetic is FP64.
 * Runs asynchronously on the handle's stream (chan_sync to wait); the
 * current device must be the handle's.  Its only scratch is a fixed 32 MiB
 * device array inside the library (held on every GPU that loads it until
 * exit), so Ny * Nz * (Nx/2) must be <= 2097152, else CHAN_EINVAL.  The
 * first call on a device looks up that array's address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (the
 * kernel writes every value before reading it, so nothing needs clearing);
 * calls whose work overlaps on the GPU race on it.
 */
int chan_rhs_terms_noalloc(chan_t h, const void* H, void* N);

/*
 * Packed stepping of several independent channels (the serving mode; the
 * paper has no counterpart).  A batch holds n >= 1 handles of one precision
 * on one device, each with its state set; they may differ in every size and
 * be at different RK3 phases.  chan_batch_step advances every run by nsub
 * substeps with one launch per kernel covering all runs (at most 16 runs per
 * launch; more runs take more launches), on the batch's stream (the given
 * stream, or a stream of its own when NULL).  It first makes the batch stream
 * wait for each run's stream and afterwards makes each run's stream wait for
 * the batch, so per-run calls stay ordered.  Whole RK3 steps are replayed from
 * a CUDA graph captured on first use when all runs sit at a step boundary.
 * Each run's result is bitwise the one chan_step gives.  The handles must
 * outlive the batch and must not be stepped elsewhere while a batch step
 * is in flight.
 */
typedef struct chan_batch_s* chan_batch_t;
int chan_batch_create(chan_batch_t* out, chan_t* runs, int n, void* stream);
int chan_batch_step(chan_batch_t b, int nsub);
const char* chan_batch_last_error(chan_batch_t b);
void chan_batch_free(chan_batch_t b);

/*
 * A batch created with CHAN_BATCH_PERSISTENT (at most 16 runs; no paper
 * counterpart) steps with persistent launches instead of one launch per
 * kernel: one launch advances each run by up to 48 substeps.  A run's work is
 * its sequence of stages (substep, phase: pre, z inverse, x, z forward,
 * non-linear terms, Helmholtz, Poisson, mean flow), each stage the blocks of
 * that phase's kernel; the launch's CTAs take blocks of any run whose previous
 * stage is complete, so the phases of different runs run at once and every run
 * goes on to its next substep without waiting for the others.  A CTA that finds
 * no ready block polls again, a bounded number of times (chan_batch_set_wait);
 * when the polls run out the launch is void (its remaining blocks are skipped)
 * and chan_batch_status then returns CHAN_ETIMEOUT.  Each run's result is
 * bitwise the one chan_step gives.  The plan (stage table and an argument table
 * in device memory) is built at creation from the runs' current buffers and
 * launch shapes.  chan_batch_step(b, nsub) advances every run by nsub;
 * chan_batch_step_each(b, nsub) advances run r by nsub[r] >= 0 (runs may differ).
 */
#define CHAN_BATCH_PERSISTENT 1
int chan_batch_create_ex(chan_batch_t* out, chan_t* runs, int n, void* stream, int flags);
int chan_batch_step_each(chan_batch_t b, const int* nsub);
/* Wait for the batch stream; CHAN_ETIMEOUT if a persistent launch ran out of polls since
 * the last call (the runs' states are then void and must be set again), else CHAN_OK. */
int chan_batch_status(chan_batch_t b);
/* Persistent batches: empty polls (>= 1, about 0.13 us each) after which a CTA gives up
 * (default 2^23, about a second); hold_run, hold_stage >= 0 make that run's stage
 * (substep of the launch * 8 + phase, phases in the order above) need one completion more
 * than it can get, so that the polls run out (a test of the timeout path); -1, -1: none. */
int chan_batch_set_wait(chan_batch_t b, long long polls, int hold_run, int hold_stage);
/* CTAs of a persistent launch (resident CTAs per SM x SMs); 0 for other batches. */
int chan_batch_persistent_grid(chan_batch_t b);

/* Wait for the handle's stream (a library interface; the paper has no counterpart). */
int chan_sync(chan_t h);

/* Simulated time and substeps taken since chan_set_state. */
double chan_time(chan_t h);
long long chan_substeps(chan_t h);

#ifdef __cplusplus
}
#endif
#endif /* CHAN_H */
