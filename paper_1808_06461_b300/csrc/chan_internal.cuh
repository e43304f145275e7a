// Internal declarations of the channel library (device state, kernel
// launchers).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/chan.h"
#include "chan_host.h"
#include "df.cuh"

// Precision-mode properties (host side): transforms and products in FP32; Fourier
// fields stored as double-float pairs, with the substep's wall-normal sweeps in pairs.
inline bool prec_t32(int p) { return p == CHAN_PREC_MIXED || p == CHAN_PREC_MIXED_DF; }
inline bool prec_pairs(int p) { return p == CHAN_PREC_F64X || p == CHAN_PREC_MIXED_DF; }
// Where the wall-normal sweeps read their mode-independent tables (ytab as in chan_s): in
// place from global memory when asked, or by default when staging them (23 values per y
// point in the Poisson kernel) would pass 16 KB beside the sweeps' prefetch rings.
inline bool ytab_in_place(int ytab, int Ny) { return ytab > 0 || (ytab < 0 && 23 * (size_t)Ny * sizeof(double) > 16 * 1024); }

// Fourier fields: double2 arrays [Ny][M], M = Nz * (Nx/2), mode m = jz*nxh + kx.
// Mixed fields (physical z, Fourier kx): [Ny][L3][nxh] of float2 or double2.
// Wavenumber classes (shared LU factors): c = |kz| * nxh + kx, |kz| < Nz/2.

#define CHAN_MAXFIELDS 12
#define CHAN_MAXBATCH 16  // runs per packed launch (kernel parameters stay below 32 KB)

struct YTabs {            // mode-independent wall-normal tables (device)
  const double* A2;       // [Ny][7]
  const double* B2;
  const double* B1;
  const double* lu1;      // LU of A1
  const double* lu2f;     // LU of A2 (all rows)
  const double* d0;       // [Ny]
  const double* dN;
  const double* wq;
  // FP32-pair copies for the double-float sweeps (that mode only)
  const dfr *A2p, *B2p, *B1p, *lu1p, *d0p, *dNp;
};

struct Geo {
  int Nx, Ny, Nz, nxh, M, C, L1, L3;
  int pair;               // Fourier fields hold FP32 (hi, lo) pairs (double-float mode)
  int gtab;               // sweeps read the y tables from global memory (L1) instead of staging them
  double dt, nu;
  const double* k1;       // [nxh]
  const double* k3;       // [Nz]
};

struct FftPlan {
  int L, np;
  int radix[16];
  // ceil(2^32 / d) for the divisors of each stage (exact quotients via __umulhi for
  // operand n and divisor d with n d < 2^32; 0 stands for d = 1): L/R, and the span
  // Ls/R of the DIF and DIT stage
  unsigned mag_nbf[16], mag_mdif[16], mag_mdit[16];
  // inverse (natural in, digit-reversed out) Cooley-Tukey stages: twiddle exponent unit
  // K m of block b of stage s at revK[revoff[s] + b] (K the digit reversal of b over the
  // radices of stages 0 .. s-1, m = Ls/R); device table of at most L entries
  const int* revK;
  int revoff[16];
  // FP32 two-pass transforms (see fft_split): L = r1 r2, 0 when the stages above serve
  // this length; mag_r1 = ceil(2^32 / r1)
  int r1, r2;
  unsigned mag_r1;
  // their twiddles w_L^(-n2 k1) at [k1 (r2 + 1) + n2] (rows padded by one), staged into
  // shared memory by each CTA
  const float2* tw2p;
};

enum { KID_PRE = 0, KID_ZINV, KID_XPASS, KID_ZFWD, KID_NONLIN, KID_HELM, KID_POISSON, KID_MEAN,
       KID_FILTER_OUT, KID_STATS, KID_DERIVE, KID_APPLY_G, KID_GATHER, KID_SPECTRA, KID_PRESSURE, KID_TABLES,
       KID_SETUP_POIS, KID_COPY_MEAN, KID_COUNT };
static_assert(KID_COUNT == CHAN_NKERNELS, "every traced kernel id has a name in the ABI's count");

struct ProfRec {
  int k;
  cudaEvent_t a, b;
};

struct chan_s {
  // configuration
  double re, Lx, Lz, dt, nu, eta_w, grid_re;
  int Nx, Ny, Nz, nxh, M, C, L1, L3, prec;
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t side;       // the mean-flow solve of a substep, beside the wall-normal sweeps
  cudaEvent_t ev_fork, ev_join;
  int device;
  // host copies
  std::vector<double> y, wq;
  // state (device)
  double2 *v, *om, *chi, *dv, *Nchi_p, *Nom_p;
  double2 *Rom, *Rchi;     // interior right-hand sides of the last Helmholtz solves (valid when scal[2] != 0;
                           // NULL for a lean box, whose Helmholtz steps always form B X)
  double *U1, *U3, *H1m_p, *H3m_p;
  double* scal;            // [0] f of last substep, [1] Q0, [2] Rom / Rchi valid
  // tables (device)
  double *tab_A2, *tab_B2, *tab_B1, *tab_lu1, *tab_lu2f, *tab_d0, *tab_dN, *tab_wq;
  dfr* tab_pairs;          // double-float mode: A2, B2, B1, lu1 ([Ny][7] each), d0, dN as pairs
  double *k1, *k3;
  double* helm;            // [3][Ny][11][C], or [1][Ny][11][C] refilled per substep (lean)
  double* pois;            // [Ny][7][C]
  double* infl;            // [3][4][C] (lean: [1][4][C])
  int lean;                // 0: Helmholtz tables of all three substeps; 1: one slot, refilled each substep;
                           // 2: one slot and the Poisson factors, both in the work slots 2..6 (dead from the
                           // non-linear terms to the Poisson step) and both recomputed in every substep
  int lean_slot;           // the substep whose tables the slot holds
  double* mean_tab;        // lean 2: the (0,0) class of each substep's Helmholtz tables [3][Ny][11], read by
                           // the mean-flow solve, which runs beside the table set-up
  double2* h00;            // lean 2: the (0,0) modes of H_1, H_3 of the current substep [2][Ny]
  double* pois_prs;        // lean 2: Poisson factors of the filtered pressure (allocated on its first call)
  dfr *helm_df, *pois_df, *infl_df;   // pair copies for the double-float y-kernels (that mode only)
  double* meanh;           // [3][Ny+1]: U_h of each substep and its flux
  void *tw1, *tw3;         // twiddles of L1, L3 in the FFT precision
  // work (device)
  double2* wf;             // Fourier work fields [NWF][Ny][M]
  int nwf;
  void* mixed;             // mixed fields of one slab [NMIX][slab][L3][nxh]
  int nmix;
  int slab;                // planes per transform slab (Ny unless the mixed fields would pass 8 GiB)
  int fslab;               // planes per slab of the filter pass (its products and outputs within 4 GiB)
  double2* pbb;            // filter pass: products of the filtered velocities of one slab [6][slab][M]
  double2* fout;           // filter pass: ubar_i, tau_ij of one slab [9][slab][M]
  double2* scr;            // wall-normal sweep scratch [2][Ny][M] (aliases the u_1, u_3 work slots)
  double* G;               // filter transfer [M]
  double* prs;             // filtered-pressure homogeneous solutions [Ny][2][C] (lazy)
  double* prsinv;          // their inverse wall-derivative matrices [4][C]
  double2* dbrec;          // compact database record (lazily allocated)
  size_t dbrec_n;          // its capacity in complex values
  int g_kind;              // filter whose transfer function G holds (-1: none)
  double g_p1, g_p3;
  double* stat;            // [CHAN_NSTAT][Ny] + [2] (utau, ubulk)
  // bookkeeping
  bool have_state, have_filter;
  long long nsub;
  double t;
  size_t dev_bytes;
  std::string err;
  FftPlan p1, p3;
  std::vector<void*> allocs;
  // launch shapes (0: default), set by chan_autotune
  int kb_z;                // columns per z-pass CTA
  int xthreads;            // threads per x-pass CTA
  int ytab;                // y sweeps: 1 read tables from global memory, 0 stage them in shared memory,
                           // -1 (default) stage them unless that needs more than 16 KB per CTA
  // CUDA graph of one full RK3 step (three substeps), captured on first use
  bool use_graph;
  cudaGraphExec_t gexec;
  long long graph_launches[KID_COUNT];   // kernels one replay runs, per kernel id
  // tracing
  bool prof;
  long long launches[KID_COUNT];
  std::vector<ProfRec> recs;     // event pairs recorded since the last reset
  size_t nrec;                   // pairs in use
};

// Work-field pointers of one run in a packed substep.
struct BatchWork {
  double2 *u1, *u3, *om1, *om3, *H1, *H2, *H3, *Nchi, *Nom;
  void* mixed[6];
};

// Kernel launchers (return cudaGetLastError()).
cudaError_t launch_setup_tables(chan_s* h);
// Lean tables: refill the single Helmholtz slot for substep s (no-op otherwise).
cudaError_t launch_setup_substep(chan_s* h, int s);
// Poisson factors [Ny][7][C] into dst (lean 2: h->pois each substep, or the filtered pressure's own).
cudaError_t launch_setup_pois(chan_s* h, double* dst);
// Lean 2: the (0,0) modes of H1, H3 into h->h00, for the mean-flow solve.
cudaError_t launch_copy_mean_modes(chan_s* h, const double2* H1, const double2* H3);
cudaError_t launch_derive(chan_s* h);
// f32: the mixed mode's substep variant (float2 transform inputs, see substep_inputs).
cudaError_t launch_pre(chan_s* h, double2* u1, double2* u3, double2* om1, double2* om3, bool f32 = false);
cudaError_t launch_nonlin(chan_s* h, const double2* H1, const double2* H2, const double2* H3,
                          double2* Nchi, double2* Nom);
// k_nonlin with a caller-chosen scratch buffer of Ny * M double2.
cudaError_t launch_nonlin_scratch(chan_s* h, const double2* H1, const double2* H2, const double2* H3,
                                  double2* Nchi, double2* Nom, double2* scr);
cudaError_t launch_helm(chan_s* h, const double2* Nchi, const double2* Nom, int s);
cudaError_t launch_poisson(chan_s* h, int s);
// st: the stream to launch on (NULL: the handle's stream)
cudaError_t launch_mean(chan_s* h, const double2* H1, const double2* H3, int s, cudaStream_t st = nullptr);
// Filter epilogue over ny planes (pointers at the slab's first plane).
// puu holds P(u'_i u'_j) of the fluctuations on entry and P(u_i u_j) on return; the planes
// start at y0.
cudaError_t launch_filter_out(chan_s* h, const double2* const* u, double2* const* puu,
                              const double2* const* pbb, double2* const* ubar, double2* const* tau, int y0, int ny);
cudaError_t launch_apply_G(chan_s* h, const double2* in, double2* out);
// Double-float storage: n complex values to (hi, lo) pairs in place; pairs back to FP64
// (src == dst allowed).
cudaError_t launch_to_pairs(chan_s* h, double2* p, size_t n);
cudaError_t launch_from_pairs(chan_s* h, const double2* src, double2* dst, size_t n);
cudaError_t launch_pressure(chan_s* h, const double2* const* P, double2* out);
cudaError_t launch_setup_pressure(chan_s* h);
// Retained modes of ny planes (src at the first plane, dst at its first row).
cudaError_t launch_gather_retained(chan_s* h, const double2* src, double2* dst, int M1, int M3, int ny);
cudaError_t launch_spectra(chan_s* h, const double2* u1, const double2* u3, double* E);
cudaError_t launch_stats(chan_s* h, const double2* u1, const double2* u3, int zero_filtered);
// <ubar_i ubar_j> and <tau_ij> rows of planes y0 .. y0+ny-1 from the slab's filter outputs.
cudaError_t launch_stats_filtered(chan_s* h, const double2* const* ubar, const double2* const* tau, int y0, int ny);

// Persistent work-list launches of a batch (kernels_persist.cu): the stage table and device
// argument table of n <= CHAN_MAXBATCH runs; one launch of nsub[r] (0 .. persist_max_substeps())
// substeps of each run r; whether a bounded wait of a launch gave up since the last status
// call; the wait limit and a (run, stage) that is made to need one completion more (tests).
struct PersistPlan;
cudaError_t persist_create(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st, PersistPlan** out);
cudaError_t persist_launch(PersistPlan* P, chan_s* const* hs, const int* nsub, cudaStream_t st);
int persist_max_substeps();
cudaError_t persist_status(PersistPlan* P, cudaStream_t st, int* timed_out);
void persist_set_wait(PersistPlan* P, long long spins, int hold_run, int hold_stage);
int persist_grid(const PersistPlan* P);
void persist_free(PersistPlan* P, cudaStream_t st);

// Packed launches over n <= CHAN_MAXBATCH runs of one precision, on `st`.
cudaError_t launch_pre_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);
cudaError_t launch_nonlin_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);
cudaError_t launch_helm_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);
cudaError_t launch_poisson_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);
cudaError_t launch_mean_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);
cudaError_t launch_zinv_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);
cudaError_t launch_xpass_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);
cudaError_t launch_zfwd_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st);

// FFT passes.  in/out are arrays of nf device pointers.
// Transform passes over ny planes; the pointers address the first plane of the slab.
// f32_mask (mixed mode only): bit f set = input f is stored as float2 [Ny][M].
// skip00: every field's (0,0) mode (its plane mean) is transformed as zero.
cudaError_t launch_zinv(chan_s* h, const double2* const* in, const int* apply_G, void* const* out, int nf, int ny,
                        int f32_mask, int skip00 = 0);
// The six substep transform inputs (u1, v, u3, w1, w2, w3) from plane y0 on, given the
// work slots of the pre kernel's outputs, and their float2 mask: in the mixed mode the
// substep's pre kernel leaves u1, u3 as float2 [2][Ny][M] in the w1 slot and w1, w3 in
// the w3 slot (its u1, u3 slots hold the forward sweep).
int substep_inputs(const chan_s* h, double2* u1, double2* u3, double2* om1, double2* om3, size_t y0,
                   const double2** in);
cudaError_t launch_xpass(chan_s* h, int mode, void* const* in, void* const* out, int ny);
// pair_out: in the double-float mode write (hi, lo) pairs (substep fields) instead of FP64.
cudaError_t launch_zfwd(chan_s* h, void* const* in, double2* const* out, int nf, int ny, int pair_out);
cudaError_t fft_configure(chan_s* h);
// Default z-pass columns per CTA: as many as fit 56 KB of shared memory, at most 16.
int pick_kb(int nxh, int L3, size_t es);
// Row stride (elements) of an in-CTA transform buffer of length L and element size es.
int fft_ld(int L, size_t es);
// The same for the x-pass rows (the FP32 two-pass layout when L has a split).
int fft_ld_x(int L, size_t es);
// The two factors of an FP32 two-pass transform of length L (both register-resident
// transform sizes, r1 even); false when L has no such split (the stage transforms serve it).
bool fft_split(int L, int* r1, int* r2);
// Register-transform category of a plan (0: stage transforms; 3: at most 256 x-pass threads).
int fft_plan_category(const FftPlan& pl);
