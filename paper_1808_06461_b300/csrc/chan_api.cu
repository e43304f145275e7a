// C ABI of the channel library (declared in include/chan.h): handle life
// cycle, device memory, state I/O and the ordering of the substep kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

#include "chan_internal.cuh"

double chan_rk3_weight(int s);

namespace {

thread_local std::string g_init_err;

struct Fail {
  int code;
};

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      throw Fail{e_ == cudaErrorMemoryAllocation ? CHAN_ENOMEM : CHAN_ECUDA};           \
    }                                                                                   \
  } while (0)

int bad(chan_s* h, const std::string& msg, int code = CHAN_EINVAL) {
  if (h) h->err = msg;
  else g_init_err = msg;
  return code;
}

// Device memory of a handle comes from the device's stream-ordered pool on the handle's
// stream (cudaMallocAsync / cudaFreeAsync): releasing a run does not synchronise the
// device, so a serving loop that retires runs keeps the other runs' work in flight.
template <typename T>
T* dalloc(chan_s* h, size_t n) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, n * sizeof(T), h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();   // a failed allocation must not surface later as a launch error
    h->err = std::string("cudaMalloc of ") + std::to_string(n * sizeof(T)) + " bytes: " + cudaGetErrorString(e);
    throw Fail{CHAN_ENOMEM};
  }
  h->allocs.push_back(p);
  h->dev_bytes += n * sizeof(T);
  return static_cast<T*>(p);
}

bool is_2a3b(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

__global__ void k_flux(const double* U1, const double* wq, int Ny, double* scal) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double q = 0.0;
    for (int i = 0; i < Ny; ++i) q += wq[i] * U1[i];
    scal[1] = q;
    scal[0] = 0.0;
    scal[2] = 0.0;   // no Helmholtz right-hand sides of a previous substep yet
  }
}

size_t fsize(const chan_s* h) { return (size_t)h->Ny * h->M; }

const char* const kKernelNames[KID_COUNT] = {"k_pre",     "k_zinv",       "k_xpass", "k_zfwd",
                                             "k_nonlin",  "k_helm",       "k_poisson", "k_mean",
                                             "k_filter_out", "k_stats",   "k_derive", "k_apply_G",
                                             "k_gather_retained", "k_spectra", "k_pressure", "k_setup_helm",
                                             "k_setup_pois", "k_copy_mean_modes"};

// Launch bracket: counts the launch and, when tracing, records an event pair.
struct Traced {
  chan_s* h;
  ProfRec* r;
  cudaStream_t st;
  Traced(chan_s* hh, int k, cudaStream_t s = nullptr) : h(hh), r(nullptr), st(s ? s : hh->stream) {
    h->launches[k] += 1;
    if (!h->prof) return;
    if (h->nrec == h->recs.size()) {
      ProfRec n{k, nullptr, nullptr};
      if (cudaEventCreate(&n.a) != cudaSuccess || cudaEventCreate(&n.b) != cudaSuccess) return;
      h->recs.push_back(n);
    }
    r = &h->recs[h->nrec++];
    r->k = k;
    cudaEventRecord(r->a, st);
  }
  ~Traced() {
    if (r) cudaEventRecord(r->b, st);
  }
};

// Work-field slots (Fourier layout)
// (u_1, u_3 double as the sweep scratch once the transforms have read them; the
// filter pass puts P(u_i u_j) in slots 2..7 and the filtered pressure its output in 8)
enum { WF_U1 = 0, WF_U3 = 1, WF_OM1 = 2, WF_OM3 = 3, WF_H1 = 4, WF_H2 = 5, WF_H3 = 6, WF_NCHI = 7, WF_NOM = 8, NWF = 9 };

double2* wf(chan_s* h, int k) { return h->wf + (size_t)k * fsize(h); }
void* mixed(chan_s* h, int k) {
  const size_t es = prec_t32(h->prec) ? sizeof(float2) : sizeof(double2);
  return static_cast<char*>(h->mixed) + (size_t)k * h->slab * h->L3 * h->nxh * es;
}

// Planes per slab of the transform passes (see chan_opts.slab_planes).
int slab_planes(int Nx, int Ny, int Nz, int prec, int req) {
  if (req > 0) return req < Ny ? req : Ny;
  const size_t es = prec_t32(prec) ? sizeof(float2) : sizeof(double2);
  const size_t plane = 12 * (size_t)(3 * Nz / 2) * (size_t)(Nx / 2) * es;
  size_t smax = ((size_t)8 << 30) / plane;
  if (smax < 1) smax = 1;
  if ((size_t)Ny <= smax) return Ny;
  const size_t nslab = (Ny + smax - 1) / smax;
  return (int)((Ny + nslab - 1) / nslab);
}

// Planes per slab of the filter pass: its six products and nine outputs ([15][slab][M]
// complex doubles) within 4 GiB, and no more planes than a transform slab.
int filter_slab(int Nx, int Nz, int slab) {
  const size_t per_plane = 15 * (size_t)Nz * (size_t)(Nx / 2) * sizeof(double2);
  size_t s = ((size_t)4 << 30) / per_plane;
  if (s < 1) s = 1;
  return (size_t)slab < s ? slab : (int)s;
}

void clean_modes(chan_s* h, double2* f) {
  const size_t pitch = (size_t)h->M * sizeof(double2);
  CK(cudaMemset2DAsync(f, pitch, 0, sizeof(double2), h->Ny, h->stream));                    // (0,0) mode
  CK(cudaMemset2DAsync(f + (size_t)(h->Nz / 2) * h->nxh, pitch, 0, (size_t)h->nxh * sizeof(double2), h->Ny,
                       h->stream));                                                             // kz Nyquist row
}

void after_state_upload(chan_s* h) {
  clean_modes(h, h->v);
  clean_modes(h, h->om);
  { Traced t(h, KID_DERIVE); CK(launch_derive(h)); }
  if (prec_pairs(h->prec))   // the substep keeps its Fourier fields as FP32 pairs
    for (double2* f : {h->v, h->om, h->chi, h->dv}) CK(launch_to_pairs(h, f, fsize(h)));
  CK(cudaMemsetAsync(h->Nchi_p, 0, fsize(h) * sizeof(double2), h->stream));
  CK(cudaMemsetAsync(h->Nom_p, 0, fsize(h) * sizeof(double2), h->stream));
  CK(cudaMemsetAsync(h->H1m_p, 0, h->Ny * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->H3m_p, 0, h->Ny * sizeof(double), h->stream));
  k_flux<<<1, 32, 0, h->stream>>>(h->U1, h->tab_wq, h->Ny, h->scal);
  CK(cudaGetLastError());
  h->have_state = true;
  h->have_filter = false;
  h->nsub = 0;
  h->t = 0.0;
}

}  // namespace

int substep_inputs(const chan_s* h, double2* u1, double2* u3, double2* om1, double2* om3, size_t y0,
                   const double2** in) {
  const size_t o = y0 * h->M, nf = fsize(h);
  in[1] = h->v + o;
  in[4] = h->om + o;
  if (!prec_t32(h->prec)) {
    in[0] = u1 + o; in[2] = u3 + o; in[3] = om1 + o; in[5] = om3 + o;
    return 0;
  }
  const float2* fu = reinterpret_cast<const float2*>(om1);
  const float2* fw = reinterpret_cast<const float2*>(om3);
  in[0] = reinterpret_cast<const double2*>(fu + o);
  in[2] = reinterpret_cast<const double2*>(fu + nf + o);
  in[3] = reinterpret_cast<const double2*>(fw + o);
  in[5] = reinterpret_cast<const double2*>(fw + nf + o);
  return (1 << 0) | (1 << 2) | (1 << 3) | (1 << 5);
}

namespace {

// u_1, u_3, omega_1, omega_3 of the current state into the work slots (f32: the mixed
// mode's substep layout, see substep_inputs).
void run_pre(chan_s* h, bool f32 = false) {
  Traced t(h, KID_PRE);
  CK(launch_pre(h, wf(h, WF_U1), wf(h, WF_U3), wf(h, WF_OM1), wf(h, WF_OM3), f32));
}

// H = u x omega of the current state into WF_H1..WF_H3 (after run_pre).
// The transforms are plane-local: slab by slab through the mixed buffers (after
// run_pre(h, true)).
void run_nonlinear(chan_s* h) {
  void* mx[6] = {mixed(h, 0), mixed(h, 1), mixed(h, 2), mixed(h, 3), mixed(h, 4), mixed(h, 5)};
  for (int y0 = 0; y0 < h->Ny; y0 += h->slab) {
    const int ny = h->Ny - y0 < h->slab ? h->Ny - y0 : h->slab;
    const size_t o = (size_t)y0 * h->M;
    const double2* in[6];
    const int mask = substep_inputs(h, wf(h, WF_U1), wf(h, WF_U3), wf(h, WF_OM1), wf(h, WF_OM3), (size_t)y0, in);
    { Traced t(h, KID_ZINV); CK(launch_zinv(h, in, nullptr, mx, 6, ny, mask)); }
    { Traced t(h, KID_XPASS); CK(launch_xpass(h, 0, mx, mx, ny)); }
    double2* Hout[3] = {wf(h, WF_H1) + o, wf(h, WF_H2) + o, wf(h, WF_H3) + o};
    { Traced t(h, KID_ZFWD); CK(launch_zfwd(h, mx, Hout, 3, ny, 1)); }
  }
}

void run_substep(chan_s* h) {
  const int s = (int)(h->nsub % 3);
  if (h->lean == 1) { Traced t(h, KID_TABLES); CK(launch_setup_substep(h, s)); }
  run_pre(h, true);
  run_nonlinear(h);
  // The mean-flow solve (one CTA) needs only the (0,0) modes of H and the mean profiles,
  // which the wall-normal sweeps neither read nor write: it runs on the side stream beside
  // them, and the next substep waits for it.  With the tables in the work slots it reads
  // copies of the (0,0) modes, since the table set-up below overwrites H.
  if (h->lean == 2) { Traced t(h, KID_COPY_MEAN); CK(launch_copy_mean_modes(h, wf(h, WF_H1), wf(h, WF_H3))); }
  CK(cudaEventRecord(h->ev_fork, h->stream));
  CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  { Traced t(h, KID_MEAN, h->side); CK(launch_mean(h, wf(h, WF_H1), wf(h, WF_H3), s, h->side)); }
  CK(cudaEventRecord(h->ev_join, h->side));
  { Traced t(h, KID_NONLIN); CK(launch_nonlin(h, wf(h, WF_H1), wf(h, WF_H2), wf(h, WF_H3), wf(h, WF_NCHI), wf(h, WF_NOM))); }
  if (h->lean == 2) {   // omega_1 .. H_3 are dead until the next substep: the tables go there
    { Traced t(h, KID_SETUP_POIS); CK(launch_setup_pois(h, h->pois)); }
    { Traced t(h, KID_TABLES); CK(launch_setup_substep(h, s)); }
  }
  { Traced t(h, KID_HELM); CK(launch_helm(h, wf(h, WF_NCHI), wf(h, WF_NOM), s)); }
  { Traced t(h, KID_POISSON); CK(launch_poisson(h, s)); }
  CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  h->t += chan_rk3_weight(s) * h->dt;
  h->nsub += 1;
}

void ensure_filter_buffers(chan_s* h) {
  if (h->G) return;
  h->G = dalloc<double>(h, h->M);
}

// Filter transfer function on the stored modes (Sec. 3.1; kz Nyquist row zero) into h->G.
void set_filter(chan_s* h, int kind, double p1, double p3) {
  ensure_filter_buffers(h);
  if (h->g_kind == kind && h->g_p1 == p1 && h->g_p3 == p3) return;   // already on the device
  std::vector<double> G(h->M);
  for (int jz = 0; jz < h->Nz; ++jz)
    for (int kx = 0; kx < h->nxh; ++kx) {
      const double k1 = 2.0 * M_PI / h->Lx * kx;
      const double k3 = 2.0 * M_PI / h->Lz * (jz < h->Nz / 2 ? jz : jz - h->Nz);
      double g;
      if (kind == CHAN_FILTER_SHARP) {
        g = (std::fabs(k1) < M_PI * h->re / p1 && std::fabs(k3) < M_PI * h->re / p3) ? 1.0 : 0.0;
      } else {
        const double a = 0.5 * k1 * p1 / h->re, b = 0.5 * k3 * p3 / h->re;
        g = (a == 0.0 ? 1.0 : std::sin(a) / a) * (b == 0.0 ? 1.0 : std::sin(b) / b);
      }
      G[(size_t)jz * h->nxh + kx] = (jz == h->Nz / 2) ? 0.0 : g;
    }
  CK(cudaMemcpyAsync(h->G, G.data(), h->M * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));   // the host vector dies here
  h->g_kind = kind;
  h->g_p1 = p1;
  h->g_p3 = p3;
}

// Device bytes chan_init_ex requests for a box (the filter transfer function,
// allocated on the first filter call, included).  Mirrors the allocations below.
size_t footprint_ex(int Nx, int Ny, int Nz, int prec, int slab_req, int lean, int keep) {
  const size_t nxh = Nx / 2, M = (size_t)Nz * nxh, C = (size_t)(Nz / 2) * nxh, n = (size_t)Ny * M;
  const size_t nslot = lean ? 1 : 3;
  const size_t ntab = lean == 2 ? 0 : (size_t)Ny * 7 * C + nslot * (size_t)Ny * 11 * C;   // lean 2: in the work slots
  const size_t L1 = 3 * (size_t)Nx / 2, L3 = 3 * (size_t)Nz / 2;
  const size_t es = prec_t32(prec) ? sizeof(float2) : sizeof(double2);
  size_t b = 0;
  b += (keep ? 8 : 6) * n * sizeof(double2) + 4 * Ny * sizeof(double) + 3 * sizeof(double);   // state
  b += 5 * 7 * (size_t)Ny * sizeof(double) + 3 * (size_t)Ny * sizeof(double);              // y tables
  b += (nxh + Nz) * sizeof(double);                                                          // wavenumbers
  b += (ntab + nslot * 4 * C + 3 * ((size_t)Ny + 1)) * sizeof(double);
  if (lean == 2) b += 3 * 11 * (size_t)Ny * sizeof(double) + 2 * (size_t)Ny * sizeof(double2);   // mean_tab, h00
  if (prec_pairs(prec))
    b += ((size_t)Ny * 7 * C + nslot * (size_t)Ny * 11 * C + nslot * 4 * C + 30 * (size_t)Ny) * sizeof(dfr);
  b += (L1 + L3) * (prec_t32(prec) ? sizeof(float2) : sizeof(double2));             // twiddles
  {                                                                                          // two-pass twiddles (x)
    int r1, r2;
    if (prec_t32(prec) && fft_split((int)L1, &r1, &r2)) b += (size_t)r1 * (r2 + 1) * sizeof(float2);
  }
  b += (L1 + L3) * sizeof(int);                                                              // block twiddle exponents
  const size_t S = slab_planes(Nx, Ny, Nz, prec, slab_req);
  b += (size_t)NWF * n * sizeof(double2);                                                    // work fields
  b += 12 * S * L3 * nxh * es;                                                               // mixed fields
  b += (6 + 9) * (size_t)filter_slab(Nx, Nz, (int)S) * M * sizeof(double2);                 // filter products, outputs
  b += (CHAN_NSTAT * (size_t)Ny + 2) * sizeof(double);                                       // statistics
  b += M * sizeof(double);                                                                   // filter G
  return b;
}

// Table placement (see chan_s::lean): as asked, or automatically: one substep's tables when
// the box would pass 200 GB with all three, and those in the work slots when it would still
// pass 150 GB without the kept right-hand sides.  The pair modes keep pair copies of the
// tables beside the FP64 ones, which the work slots cannot hold: level 2 is level 1 there.
int lean_tables(int Nx, int Ny, int Nz, int prec, int slab_req, int req) {
  if (req < 0) return 0;
  if (req > 0) return req == 2 && !prec_pairs(prec) ? 2 : 1;
  if (footprint_ex(Nx, Ny, Nz, prec, slab_req, 0, 1) <= (size_t)200e9) return 0;
  if (prec_pairs(prec) || footprint_ex(Nx, Ny, Nz, prec, slab_req, 1, 0) <= (size_t)150e9) return 1;
  return 2;
}

// Kept Helmholtz right-hand sides unless asked not to, or automatically when the box would
// pass 150 GB with them.
int keep_rhs(int Nx, int Ny, int Nz, int prec, int slab_req, int lean, int req) {
  if (req != 0) return req > 0;
  return footprint_ex(Nx, Ny, Nz, prec, slab_req, lean, 1) <= (size_t)150e9;
}

size_t footprint(int Nx, int Ny, int Nz, int prec) {   // automatic slab, table and right-hand-side choice
  const int lean = lean_tables(Nx, Ny, Nz, prec, 0, 0);
  return footprint_ex(Nx, Ny, Nz, prec, 0, lean, keep_rhs(Nx, Ny, Nz, prec, 0, lean, 0));
}

// Capture one RK3 step (substeps 0, 1, 2) into a graph; the handle's
// counters are left untouched.
void capture_step_graph(chan_s* h) {
  const long long nsub0 = h->nsub;
  const double t0 = h->t;
  long long before[KID_COUNT];
  for (int k = 0; k < KID_COUNT; ++k) before[k] = h->launches[k];
  const bool prof = h->prof;
  h->prof = false;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
  try {
    for (int k = 0; k < 3; ++k) run_substep(h);
  } catch (Fail f) {
    cudaStreamEndCapture(h->stream, &g);
    if (g) cudaGraphDestroy(g);
    h->prof = prof;
    throw;
  }
  CK(cudaStreamEndCapture(h->stream, &g));
  cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  for (int k = 0; k < KID_COUNT; ++k) {
    h->graph_launches[k] = h->launches[k] - before[k];
    h->launches[k] = before[k];
  }
  h->nsub = nsub0;
  h->t = t0;
  h->prof = prof;
}

BatchWork batch_work(chan_s* h) {
  BatchWork w;
  w.u1 = wf(h, WF_U1); w.u3 = wf(h, WF_U3); w.om1 = wf(h, WF_OM1); w.om3 = wf(h, WF_OM3);
  w.H1 = wf(h, WF_H1); w.H2 = wf(h, WF_H2); w.H3 = wf(h, WF_H3); w.Nchi = wf(h, WF_NCHI); w.Nom = wf(h, WF_NOM);
  for (int f = 0; f < 6; ++f) w.mixed[f] = mixed(h, f);
  return w;
}

}  // namespace

struct chan_batch_s {
  std::vector<chan_s*> runs;
  cudaStream_t stream;
  bool own_stream;
  std::vector<cudaEvent_t> ev;   // one per run (join) + one (fork)
  cudaGraphExec_t gexec;
  PersistPlan* plan;             // persistent work-list launches (CHAN_BATCH_PERSISTENT), else NULL
  std::string err;
};

namespace {

#define BK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      throw Fail{CHAN_ECUDA};                                                           \
    }                                                                                   \
  } while (0)

// One substep of every run of the batch, in packed launches of up to
// CHAN_MAXBATCH runs each (all runs are at their own RK3 phase).
void batch_substep(chan_batch_s* b) {
  const int n = (int)b->runs.size();
  for (int r0 = 0; r0 < n; r0 += CHAN_MAXBATCH) {
    const int m = n - r0 < CHAN_MAXBATCH ? n - r0 : CHAN_MAXBATCH;
    chan_s* const* hs = b->runs.data() + r0;
    BatchWork w[CHAN_MAXBATCH];
    for (int r = 0; r < m; ++r) w[r] = batch_work(hs[r]);
    BK(launch_pre_batch(hs, m, w, b->stream));
    BK(launch_zinv_batch(hs, m, w, b->stream));
    BK(launch_xpass_batch(hs, m, w, b->stream));
    BK(launch_zfwd_batch(hs, m, w, b->stream));
    BK(launch_nonlin_batch(hs, m, w, b->stream));
    BK(launch_helm_batch(hs, m, w, b->stream));
    BK(launch_poisson_batch(hs, m, w, b->stream));
    BK(launch_mean_batch(hs, m, w, b->stream));
  }
  for (chan_s* h : b->runs) {
    h->t += chan_rk3_weight((int)(h->nsub % 3)) * h->dt;
    h->nsub += 1;
    h->have_filter = false;
  }
}

}  // namespace

// The filter outputs of one slab: ubar_i (k = 0..2) and tau_ij (k = 3..8), [slab][M] each.
static double2* filt(chan_s* h, int k) { return h->fout + (size_t)k * h->fslab * h->M; }

// The filter pass (Sec. 3.1), slab by slab: P(u_i u_j) to work slots 2..7 (kept for the
// filtered pressure and the database record), P(ubar_i ubar_j) to the slab buffer, then
// ubar_i and tau_ij of the slab, which leave for the host arrays (when given), for the
// filtered statistics rows and, when a database record is being built (rec != NULL),
// for its ubar_i blocks on the retained modes (M1 x M3).
static void filter_pass(chan_s* h, int kind, double p1, double p3, double* host_ubar, double* host_tau,
                        double2* rec, int M1, int M3) {
  set_filter(h, kind, p1, p3);
  run_pre(h);
  const int applyG[6] = {0, 0, 0, 1, 1, 1};
  void* mx[12];
  for (int k = 0; k < 12; ++k) mx[k] = mixed(h, k);
  const size_t n = fsize(h), sn = (size_t)h->fslab * h->M;
  for (int y0 = 0; y0 < h->Ny; y0 += h->fslab) {
    const int ny = h->Ny - y0 < h->fslab ? h->Ny - y0 : h->fslab;
    const size_t o = (size_t)y0 * h->M;
    const double2* u[3] = {wf(h, WF_U1) + o, h->v + o, wf(h, WF_U3) + o};
    const double2* in[6] = {u[0], u[1], u[2], u[0], u[1], u[2]};
    // the products are formed from the fluctuations (the (0,0) modes taken as zero); the
    // epilogue adds the mean parts back where they do not cancel
    { Traced t(h, KID_ZINV); CK(launch_zinv(h, in, applyG, mx, 6, ny, 0, 1)); }
    { Traced t(h, KID_XPASS); CK(launch_xpass(h, 1, mx + 3, mx + 6, ny)); }   // ubar'_i ubar'_j -> slots 6..11
    { Traced t(h, KID_XPASS); CK(launch_xpass(h, 1, mx, mx, ny)); }           // u'_i u'_j       -> slots 0..5
    double2* fo[12];
    for (int k = 0; k < 6; ++k) { fo[k] = wf(h, 2 + k) + o; fo[6 + k] = h->pbb + k * sn; }
    { Traced t(h, KID_ZFWD); CK(launch_zfwd(h, mx, fo, 12, ny, 0)); }
    double2* puu[6] = {fo[0], fo[1], fo[2], fo[3], fo[4], fo[5]};
    const double2* pbb[6] = {fo[6], fo[7], fo[8], fo[9], fo[10], fo[11]};
    double2* ub[3];
    double2* ta[6];
    for (int k = 0; k < 3; ++k) ub[k] = filt(h, k);
    for (int k = 0; k < 6; ++k) ta[k] = filt(h, 3 + k);
    { Traced t(h, KID_FILTER_OUT); CK(launch_filter_out(h, u, puu, pbb, ub, ta, y0, ny)); }
    const double2* cub[3] = {ub[0], ub[1], ub[2]};
    const double2* cta[6] = {ta[0], ta[1], ta[2], ta[3], ta[4], ta[5]};
    { Traced t(h, KID_STATS); CK(launch_stats_filtered(h, cub, cta, y0, ny)); }
    const size_t bytes = (size_t)ny * h->M * sizeof(double2);
    for (int k = 0; k < 3 && host_ubar; ++k)
      CK(cudaMemcpyAsync(reinterpret_cast<double2*>(host_ubar) + k * n + o, ub[k], bytes, cudaMemcpyDeviceToHost,
                         h->stream));
    for (int k = 0; k < 6 && host_tau; ++k)
      CK(cudaMemcpyAsync(reinterpret_cast<double2*>(host_tau) + k * n + o, ta[k], bytes, cudaMemcpyDeviceToHost,
                         h->stream));
    if (rec) {
      const size_t blk = (size_t)h->Ny * M3 * M1;
      for (int k = 0; k < 3; ++k) {
        Traced t(h, KID_GATHER);
        CK(launch_gather_retained(h, ub[k], rec + k * blk + (size_t)y0 * M3 * M1, M1, M3, ny));
      }
    }
  }
  if (host_ubar || host_tau) CK(cudaStreamSynchronize(h->stream));
  h->have_filter = true;
}

extern "C" {

void chan_opts_default(chan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eta_w = 1.0;
  o->grid_re = 0.0;
  o->precision = CHAN_PREC_FP64;
  o->stream = nullptr;
}

int chan_init(chan_t* out, double re_tau, double Lx, double Lz, int Nx, int Ny, int Nz, double dt) {
  chan_opts o;
  chan_opts_default(&o);
  o.re_tau = re_tau; o.Lx = Lx; o.Lz = Lz; o.Nx = Nx; o.Ny = Ny; o.Nz = Nz; o.dt = dt;
  return chan_init_ex(out, &o);
}

int chan_init_ex(chan_t* out, const chan_opts* o) {
  if (!out) return bad(nullptr, "chan_init: out is NULL");
  *out = nullptr;
  if (!o) return bad(nullptr, "chan_init: opts is NULL");
  if (!(o->re_tau > 0) || !(o->Lx > 0) || !(o->Lz > 0) || !(o->dt > 0) || !std::isfinite(o->dt))
    return bad(nullptr, "chan_init: re_tau, Lx, Lz and dt must be positive");
  if (o->Nx < 2 || o->Nx % 2 || !is_2a3b(o->Nx)) return bad(nullptr, "chan_init: Nx must be even and 2^a 3^b");
  if (o->Nz < 4 || o->Nz % 4 || !is_2a3b(o->Nz)) return bad(nullptr, "chan_init: Nz must be a multiple of 4 and 2^a 3^b");
  if (o->Ny < 9 || o->Ny % 2 == 0) return bad(nullptr, "chan_init: Ny must be odd and >= 9");
  if (o->precision != CHAN_PREC_FP64 && o->precision != CHAN_PREC_MIXED && o->precision != CHAN_PREC_F64X &&
      o->precision != CHAN_PREC_MIXED_DF)
    return bad(nullptr, "chan_init: unknown precision");
  if (o->slab_planes < 0) return bad(nullptr, "chan_init: slab_planes must be >= 0");
  if (o->y_tables < 0 || o->y_tables > 2) return bad(nullptr, "chan_init: y_tables must be 0, 1 or 2");
  const int L1 = 3 * o->Nx / 2, L3 = 3 * o->Nz / 2;
  const size_t es = prec_t32(o->precision) ? 8 : 16;
  if (2 * 6 * (size_t)fft_ld_x(L1, es) * es > 227 * 1024 || 2 * (size_t)fft_ld(L3, es) * es > 100 * 1024)
    return bad(nullptr, "chan_init: 3Nx/2 or 3Nz/2 too long for an in-block transform at this precision "
                        "(FP64 and double-float: Nx <= 768, the two mixed modes: Nx <= 1536)");
  chan_s* h = new (std::nothrow) chan_s();
  if (!h) return bad(nullptr, "chan_init: out of host memory", CHAN_ENOMEM);
  h->re = o->re_tau; h->Lx = o->Lx; h->Lz = o->Lz; h->dt = o->dt; h->nu = 1.0 / o->re_tau;
  h->eta_w = o->eta_w > 0 ? o->eta_w : 1.0;
  h->grid_re = o->grid_re > 0 ? o->grid_re : o->re_tau;
  h->Nx = o->Nx; h->Ny = o->Ny; h->Nz = o->Nz; h->nxh = o->Nx / 2;
  h->M = h->Nz * h->nxh; h->C = (h->Nz / 2) * h->nxh;
  h->L1 = L1; h->L3 = L3; h->prec = o->precision;
  h->have_state = h->have_filter = false;
  h->nsub = 0; h->t = 0.0; h->dev_bytes = 0;
  h->G = nullptr;
  h->g_kind = -1;
  h->dbrec = nullptr;
  h->dbrec_n = 0;
  h->prs = nullptr;
  h->prsinv = nullptr;
  int rc = CHAN_OK;
  chanh_tables tb;
  std::memset(&tb, 0, sizeof(tb));
  try {
    CK(cudaGetDevice(&h->device));
    if (o->stream) { h->stream = (cudaStream_t)o->stream; h->own_stream = false; }
    else { CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)); h->own_stream = true; }
    CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    if (o->mesh) {
      const double* m = o->mesh;
      bool ok = m[0] == -1.0 && m[h->Ny - 1] == 1.0;
      for (int j = 0; ok && j < h->Ny; ++j) ok = (j == 0 || m[j] > m[j - 1]) && m[j] == -m[h->Ny - 1 - j];
      if (!ok) { h->err = "chan_init: mesh must increase from -1 to 1 and be mirror symmetric"; throw Fail{CHAN_EINVAL}; }
    }
    int hr = chanh_build_mesh(h->Ny, h->grid_re, h->eta_w, o->mesh, &tb);
    if (hr) { h->err = "chan_init: compact-scheme set-up failed (singular coefficient system or LU pivot)"; throw Fail{CHAN_EINVAL}; }
    h->y.assign(tb.y, tb.y + h->Ny);
    h->wq.assign(tb.wq, tb.wq + h->Ny);
    for (FftPlan* pl : {&h->p1, &h->p3}) {
      pl->L = pl == &h->p1 ? L1 : L3;
      pl->np = chanh_radix_plan(pl->L, pl->radix);
      // ceil(2^32 / d) for d >= 2; 0 marks d = 1, whose quotient the kernels take as is
      auto mag = [](int d) { return d == 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + d - 1) / d); };
      int Ls = pl->L;
      for (int s = 0; s < pl->np; ++s) {         // DIF stages: block Ls shrinks
        pl->mag_nbf[s] = mag(pl->L / pl->radix[s]);
        pl->mag_mdif[s] = mag(Ls / pl->radix[s]);
        Ls /= pl->radix[s];
      }
      Ls = 1;
      for (int s = pl->np - 1; s >= 0; --s) {    // DIT stages: block grows
        Ls *= pl->radix[s];
        pl->mag_mdit[s] = mag(Ls / pl->radix[s]);
      }
      pl->r1 = pl->r2 = 0;
      pl->mag_r1 = 0;
      pl->tw2p = nullptr;
      // FP32 x transforms run as two register passes; the z transforms keep the stage form (with
      // KB columns per CTA the register passes left too few warps to hide the column loads)
      if (prec_t32(h->prec) && pl == &h->p1 && fft_split(pl->L, &pl->r1, &pl->r2)) pl->mag_r1 = mag(pl->r1);
    }
    const size_t n = fsize(h), Ny = h->Ny;
    // state
    h->v = dalloc<double2>(h, n); h->om = dalloc<double2>(h, n); h->chi = dalloc<double2>(h, n);
    h->dv = dalloc<double2>(h, n); h->Nchi_p = dalloc<double2>(h, n); h->Nom_p = dalloc<double2>(h, n);
    h->U1 = dalloc<double>(h, Ny); h->U3 = dalloc<double>(h, Ny);
    h->H1m_p = dalloc<double>(h, Ny); h->H3m_p = dalloc<double>(h, Ny);
    h->scal = dalloc<double>(h, 3);
    // tables
    double** dst[] = {&h->tab_A2, &h->tab_B2, &h->tab_B1, &h->tab_lu1, &h->tab_lu2f};
    const double* src[] = {tb.A2, tb.B2, tb.B1, tb.lu1, tb.lu2f};
    for (int k = 0; k < 5; ++k) {
      *dst[k] = dalloc<double>(h, 7 * Ny);
      CK(cudaMemcpy(*dst[k], src[k], 7 * Ny * sizeof(double), cudaMemcpyHostToDevice));
    }
    h->tab_d0 = dalloc<double>(h, Ny); h->tab_dN = dalloc<double>(h, Ny); h->tab_wq = dalloc<double>(h, Ny);
    CK(cudaMemcpy(h->tab_d0, tb.d0, Ny * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->tab_dN, tb.dN, Ny * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->tab_wq, tb.wq, Ny * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<double> k1(h->nxh), k3(h->Nz);
    for (int kx = 0; kx < h->nxh; ++kx) k1[kx] = 2.0 * M_PI / h->Lx * kx;
    for (int jz = 0; jz < h->Nz; ++jz) k3[jz] = 2.0 * M_PI / h->Lz * (jz < h->Nz / 2 ? jz : jz - h->Nz);
    h->k1 = dalloc<double>(h, h->nxh); h->k3 = dalloc<double>(h, h->Nz);
    CK(cudaMemcpy(h->k1, k1.data(), h->nxh * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->k3, k3.data(), h->Nz * sizeof(double), cudaMemcpyHostToDevice));
    h->ytab = o->y_tables == 1 ? 1 : (o->y_tables == 2 ? 0 : -1);
    h->lean = lean_tables(h->Nx, h->Ny, h->Nz, h->prec, o->slab_planes, o->lean_tables);
    const size_t nslot = h->lean ? 1 : 3;
    // kept Helmholtz right-hand sides (without them the Helmholtz steps form B X in every substep)
    h->Rom = h->Rchi = nullptr;
    if (keep_rhs(h->Nx, h->Ny, h->Nz, h->prec, o->slab_planes, h->lean, o->keep_rhs)) {
      h->Rom = dalloc<double2>(h, n);
      h->Rchi = dalloc<double2>(h, n);
    }
    if (h->lean != 2) {   // lean 2: pois and helm point into the work slots (below)
      h->pois = dalloc<double>(h, Ny * 7 * (size_t)h->C);
      h->helm = dalloc<double>(h, nslot * Ny * 11 * (size_t)h->C);
    } else {
      h->mean_tab = dalloc<double>(h, 3 * 11 * (size_t)Ny);
      h->h00 = dalloc<double2>(h, 2 * (size_t)Ny);
    }
    h->infl = dalloc<double>(h, nslot * 4 * (size_t)h->C);
    h->meanh = dalloc<double>(h, 3 * (Ny + 1));
    if (prec_pairs(h->prec)) {
      h->tab_pairs = dalloc<dfr>(h, 30 * Ny);
      h->pois_df = dalloc<dfr>(h, Ny * 7 * (size_t)h->C);
      h->helm_df = dalloc<dfr>(h, nslot * Ny * 11 * (size_t)h->C);
      h->infl_df = dalloc<dfr>(h, nslot * 4 * (size_t)h->C);
    }
    // twiddles in the transform precision
    for (int which = 0; which < 2; ++which) {
      const int L = which ? L3 : L1;
      std::vector<double> tw(2 * (size_t)L);
      chanh_twiddles(L, tw.data());
      void* d;
      if (h->prec == CHAN_PREC_FP64) {
        d = dalloc<double2>(h, L);
        CK(cudaMemcpy(d, tw.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
      } else if (h->prec == CHAN_PREC_F64X) {
        // double-float twiddles: (hi, lo) per component, hi = nearest float, lo = nearest float of the rest
        std::vector<float> twd(4 * (size_t)L);
        for (size_t k = 0; k < 2 * (size_t)L; ++k) {
          const float hi = (float)tw[k];
          twd[2 * k] = hi;
          twd[2 * k + 1] = (float)(tw[k] - (double)hi);
        }
        d = dalloc<double2>(h, L);
        CK(cudaMemcpy(d, twd.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
      } else {
        std::vector<float> twf(2 * (size_t)L);
        for (size_t k = 0; k < twf.size(); ++k) twf[k] = (float)tw[k];
        d = dalloc<float2>(h, L);
        CK(cudaMemcpy(d, twf.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
        FftPlan* pl = which ? &h->p3 : &h->p1;
        if (pl->r1) {   // two-pass twiddles w_L^(-n2 k1), rows of r2 + 1
          const int r1 = pl->r1, r2 = pl->r2;
          std::vector<float> t2(2 * (size_t)r1 * (r2 + 1), 0.f);
          for (int k1 = 0; k1 < r1; ++k1)
            for (int n2 = 0; n2 < r2; ++n2) {
              t2[2 * ((size_t)k1 * (r2 + 1) + n2)] = twf[2 * (size_t)n2 * k1];
              t2[2 * ((size_t)k1 * (r2 + 1) + n2) + 1] = twf[2 * (size_t)n2 * k1 + 1];
            }
          float2* d2 = dalloc<float2>(h, (size_t)r1 * (r2 + 1));
          CK(cudaMemcpy(d2, t2.data(), t2.size() * sizeof(float), cudaMemcpyHostToDevice));
          pl->tw2p = d2;
        }
      }
      (which ? h->tw3 : h->tw1) = d;
    }
    // block twiddle exponents of the inverse transform stages (fewer than L per plan)
    for (FftPlan* pl : {&h->p1, &h->p3}) {
      std::vector<int> tab;
      int Ls = pl->L, P = 1;
      for (int s = 0; s < pl->np; ++s) {
        const int R = pl->radix[s], m = Ls / R, nblk = pl->L / Ls;
        pl->revoff[s] = (int)tab.size();
        for (int b = 0; b < nblk; ++b) {
          int K = 0, bb = b, w = P;
          for (int i = s - 1; i >= 0; --i) {   // least significant digit of b = radix of stage s-1
            w /= pl->radix[i];
            K += (bb % pl->radix[i]) * w;
            bb /= pl->radix[i];
          }
          tab.push_back(K * m);
        }
        Ls = m;
        P *= R;
      }
      int* d = dalloc<int>(h, pl->L);
      CK(cudaMemcpy(d, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice));
      pl->revK = d;
    }
    // work
    h->nwf = NWF;
    h->wf = dalloc<double2>(h, (size_t)h->nwf * n);
    h->nmix = 12;
    h->slab = slab_planes(h->Nx, h->Ny, h->Nz, h->prec, o->slab_planes);
    h->mixed = dalloc<unsigned char>(h, (size_t)h->nmix * h->slab * L3 * h->nxh * es);
    h->fslab = filter_slab(h->Nx, h->Nz, h->slab);
    h->pbb = dalloc<double2>(h, 6 * (size_t)h->fslab * h->M);
    h->fout = dalloc<double2>(h, 9 * (size_t)h->fslab * h->M);
    h->scr = wf(h, WF_U1);   // [2][Ny][M]: the u_1, u_3 slots
    if (h->lean == 2) {
      // Poisson factors, then one substep's Helmholtz tables (256-byte aligned), in the slots
      // omega_1 .. H_3 (2..6): 18 Ny C doubles = 9 Ny M of the 10 Ny M those five slots hold
      const size_t np = ((Ny * 7 * (size_t)h->C + 31) / 32) * 32;
      h->pois = reinterpret_cast<double*>(wf(h, WF_OM1));
      h->helm = h->pois + np;
      if (np + Ny * 11 * (size_t)h->C > 5 * 2 * n) { h->err = "chan_init: tables do not fit the work slots"; throw Fail{CHAN_EINVAL}; }
    }
    h->stat = dalloc<double>(h, CHAN_NSTAT * Ny + 2);
    CK(fft_configure(h));
    CK(launch_setup_tables(h));
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    rc = f.code;
  }
  chanh_free(&tb);
  if (rc != CHAN_OK) {
    g_init_err = h->err;
    chan_free(h);
    return rc;
  }
  *out = h;
  return CHAN_OK;
}

void chan_free(chan_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (ProfRec& r : h->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (void* p : h->allocs)
    if (p) cudaFreeAsync(p, h->stream);
  // wait for this stream only: the frees complete and the pool hands the memory back
  // (its release threshold is 0), so a following large allocation finds it
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  delete h;
}

const char* chan_last_error(chan_t h) { return h ? h->err.c_str() : g_init_err.c_str(); }

size_t chan_fourier_count(chan_t h) { return h ? fsize(h) : 0; }
size_t chan_device_bytes(chan_t h) { return h ? h->dev_bytes : 0; }

int chan_get_grid(chan_t h, double* y) {
  if (!h || !y) return bad(h, "chan_get_grid: NULL argument");
  std::memcpy(y, h->y.data(), h->Ny * sizeof(double));
  return CHAN_OK;
}

static int set_state_impl(chan_t h, const void* v, const void* om, const void* U1, const void* U3, cudaMemcpyKind k) {
  if (!h) return bad(nullptr, "chan_set_state: NULL handle");
  if (!v || !om || !U1 || !U3) return bad(h, "chan_set_state: NULL array");
  try {
    const size_t n = fsize(h);
    CK(cudaMemcpyAsync(h->v, v, n * sizeof(double2), k, h->stream));
    CK(cudaMemcpyAsync(h->om, om, n * sizeof(double2), k, h->stream));
    CK(cudaMemcpyAsync(h->U1, U1, h->Ny * sizeof(double), k, h->stream));
    CK(cudaMemcpyAsync(h->U3, U3, h->Ny * sizeof(double), k, h->stream));
    after_state_upload(h);
    if (k == cudaMemcpyHostToDevice) CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_set_state(chan_t h, const double* v, const double* om, const double* U1, const double* U3) {
  return set_state_impl(h, v, om, U1, U3, cudaMemcpyHostToDevice);
}
int chan_set_state_device(chan_t h, const void* v, const void* om, const void* U1, const void* U3) {
  return set_state_impl(h, v, om, U1, U3, cudaMemcpyDeviceToDevice);
}

static int get_state_impl(chan_t h, void* v, void* om, void* U1, void* U3, cudaMemcpyKind k) {
  if (!h) return bad(nullptr, "chan_get_state: NULL handle");
  if (!h->have_state) return bad(h, "chan_get_state: no state set", CHAN_ESTATE);
  try {
    const size_t n = fsize(h);
    const double2* sv = h->v;
    const double2* so = h->om;
    if (prec_pairs(h->prec)) {   // pairs back to FP64: into the caller's device arrays, or the u_1, u_3 slots
      double2* dv_ = k == cudaMemcpyDeviceToDevice ? static_cast<double2*>(v) : wf(h, WF_U1);
      double2* do_ = k == cudaMemcpyDeviceToDevice ? static_cast<double2*>(om) : wf(h, WF_U3);
      if (v) { CK(launch_from_pairs(h, h->v, dv_, n)); sv = dv_; }
      if (om) { CK(launch_from_pairs(h, h->om, do_, n)); so = do_; }
    }
    if (v && sv != v) CK(cudaMemcpyAsync(v, sv, n * sizeof(double2), k, h->stream));
    if (om && so != om) CK(cudaMemcpyAsync(om, so, n * sizeof(double2), k, h->stream));
    if (U1) CK(cudaMemcpyAsync(U1, h->U1, h->Ny * sizeof(double), k, h->stream));
    if (U3) CK(cudaMemcpyAsync(U3, h->U3, h->Ny * sizeof(double), k, h->stream));
    if (k == cudaMemcpyDeviceToHost) {
      CK(cudaStreamSynchronize(h->stream));
      if (U1) {
        const double* u = static_cast<const double*>(U1);
        for (int i = 0; i < h->Ny; ++i)
          if (!std::isfinite(u[i])) return bad(h, "chan_get_state: non-finite mean profile", CHAN_ENAN);
      }
    }
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_get_state(chan_t h, double* v, double* om, double* U1, double* U3) {
  return get_state_impl(h, v, om, U1, U3, cudaMemcpyDeviceToHost);
}
int chan_get_state_device(chan_t h, void* v, void* om, void* U1, void* U3) {
  return get_state_impl(h, v, om, U1, U3, cudaMemcpyDeviceToDevice);
}

// Checkpoint layout: header, then the device arrays in the order of ckpt_arrays.
struct CkptHeader {
  char magic[8];
  int Nx, Ny, Nz, prec;
  double re, Lx, Lz, dt, eta_w, grid_re;
  long long nsub;
  double t;
  int keep_rhs;   // the Helmholtz right-hand sides follow (not for a lean box)
};

static int ckpt_arrays(chan_s* h, void** p, size_t* bytes) {
  const size_t n = fsize(h) * sizeof(double2), ny = h->Ny * sizeof(double);
  void* ptr[] = {h->v, h->om, h->chi, h->dv, h->Nchi_p, h->Nom_p, h->Rom, h->Rchi,
                 h->U1, h->U3, h->H1m_p, h->H3m_p, h->scal};
  const size_t sz[] = {n, n, n, n, n, n, n, n, ny, ny, ny, ny, 3 * sizeof(double)};
  int na = 0;
  for (int k = 0; k < 13; ++k)
    if (ptr[k]) { p[na] = ptr[k]; bytes[na] = sz[k]; ++na; }   // a handle may keep no right-hand sides
  return na;
}

size_t chan_checkpoint_bytes(chan_t h) {
  if (!h) return 0;
  void* p[16];
  size_t b[16], tot = sizeof(CkptHeader);
  const int na = ckpt_arrays(h, p, b);
  for (int k = 0; k < na; ++k) tot += b[k];
  return tot;
}

int chan_checkpoint_save(chan_t h, void* buf) {
  if (!h || !buf) return bad(h, "chan_checkpoint_save: NULL argument");
  if (!h->have_state) return bad(h, "chan_checkpoint_save: no state set", CHAN_ESTATE);
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "CHANCKP2", 8);
  hd.Nx = h->Nx; hd.Ny = h->Ny; hd.Nz = h->Nz; hd.prec = h->prec;
  hd.re = h->re; hd.Lx = h->Lx; hd.Lz = h->Lz; hd.dt = h->dt; hd.eta_w = h->eta_w; hd.grid_re = h->grid_re;
  hd.nsub = h->nsub; hd.t = h->t; hd.keep_rhs = h->Rom != nullptr;
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  try {
    void* p[16];
    size_t b[16];
    const int na = ckpt_arrays(h, p, b);
    for (int k = 0; k < na; ++k) {
      CK(cudaMemcpyAsync(out + off, p[k], b[k], cudaMemcpyDeviceToHost, h->stream));
      off += b[k];
    }
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_checkpoint_load(chan_t h, const void* buf) {
  if (!h || !buf) return bad(h, "chan_checkpoint_load: NULL argument");
  CkptHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "CHANCKP2", 8) != 0) return bad(h, "chan_checkpoint_load: not a checkpoint");
  if (hd.Nx != h->Nx || hd.Ny != h->Ny || hd.Nz != h->Nz || hd.prec != h->prec || hd.re != h->re ||
      hd.Lx != h->Lx || hd.Lz != h->Lz || hd.dt != h->dt || hd.eta_w != h->eta_w || hd.grid_re != h->grid_re)
    return bad(h, "chan_checkpoint_load: written by a handle of another box, grid, time step or precision");
  if (hd.keep_rhs != (h->Rom != nullptr))
    return bad(h, "chan_checkpoint_load: written by a handle that keeps its Helmholtz right-hand sides differently "
                  "(lean_tables)");
  const char* in = static_cast<const char*>(buf);
  size_t off = sizeof(hd);
  try {
    void* p[16];
    size_t b[16];
    const int na = ckpt_arrays(h, p, b);
    for (int k = 0; k < na; ++k) {
      CK(cudaMemcpyAsync(p[k], in + off, b[k], cudaMemcpyHostToDevice, h->stream));
      off += b[k];
    }
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  h->nsub = hd.nsub;
  h->t = hd.t;
  h->have_state = true;
  h->have_filter = false;
  return CHAN_OK;
}

int chan_step(chan_t h, int nsub) {
  if (!h) return bad(nullptr, "chan_step: NULL handle");
  if (nsub < 0) return bad(h, "chan_step: nsub < 0");
  if (!h->have_state) return bad(h, "chan_step: no state set", CHAN_ESTATE);
  try {
    int k = 0;
    const bool graph = h->use_graph && !h->prof;
    // substeps up to the next RK3 step boundary, then whole steps from the graph
    while (k < nsub && (!graph || h->nsub % 3 != 0 || nsub - k < 3)) { run_substep(h); ++k; }
    while (graph && nsub - k >= 3) {
      if (!h->gexec) capture_step_graph(h);
      CK(cudaGraphLaunch(h->gexec, h->stream));
      for (int q = 0; q < KID_COUNT; ++q) h->launches[q] += h->graph_launches[q];
      for (int s = 0; s < 3; ++s) h->t += chan_rk3_weight(s) * h->dt;
      h->nsub += 3;
      k += 3;
    }
    while (k < nsub) { run_substep(h); ++k; }
  } catch (Fail f) {
    return f.code;
  }
  h->have_filter = false;
  return CHAN_OK;
}

int chan_nonlinear(chan_t h, double* H) {
  if (!h || !H) return bad(h, "chan_nonlinear: NULL argument");
  if (!h->have_state) return bad(h, "chan_nonlinear: no state set", CHAN_ESTATE);
  try {
    run_pre(h, true);
    run_nonlinear(h);
    if (prec_pairs(h->prec)) CK(launch_from_pairs(h, wf(h, WF_H1), wf(h, WF_H1), 3 * fsize(h)));
    CK(cudaMemcpyAsync(H, wf(h, WF_H1), 3 * fsize(h) * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_rhs_terms(chan_t h, double* N) {
  if (!h || !N) return bad(h, "chan_rhs_terms: NULL argument");
  if (!h->have_state) return bad(h, "chan_rhs_terms: no state set", CHAN_ESTATE);
  try {
    run_pre(h, true);
    run_nonlinear(h);
    { Traced t(h, KID_NONLIN); CK(launch_nonlin(h, wf(h, WF_H1), wf(h, WF_H2), wf(h, WF_H3), wf(h, WF_NCHI), wf(h, WF_NOM))); }
    if (prec_pairs(h->prec)) CK(launch_from_pairs(h, wf(h, WF_NCHI), wf(h, WF_NCHI), 2 * fsize(h)));
    CK(cudaMemcpyAsync(N, wf(h, WF_NCHI), 2 * fsize(h) * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_filter_stresses(chan_t h, int kind, double p1, double p3, double* ubar, double* tau) {
  if (!h) return bad(nullptr, "chan_filter_stresses: NULL handle");
  if (kind != CHAN_FILTER_SHARP && kind != CHAN_FILTER_BOX) return bad(h, "chan_filter_stresses: unknown kind");
  if (!(p1 > 0) || !(p3 > 0)) return bad(h, "chan_filter_stresses: widths must be positive");
  if (!h->have_state) return bad(h, "chan_filter_stresses: no state set", CHAN_ESTATE);
  try {
    filter_pass(h, kind, p1, p3, ubar, tau, nullptr, 0, 0);
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_filtered_enstrophy(chan_t h, int kind, double p1, double p3, double* ens) {
  if (!h) return bad(nullptr, "chan_filtered_enstrophy: NULL handle");
  if (kind != CHAN_FILTER_SHARP && kind != CHAN_FILTER_BOX) return bad(h, "chan_filtered_enstrophy: unknown kind");
  if (!(p1 > 0) || !(p3 > 0)) return bad(h, "chan_filtered_enstrophy: widths must be positive");
  if (!h->have_state) return bad(h, "chan_filtered_enstrophy: no state set", CHAN_ESTATE);
  try {
    set_filter(h, kind, p1, p3);
    run_pre(h);
    void* mx[3] = {mixed(h, 0), mixed(h, 1), mixed(h, 2)};
    for (int y0 = 0; y0 < h->Ny; y0 += h->slab) {
      const int ny = h->Ny - y0 < h->slab ? h->Ny - y0 : h->slab;
      const size_t o = (size_t)y0 * h->M;
      const double2* in[3] = {wf(h, WF_OM1) + o, h->om + o, wf(h, WF_OM3) + o};
      { Traced t(h, KID_ZINV); CK(launch_zinv(h, in, nullptr, mx, 3, ny, 0)); }
      { Traced t(h, KID_XPASS); CK(launch_xpass(h, 2, mx, mx, ny)); }
      double2* fo[1] = {wf(h, 4) + o};
      { Traced t(h, KID_ZFWD); CK(launch_zfwd(h, mx, fo, 1, ny, 0)); }
    }
    { Traced t(h, KID_APPLY_G); CK(launch_apply_G(h, wf(h, 4), wf(h, 5))); }
    if (ens) {
      CK(cudaMemcpyAsync(ens, wf(h, 5), fsize(h) * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

// Retained-mode counts of the sharp filter: kx < M1, |kz| <= K3 (and below Nz/2).
static void retained(const chan_s* h, double p1, double p3, int* M1, int* M3) {
  const double k1c = M_PI * h->re / p1, k3c = M_PI * h->re / p3;
  int m1 = 0;
  while (m1 < h->nxh && 2.0 * M_PI / h->Lx * m1 < k1c) ++m1;
  int K3 = -1;
  while (K3 + 1 < h->Nz / 2 && 2.0 * M_PI / h->Lz * (K3 + 1) < k3c) ++K3;
  *M1 = m1;
  *M3 = K3 >= 0 ? 2 * K3 + 1 : 0;
}

int chan_database_record(chan_t h, double p1, double p3, double* rec, int* m1, int* m3) {
  if (!h) return bad(nullptr, "chan_database_record: NULL handle");
  if (!(p1 > 0) || !(p3 > 0)) return bad(h, "chan_database_record: cut-off lengths must be positive");
  int M1, M3;
  retained(h, p1, p3, &M1, &M3);
  if (m1) *m1 = M1;
  if (m3) *m3 = M3;
  if (!rec) return CHAN_OK;
  if (!h->have_state) return bad(h, "chan_database_record: no state set", CHAN_ESTATE);
  if (M1 == 0 || M3 == 0) return bad(h, "chan_database_record: the cut-off retains no mode");
  try {
    const size_t blk = (size_t)h->Ny * M3 * M1;
    if (h->dbrec_n < 10 * blk) {
      if (h->dbrec) {
        cudaFreeAsync(h->dbrec, h->stream);
        for (auto& p : h->allocs)
          if (p == h->dbrec) p = nullptr;
        h->dev_bytes -= h->dbrec_n * sizeof(double2);
        h->dbrec = nullptr;
      }
      h->dbrec = dalloc<double2>(h, 10 * blk);
      h->dbrec_n = 10 * blk;
    }
    // filt(omega_i omega_i) first (its pass reuses work slots the stress pass needs)
    int rc = chan_filtered_enstrophy(h, CHAN_FILTER_SHARP, p1, p3, nullptr);
    if (rc != CHAN_OK) return rc;
    { Traced t(h, KID_GATHER); CK(launch_gather_retained(h, wf(h, 5), h->dbrec + 9 * blk, M1, M3, h->Ny)); }
    // ubar_i (gathered slab by slab inside the pass), then filt(u_i u_j) = G P(u_i u_j) =
    // P(u_i u_j) on the retained modes (G = 1 there)
    filter_pass(h, CHAN_FILTER_SHARP, p1, p3, nullptr, nullptr, h->dbrec, M1, M3);
    for (int p = 0; p < 6; ++p) {
      Traced t(h, KID_GATHER);
      CK(launch_gather_retained(h, wf(h, 2 + p), h->dbrec + (3 + p) * blk, M1, M3, h->Ny));
    }
    CK(cudaMemcpyAsync(rec, h->dbrec, 10 * blk * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_filtered_pressure(chan_t h, int kind, double p1, double p3, double* pr) {
  if (!h) return bad(nullptr, "chan_filtered_pressure: NULL handle");
  if (!pr) return bad(h, "chan_filtered_pressure: NULL output");
  int rc = chan_filter_stresses(h, kind, p1, p3, nullptr, nullptr);   // G P(u_i u_j) in work slots 2..7
  if (rc != CHAN_OK) return rc;
  try {
    if (!h->prs) {
      if (h->lean == 2) {   // the substep's Poisson factors live in the slots that now hold P
        h->pois_prs = dalloc<double>(h, (size_t)h->Ny * 7 * h->C);
        CK(launch_setup_pois(h, h->pois_prs));
      }
      h->prs = dalloc<double>(h, (size_t)h->Ny * 2 * h->C);
      h->prsinv = dalloc<double>(h, 4 * (size_t)h->C);
      CK(launch_setup_pressure(h));
    }
    const double2* P[6] = {wf(h, 2), wf(h, 3), wf(h, 4), wf(h, 5), wf(h, 6), wf(h, 7)};   // 11 22 33 12 13 23
    { Traced t(h, KID_PRESSURE); CK(launch_pressure(h, P, wf(h, 8))); }
    CK(cudaMemcpyAsync(pr, wf(h, 8), fsize(h) * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_spectra(chan_t h, double* E) {
  if (!h || !E) return bad(h, "chan_spectra: NULL argument");
  if (!h->have_state) return bad(h, "chan_spectra: no state set", CHAN_ESTATE);
  try {
    run_pre(h);
    double* dst = reinterpret_cast<double*>(wf(h, WF_H1));   // 3 real fields fit in 2 complex slots
    { Traced t(h, KID_SPECTRA); CK(launch_spectra(h, wf(h, WF_U1), wf(h, WF_U3), dst)); }
    CK(cudaMemcpyAsync(E, dst, 3 * fsize(h) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_stats(chan_t h, double* out, double* utau, double* ubulk, double* f) {
  if (!h) return bad(nullptr, "chan_stats: NULL handle");
  if (!h->have_state) return bad(h, "chan_stats: no state set", CHAN_ESTATE);
  try {
    run_pre(h);
    {
      Traced t(h, KID_STATS);
      CK(launch_stats(h, wf(h, WF_U1), wf(h, WF_U3), h->have_filter ? 0 : 1));
    }
    std::vector<double> st(CHAN_NSTAT * (size_t)h->Ny + 2);
    double sc[2];
    CK(cudaMemcpyAsync(st.data(), h->stat, st.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(sc, h->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (out) std::memcpy(out, st.data(), CHAN_NSTAT * (size_t)h->Ny * sizeof(double));
    if (utau) *utau = st[CHAN_NSTAT * (size_t)h->Ny];
    if (ubulk) *ubulk = st[CHAN_NSTAT * (size_t)h->Ny + 1];
    if (f) *f = sc[0];
    for (size_t k = 0; k < st.size(); ++k)
      if (!std::isfinite(st[k])) return bad(h, "chan_stats: non-finite statistics", CHAN_ENAN);
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_sync(chan_t h) {
  if (!h) return bad(nullptr, "chan_sync: NULL handle");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bad(h, std::string("chan_sync: ") + cudaGetErrorString(e), CHAN_ECUDA);
  return CHAN_OK;
}

int chan_profile(chan_t h, int enable) {
  if (!h) return bad(nullptr, "chan_profile: NULL handle");
  if (enable) {
    for (int k = 0; k < KID_COUNT; ++k) h->launches[k] = 0;
    h->nrec = 0;
  }
  h->prof = enable != 0;
  return CHAN_OK;
}

int chan_profile_read(chan_t h, double* ms, long long* launches) {
  if (!h) return bad(nullptr, "chan_profile_read: NULL handle");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bad(h, std::string("chan_profile_read: ") + cudaGetErrorString(e), CHAN_ECUDA);
  if (ms) {
    for (int k = 0; k < KID_COUNT; ++k) ms[k] = 0.0;
    for (size_t i = 0; i < h->nrec; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, h->recs[i].a, h->recs[i].b) == cudaSuccess) ms[h->recs[i].k] += t;
    }
  }
  if (launches)
    for (int k = 0; k < KID_COUNT; ++k) launches[k] = h->launches[k];
  return CHAN_OK;
}

// Launch shapes found by chan_autotune, per (Nx, Ny, Nz, precision), shared by the process.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, std::tuple<int, int, int>> g_tune;

int chan_autotune(chan_t h) {
  if (!h) return bad(nullptr, "chan_autotune: NULL handle");
  if (!h->have_state) return bad(h, "chan_autotune: no state set", CHAN_ESTATE);
  const auto key = std::make_tuple(h->Nx, h->Ny, h->Nz, h->prec);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      std::tie(h->kb_z, h->xthreads, h->ytab) = it->second;
      return CHAN_OK;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const size_t es = prec_t32(h->prec) ? sizeof(float2) : sizeof(double2);
    run_pre(h);
    const double2* in[6] = {wf(h, WF_U1), h->v, wf(h, WF_U3), wf(h, WF_OM1), h->om, wf(h, WF_OM3)};
    void* mx[6] = {mixed(h, 0), mixed(h, 1), mixed(h, 2), mixed(h, 3), mixed(h, 4), mixed(h, 5)};
    const int ny = h->slab;   // timed on the first slab
    auto timed = [&](auto fn) {
      float best = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0, h->stream));
        fn();
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        best = ms < best ? ms : best;
      }
      return best;
    };
    int best_kb = pick_kb(h->nxh, h->L3, es), best_nt = 256;
    float best_t = 1e30f;
    for (int kb = 1; kb <= 16 && kb <= h->nxh; kb *= 2) {
      if ((size_t)kb * fft_ld(h->L3, es) * es > 110 * 1024) break;
      h->kb_z = kb;
      float t = timed([&] { CK(launch_zinv(h, in, nullptr, mx, 6, ny, 0)); });
      if (t < best_t) { best_t = t; best_kb = kb; }
    }
    h->kb_z = best_kb;
    // x-pass alone (fresh inputs from an untimed z-pass before each run); the default
    // 256 threads stay unless another shape is more than 2 % faster
    // (192, 288 and 384 divide the butterfly counts of the 576-point stages: no ragged
    // last round of a stage loop)
    constexpr int NNT = 9;
    float t_nt[NNT];
    for (float& t : t_nt) t = 1e30f;
    // (96, 144 and 160 suit the FP32 two-pass transforms: 6 x 24 register transforms per pass)
    const int nts[NNT] = {256, 128, 192, 288, 384, 512, 96, 160, 144};
    const int ntmax = fft_plan_category(h->p1) == 3 ? 256 : 512;   // the largest register transforms
    for (int rep = 0; rep < 5; ++rep)
      for (int k = 0; k < NNT; ++k) {
        if (nts[k] > ntmax) continue;
        h->xthreads = nts[k];
        CK(launch_zinv(h, in, nullptr, mx, 6, ny, 0));
        CK(cudaEventRecord(e0, h->stream));
        CK(launch_xpass(h, 0, mx, mx, ny));
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        t_nt[k] = ms < t_nt[k] ? ms : t_nt[k];
      }
    int bk = 0;   // 256 threads
    for (int k = 1; k < NNT; ++k)
      if (t_nt[k] < 0.98f * t_nt[0] && t_nt[k] < t_nt[bk]) bk = k;
    best_nt = nts[bk];
    h->xthreads = best_nt;
    // wall-normal sweeps: y tables staged in shared memory or read in place (work slots only)
    best_t = 1e30f;
    int best_yt = 0;
    for (int yt : {0, 1}) {
      h->ytab = yt;
      float t = timed([&] {
        CK(launch_pre(h, wf(h, WF_U1), wf(h, WF_U3), wf(h, WF_OM1), wf(h, WF_OM3)));
        CK(launch_nonlin(h, wf(h, WF_H1), wf(h, WF_H2), wf(h, WF_H3), wf(h, WF_NCHI), wf(h, WF_NOM)));
      });
      if (t < best_t) { best_t = t; best_yt = yt; }
    }
    h->ytab = best_yt;
    CK(cudaStreamSynchronize(h->stream));
  } catch (Fail f) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->kb_z = 0;
    h->xthreads = 0;
    h->ytab = -1;
    return f.code;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = std::make_tuple(h->kb_z, h->xthreads, h->ytab);
  return CHAN_OK;
}

int chan_tuned_shape(chan_t h, int* kb_z, int* xthreads, int* ytab_global) {
  if (!h) return bad(nullptr, "chan_tuned_shape: NULL handle");
  const size_t es = prec_t32(h->prec) ? sizeof(float2) : sizeof(double2);
  if (kb_z) *kb_z = h->kb_z > 0 ? h->kb_z : pick_kb(h->nxh, h->L3, es);
  if (xthreads) *xthreads = h->xthreads > 0 ? h->xthreads : 256;
  if (ytab_global)
    *ytab_global = ytab_in_place(h->ytab, h->Ny) ? 1 : 0;
  return CHAN_OK;
}

int chan_optimize_mesh(const chan_opts* o, int iters, double C, double* y, double* err_before, double* err_after) {
  if (!o || !y) return bad(nullptr, "chan_optimize_mesh: NULL argument");
  if (o->Ny < 9 || o->Ny % 2 == 0 || !(o->re_tau > 0) || !(o->dt > 0) || o->Nx < 2 || o->Nz < 4 || iters < 0)
    return bad(nullptr, "chan_optimize_mesh: invalid sizes");
  std::vector<double> y0(o->Ny);
  const double gre = o->grid_re > 0 ? o->grid_re : o->re_tau;
  if (chanh_ygrid(o->Ny, gre, o->eta_w > 0 ? o->eta_w : 1.0, y0.data())) return bad(nullptr, "chan_optimize_mesh: mesh");
  // most critical wavenumber: largest k^2 of the box and the smallest RK3 beta (1/6)
  const double k1 = 2.0 * M_PI / o->Lx * (o->Nx / 2 - 1), k3 = 2.0 * M_PI / o->Lz * (o->Nz / 2 - 1);
  const double kstar = k1 * k1 + k3 * k3 + 1.0 / ((1.0 / 6.0) * (1.0 / o->re_tau) * o->dt);
  if (chanh_optimize_mesh(o->Ny, y0.data(), kstar, 21, C, iters, y, err_before, err_after))
    return bad(nullptr, "chan_optimize_mesh: coefficient system singular");
  return CHAN_OK;
}

int chan_set_graph(chan_t h, int enable) {
  if (!h) return bad(nullptr, "chan_set_graph: NULL handle");
  h->use_graph = enable != 0;
  return CHAN_OK;
}

size_t chan_footprint_bytes(int Nx, int Ny, int Nz, int precision) {
  if (Nx < 2 || Nx % 2 || Nz < 4 || Nz % 4 || Ny < 9 || Ny % 2 == 0) return 0;
  return footprint(Nx, Ny, Nz, precision);
}

const char* chan_kernel_name(int k) { return (k >= 0 && k < KID_COUNT) ? kKernelNames[k] : nullptr; }

int chan_batch_create(chan_batch_t* out, chan_t* runs, int n, void* stream) {
  return chan_batch_create_ex(out, runs, n, stream, 0);
}

int chan_batch_create_ex(chan_batch_t* out, chan_t* runs, int n, void* stream, int flags) {
  if (!out) return bad(nullptr, "chan_batch_create: out is NULL");
  if (flags & ~CHAN_BATCH_PERSISTENT) return bad(nullptr, "chan_batch_create: unknown flags");
  if ((flags & CHAN_BATCH_PERSISTENT) && n > CHAN_MAXBATCH)
    return bad(nullptr, "chan_batch_create: a persistent batch holds at most 16 runs");
  *out = nullptr;
  if (!runs || n < 1) return bad(nullptr, "chan_batch_create: no runs");
  for (int r = 0; r < n; ++r) {
    if (!runs[r]) return bad(nullptr, "chan_batch_create: NULL run");
    if (!runs[r]->have_state) return bad(nullptr, "chan_batch_create: a run has no state", CHAN_ESTATE);
    if (runs[r]->prec != runs[0]->prec || runs[r]->device != runs[0]->device)
      return bad(nullptr, "chan_batch_create: runs differ in precision or device");
    for (int q = 0; q < r; ++q)
      if (runs[q] == runs[r]) return bad(nullptr, "chan_batch_create: a run appears twice");
    if (runs[r]->slab != runs[r]->Ny || runs[r]->lean)
      return bad(nullptr, "chan_batch_create: a run's transforms are split into slabs or its tables are per "
                          "substep (too large to pack)");
  }
  chan_batch_s* b = new (std::nothrow) chan_batch_s();
  if (!b) return bad(nullptr, "chan_batch_create: out of host memory", CHAN_ENOMEM);
  b->runs.assign(runs, runs + n);
  b->gexec = nullptr;
  b->plan = nullptr;
  if (stream) { b->stream = (cudaStream_t)stream; b->own_stream = false; }
  else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return bad(nullptr, "chan_batch_create: cudaStreamCreate failed", CHAN_ECUDA);
  } else {
    b->own_stream = true;
  }
  b->ev.resize(n + 1, nullptr);
  for (int r = 0; r <= n; ++r)
    if (cudaEventCreateWithFlags(&b->ev[r], cudaEventDisableTiming) != cudaSuccess) {
      chan_batch_free(b);
      return bad(nullptr, "chan_batch_create: cudaEventCreate failed", CHAN_ECUDA);
    }
  if (flags & CHAN_BATCH_PERSISTENT) {
    std::vector<BatchWork> w(n);
    for (int r = 0; r < n; ++r) w[r] = batch_work(runs[r]);
    const cudaError_t e = persist_create(runs, n, w.data(), b->stream, &b->plan);
    if (e != cudaSuccess) {
      cudaGetLastError();
      chan_batch_free(b);
      return bad(nullptr, std::string("chan_batch_create: persistent plan: ") + cudaGetErrorString(e), CHAN_ECUDA);
    }
  }
  *out = b;
  return CHAN_OK;
}

namespace {
// nsub[r] substeps of each run r in persistent launches of up to persist_max_substeps() each.
void persist_steps(chan_batch_s* b, const int* nsub) {
  const int n = (int)b->runs.size(), kmax = persist_max_substeps();
  std::vector<int> left(nsub, nsub + n), now(n);
  for (;;) {
    bool any = false;
    for (int r = 0; r < n; ++r) {
      now[r] = left[r] < kmax ? left[r] : kmax;
      any = any || now[r] > 0;
    }
    if (!any) break;
    BK(persist_launch(b->plan, b->runs.data(), now.data(), b->stream));
    for (int r = 0; r < n; ++r) {
      chan_s* h = b->runs[r];
      for (int q = 0; q < now[r]; ++q) {
        h->t += chan_rk3_weight((int)(h->nsub % 3)) * h->dt;
        h->nsub += 1;
        h->have_filter = false;
      }
      left[r] -= now[r];
    }
  }
}
}  // namespace

int chan_batch_step(chan_batch_t b, int nsub) {
  if (!b) return bad(nullptr, "chan_batch_step: NULL batch");
  if (nsub < 0) { b->err = "chan_batch_step: nsub < 0"; return CHAN_EINVAL; }
  const int n = (int)b->runs.size();
  try {
    for (int r = 0; r < n; ++r) {   // join: the batch stream waits for each run's stream
      BK(cudaEventRecord(b->ev[r], b->runs[r]->stream));
      BK(cudaStreamWaitEvent(b->stream, b->ev[r], 0));
    }
    if (b->plan) {
      std::vector<int> each(n, nsub);
      persist_steps(b, each.data());
      BK(cudaEventRecord(b->ev[n], b->stream));   // fork: each run's stream waits for the batch
      for (int r = 0; r < n; ++r) BK(cudaStreamWaitEvent(b->runs[r]->stream, b->ev[n], 0));
      return CHAN_OK;
    }
    int k = 0;
    auto aligned = [&]() {
      for (chan_s* h : b->runs)
        if (h->nsub % 3 != 0) return false;
      return true;
    };
    while (k < nsub && (!aligned() || nsub - k < 3)) { batch_substep(b); ++k; }
    while (nsub - k >= 3) {
      if (!b->gexec) {   // capture one packed RK3 step; counters restored afterwards
        std::vector<long long> ns(n);
        std::vector<double> ts(n);
        for (int r = 0; r < n; ++r) { ns[r] = b->runs[r]->nsub; ts[r] = b->runs[r]->t; }
        cudaGraph_t g = nullptr;
        BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
        try {
          for (int q = 0; q < 3; ++q) batch_substep(b);
        } catch (Fail) {
          cudaStreamEndCapture(b->stream, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        BK(cudaStreamEndCapture(b->stream, &g));
        cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        BK(e);
        for (int r = 0; r < n; ++r) { b->runs[r]->nsub = ns[r]; b->runs[r]->t = ts[r]; }
      }
      BK(cudaGraphLaunch(b->gexec, b->stream));
      for (chan_s* h : b->runs) {
        for (int q = 0; q < 3; ++q) h->t += chan_rk3_weight(q) * h->dt;
        h->nsub += 3;
        h->have_filter = false;
      }
      k += 3;
    }
    while (k < nsub) { batch_substep(b); ++k; }
    BK(cudaEventRecord(b->ev[n], b->stream));   // fork: each run's stream waits for the batch
    for (int r = 0; r < n; ++r) BK(cudaStreamWaitEvent(b->runs[r]->stream, b->ev[n], 0));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_batch_step_each(chan_batch_t b, const int* nsub) {
  if (!b) return bad(nullptr, "chan_batch_step_each: NULL batch");
  if (!b->plan) { b->err = "chan_batch_step_each: not a persistent batch"; return CHAN_EINVAL; }
  const int n = (int)b->runs.size();
  if (!nsub) { b->err = "chan_batch_step_each: NULL counts"; return CHAN_EINVAL; }
  for (int r = 0; r < n; ++r)
    if (nsub[r] < 0) { b->err = "chan_batch_step_each: a count < 0"; return CHAN_EINVAL; }
  try {
    for (int r = 0; r < n; ++r) {   // join: the batch stream waits for each run's stream
      BK(cudaEventRecord(b->ev[r], b->runs[r]->stream));
      BK(cudaStreamWaitEvent(b->stream, b->ev[r], 0));
    }
    persist_steps(b, nsub);
    BK(cudaEventRecord(b->ev[n], b->stream));   // fork: each run's stream waits for the batch
    for (int r = 0; r < n; ++r) BK(cudaStreamWaitEvent(b->runs[r]->stream, b->ev[n], 0));
  } catch (Fail f) {
    return f.code;
  }
  return CHAN_OK;
}

int chan_batch_status(chan_batch_t b) {
  if (!b) return bad(nullptr, "chan_batch_status: NULL batch");
  if (!b->plan) {
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { b->err = std::string("chan_batch_status: ") + cudaGetErrorString(e); return CHAN_ECUDA; }
    return CHAN_OK;
  }
  int timed_out = 0;
  const cudaError_t e = persist_status(b->plan, b->stream, &timed_out);
  if (e != cudaSuccess) { b->err = std::string("chan_batch_status: ") + cudaGetErrorString(e); return CHAN_ECUDA; }
  if (timed_out) {
    b->err = "chan_batch_status: a wait of a persistent launch ran out; the runs' states are void";
    return CHAN_ETIMEOUT;
  }
  return CHAN_OK;
}

int chan_batch_set_wait(chan_batch_t b, long long polls, int hold_run, int hold_stage) {
  if (!b) return bad(nullptr, "chan_batch_set_wait: NULL batch");
  if (!b->plan) { b->err = "chan_batch_set_wait: not a persistent batch"; return CHAN_EINVAL; }
  if (polls < 1 || hold_run >= (int)b->runs.size() || hold_stage >= 8 * persist_max_substeps()) {
    b->err = "chan_batch_set_wait: polls < 1, or no such run or stage";
    return CHAN_EINVAL;
  }
  persist_set_wait(b->plan, polls, hold_run, hold_stage);
  return CHAN_OK;
}

int chan_batch_persistent_grid(chan_batch_t b) { return b && b->plan ? persist_grid(b->plan) : 0; }

const char* chan_batch_last_error(chan_batch_t b) { return b ? b->err.c_str() : g_init_err.c_str(); }

void chan_batch_free(chan_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->plan) {
    persist_free(b->plan, b->stream);
    cudaStreamSynchronize(b->stream);
  }
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

double chan_time(chan_t h) { return h ? h->t : 0.0; }
long long chan_substeps(chan_t h) { return h ? h->nsub : 0; }

}  // extern "C"
