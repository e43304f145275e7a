// Persistent work-list launch of packed serving: one launch advances each run of a batch
// by its own number of substeps (up to kMaxSub).  Each run's work is a sequence of stages
// (substep k, phase p: the single-run kernels' order), each stage a number of items (the
// blocks of that phase's kernel).  The CTAs of the launch take items from per-(run, stage)
// counters and run the block of the phase's body (the same bodies as the single-run and
// packed kernels), so the phases of different runs overlap on the device instead of one
// phase of all runs per launch, and each run goes on to its next substep as soon as its
// own previous one is done, without a batch-wide boundary.  A CTA only takes an item whose
// run's previous stage is
// complete, scanning the runs round-robin from where its last item was; it never holds
// an item it cannot run, so no CTA waits on another that is not yet resident.  A CTA that
// finds no ready item polls again; after a bounded number of empty polls it raises the
// launch's timeout flag and the sticky error word, every CTA then leaves, and the host
// reads CHAN_ETIMEOUT.  The paper has no counterpart; it serves many independent channel
// runs at once.
//
// Data written earlier in the same launch is read here, so the bodies are compiled
// without read-only (non-coherent) loads of their inputs (CHAN_RO empty).
#include <vector>

#define CHAN_RO
#include "y_bodies.cuh"
#include "fft_bodies.cuh"

namespace {

enum { PH_PRE = 0, PH_ZINV, PH_XPASS, PH_ZFWD, PH_NONLIN, PH_HELM, PH_POIS, PH_MEAN, PH_N };
constexpr int kPThreads = 128;
constexpr int kMaxSub = 48;             // substeps of a run per launch
constexpr int kTfBlocks = 8;            // transform blocks per item
constexpr int kQMax = kMaxSub * PH_N;   // stages of a run per launch

// Arguments of every phase of one run (device memory; constant while the batch lives).
struct PRun {
  PreP pre;
  ZArgs zi, zf;
  XArgs xp;
  const void *tw1, *tw3;
  NonlinP nl;
  HelmP he[3];   // per RK3 substep s
  PoisP po[3];
  MeanP me[3];
  int gxz, gyz, gxx;   // z-pass column chunks and planes, x-pass row pairs per plane
};

// The launch's schedule (kernel parameter).
// Counters of a launch (device, zeroed before it): [0] timeout flag, then per run r the
// stage being handed out, and per (run, stage q) the items taken and the items completed.
constexpr int kCtrFlag = 0;
__host__ __device__ constexpr int ctr_cur(int r) { return 1 + r; }
__host__ __device__ constexpr int ctr_take(int r, int q) { return 1 + CHAN_MAXBATCH + r * kQMax + q; }
__host__ __device__ constexpr int ctr_done(int r, int q) { return 1 + CHAN_MAXBATCH * (1 + kQMax) + r * kQMax + q; }
constexpr int kCtrWords = 1 + CHAN_MAXBATCH * (1 + 2 * kQMax);

struct PSched {
  const PRun* runs;
  unsigned* ctr;          // kCtrWords launch counters
  unsigned* sticky;       // error word that launches do not reset
  int n;                  // runs
  int nq[CHAN_MAXBATCH];  // stages of each run in this launch (8 per substep)
  int nb[CHAN_MAXBATCH][PH_N];           // items of each run's phases
  int gb[CHAN_MAXBATCH][PH_N];           // consecutive blocks of the phase's kernel per item
  int blk[CHAN_MAXBATCH][PH_N];          // blocks of the phase's kernel
  int s0[CHAN_MAXBATCH];                 // RK3 substep of each run's first substep in the launch
  long long spin_limit;                  // empty polls of a CTA before it gives up
  int hold_run, hold_q;                  // (run, stage) made to need one completion more (-1: none)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <class Y, typename T, int CAT, bool F32>
__device__ __forceinline__ void p_item(const PRun& R, int p, int s, int b) {
  typedef typename V2<T>::t T2;
  typedef typename Y::R YR;
  switch (p) {
    case PH_PRE: {
      const PreP& a = R.pre;
      pre_body<Y, F32>(a.g, a.t, a.v, a.om, a.dv, a.U1, a.U3, a.u1o, a.u3o, a.om1o, a.om3o, b);
      break;
    }
    case PH_ZINV: {
      const int bx = b % R.gxz, t = b / R.gxz;
      zinv_body<T, 0>(R.zi, static_cast<const T2*>(R.tw3), bx, t % R.gyz, t / R.gyz);
      break;
    }
    case PH_XPASS:
      xpass_body<T, 0, CAT>(R.xp, static_cast<const T2*>(R.tw1), b % R.gxx, b / R.gxx);
      break;
    case PH_ZFWD: {
      const int bx = b % R.gxz, t = b / R.gxz;
      zfwd_body<T, 0>(R.zf, static_cast<const T2*>(R.tw3), bx, t % R.gyz, t / R.gyz);
      break;
    }
    case PH_NONLIN: {
      const NonlinP& a = R.nl;
      nonlin_body<Y>(a.g, a.t, a.H1, a.H2, a.H3, a.Nchi, a.Nom, a.scr, b);
      break;
    }
    case PH_HELM: {
      const HelmP& a = R.he[s];
      helm_body<Y, 2>(a.g, a.t, static_cast<const YR*>(a.helm), a.om, a.chi, a.Nchi, a.Nom, a.Nchi_p, a.Nom_p,
                      a.Rom, a.Rchi, a.scal, a.scr, a.s, b);
      break;
    }
    case PH_POIS: {
      const PoisP& a = R.po[s];
      poisson_body<Y>(a.g, a.t, static_cast<const YR*>(a.helm), static_cast<const YR*>(a.pois),
                      static_cast<const YR*>(a.infl), a.v, a.chi, a.dv, a.scr, a.scal, a.s, b);
      break;
    }
    default: {
      const MeanP& a = R.me[s];
      mean_body(a.g, a.t, a.helm, a.meanh, a.H1, a.H3, a.U1, a.U3, a.H1p, a.H3p, a.scal, a.s, 0);
      break;
    }
  }
}

template <class Y, typename T, int CAT, bool F32>
__global__ void __launch_bounds__(kPThreads, 4) kp_step(PSched S) {
  __shared__ int sh[3];
  int next = blockIdx.x % S.n;   // run to look at first
  for (;;) {
    __syncthreads();   // the previous item's shared memory is no longer in use
    if (threadIdx.x == 0) {
      int got = -1, q = 0, b = 0;
      long long idle = 0;
      while (got < 0) {
        if (ld_acquire(S.ctr + kCtrFlag) != 0u) break;   // a CTA gave up: leave
        bool left = false;   // some run still has items to hand out
        for (int t = 0; t < S.n && got < 0; ++t) {
          const int r = (next + t) % S.n;
          const int c = (int)ld_acquire(S.ctr + ctr_cur(r));
          if (c >= S.nq[r]) continue;
          left = true;
          if (c > 0) {   // ready once the run's previous stage is complete
            const unsigned need = (unsigned)S.nb[r][(c - 1) % PH_N] + (r == S.hold_run && c - 1 == S.hold_q ? 1u : 0u);
            if (ld_acquire(S.ctr + ctr_done(r, c - 1)) < need) continue;
          }
          const int nbc = S.nb[r][c % PH_N];
          const int g = (int)atomicAdd(S.ctr + ctr_take(r, c), 1u);
          if (g < nbc) {
            got = r; q = c; b = g;
            next = g + 1 < nbc ? r : (r + 1) % S.n;
          } else {
            atomicCAS(S.ctr + ctr_cur(r), (unsigned)c, (unsigned)(c + 1));   // stage fully handed out
            --t;   // look at this run again
          }
        }
        if (got >= 0 || !left) break;
        if (++idle > S.spin_limit) {
          atomicExch(S.ctr + kCtrFlag, 1u);
          atomicOr(S.sticky, 1u);
          break;
        }
        __nanosleep(128);
      }
      sh[0] = got;
      sh[1] = q;
      sh[2] = b;
    }
    __syncthreads();
    const int r = sh[0];
    if (r < 0) break;
    const int q = sh[1], k = q / PH_N, p = q - k * PH_N;
    __threadfence();   // this thread's loads follow the completions thread 0 observed
    const int g = S.gb[r][p], b0 = sh[2] * g, b1 = min(b0 + g, S.blk[r][p]);
    for (int bb = b0; bb < b1; ++bb) {
      if (bb > b0) __syncthreads();   // the previous block's shared memory is no longer in use
      p_item<Y, T, CAT, F32>(S.runs[r], p, (S.s0[r] + k) % 3, bb);
    }
    __syncthreads();   // every thread's writes of the item are done
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(S.ctr + ctr_done(r, q), 1u);
    }
  }
}

template <class Y, typename T, int CAT, bool F32>
const void* kp_fn() { return reinterpret_cast<const void*>(kp_step<Y, T, CAT, F32>); }

// The instance for a batch of precision prec whose x transforms need category cat.
const void* kp_pick(int prec, int cat) {
  if (prec == CHAN_PREC_FP64) return kp_fn<YF64, double, 0, false>();
  if (prec == CHAN_PREC_F64X) return kp_fn<YDF, dfr, 0, false>();
  if (prec == CHAN_PREC_MIXED) {
    switch (cat) {
      case 0: return kp_fn<YF64, float, 0, true>();
      case 1: return kp_fn<YF64, float, 1, true>();
      case 2: return kp_fn<YF64, float, 2, true>();
      default: return kp_fn<YF64, float, 3, true>();
    }
  }
  switch (cat) {
    case 0: return kp_fn<YDF, float, 0, true>();
    case 1: return kp_fn<YDF, float, 1, true>();
    case 2: return kp_fn<YDF, float, 2, true>();
    default: return kp_fn<YDF, float, 3, true>();
  }
}

}  // namespace

struct PersistPlan {
  int n;
  std::vector<PRun> host;   // the uploaded table, kept until the plan dies (the copy is asynchronous)
  PRun* runs;          // device [n]
  unsigned* ctr;       // device [kCtrWords + 1]; the last word is the sticky error
  PSched S;            // schedule without the per-launch fields (nq, s0)
  const void* fn;
  size_t smem;
  int grid;
};

// Builds the stage table and the device argument table of a batch (hs[0..n), n <= CHAN_MAXBATCH,
// one precision, no slabs, no per-substep tables; w[r] = run r's work fields).
cudaError_t persist_create(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st, PersistPlan** out) {
  *out = nullptr;
  if (n < 1 || n > CHAN_MAXBATCH) return cudaErrorInvalidValue;
  PersistPlan* P = new PersistPlan();
  memset(&P->S, 0, sizeof(P->S));
  P->n = n;
  P->host.resize(n);
  std::vector<PRun>& R = P->host;
  const int prec = hs[0]->prec;
  const bool f32 = prec_t32(prec);
  int cat = 0;
  size_t sm = 0;
  auto up = [&](size_t b) { sm = b > sm ? b : sm; };
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    PRun& A = R[r];
    memset(&A, 0, sizeof(A));
    const Geo g = geo(h);
    const YTabs t = ytabs(h);
    A.pre = PreP{g, t, h->v, h->om, h->dv, h->U1, h->U3, w[r].u1, w[r].u3, w[r].om1, w[r].om3};
    A.nl = NonlinP{g, t, w[r].H1, w[r].H2, w[r].H3, w[r].Nchi, w[r].Nom, h->scr};
    for (int s = 0; s < 3; ++s) {
      A.he[s] = HelmP{g, t, helm_slot_y(h, s), h->om, h->chi, w[r].Nchi, w[r].Nom, h->Nchi_p, h->Nom_p,
                      h->Rom, h->Rchi, h->scal, h->scr, s};
      A.po[s] = PoisP{g, t, helm_slot_y(h, s), pois_y(h), infl_slot_y(h, s), h->v, h->chi, h->dv, h->scr, h->scal, s};
      A.me[s] = MeanP{g, t, helm_slot(h, s), h->meanh, w[r].H1, w[r].H3, h->U1, h->U3, h->H1m_p, h->H3m_p,
                      h->scal, s};
    }
    const size_t es = fft_esize(h);
    A.zi = zargs(h, es);
    {
      const double2* in[6];
      A.zi.f32_mask = substep_inputs(h, w[r].u1, w[r].u3, w[r].om1, w[r].om3, 0, in);
      for (int f = 0; f < 6; ++f) { A.zi.in[f] = in[f]; A.zi.out[f] = w[r].mixed[f]; A.zi.applyG[f] = 0; }
    }
    A.zf = zargs(h, es);
    {
      double2* outs[3] = {w[r].H1, w[r].H2, w[r].H3};
      for (int f = 0; f < 3; ++f) { A.zf.out[f] = w[r].mixed[f]; A.zf.outd[f] = outs[f]; }
      A.zf.pair_out = prec_pairs(h->prec);
    }
    for (int f = 0; f < 6; ++f) A.xp.in[f] = w[r].mixed[f];
    for (int f = 0; f < 3; ++f) A.xp.out[f] = w[r].mixed[f];
    A.xp.nxh = h->nxh; A.xp.L1 = h->L1; A.xp.L3 = h->L3; A.xp.ld = fft_ld_x(h->L1, es);
    A.xp.mag_nxh = h->nxh == 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + h->nxh - 1) / h->nxh);
    A.xp.scale = 1.0 / ((double)h->L1 * (double)h->L3);
    A.xp.pl = h->p1;
    A.tw1 = h->tw1;
    A.tw3 = h->tw3;
    A.gxz = (h->nxh + A.zi.KB - 1) / A.zi.KB;
    A.gyz = h->Ny;
    A.gxx = h->L3 / 2;
    const int ymb = (h->M + kPThreads - 1) / kPThreads;
    int* blk = P->S.blk[r];
    blk[PH_PRE] = ymb + 1;   // + the block of the (0,0) mode
    blk[PH_ZINV] = A.gxz * A.gyz * 6;
    blk[PH_XPASS] = A.gxx * h->Ny;
    blk[PH_ZFWD] = A.gxz * A.gyz * 3;
    blk[PH_NONLIN] = ymb;
    blk[PH_HELM] = ymb;
    blk[PH_POIS] = ymb;
    blk[PH_MEAN] = 1;
    // a transform item is kTfBlocks consecutive blocks (a few microseconds each), so taking an
    // item costs little against its work; a wall-normal block is one long sweep already
    for (int p = 0; p < PH_N; ++p) {
      const bool tf = p == PH_ZINV || p == PH_XPASS || p == PH_ZFWD;
      P->S.gb[r][p] = tf ? kTfBlocks : 1;
      P->S.nb[r][p] = (blk[p] + P->S.gb[r][p] - 1) / P->S.gb[r][p];
    }
    const int c = plan_cat(h->p1);
    cat = c > cat ? c : cat;
    up(ysm_n(h, 14, kRingPre, kPThreads));
    up(ysm_n(h, 14, kRingNonlin, kPThreads));
    up(ysm_n(h, 14, kRingHelm, kPThreads));
    up(ysm_n(h, 23, kRingPois, kPThreads));
    up((size_t)A.zi.KB * A.zi.ld * es + tw2p_bytes(h->p3));
    up(6 * (size_t)A.xp.ld * es + tw2p_bytes(h->p1));
    up(sizeof(double) * (9 * (size_t)h->Ny + 256));
  }
  P->S.n = n;
  P->S.spin_limit = 1 << 23;   // about a second of empty 128 ns polls
  P->S.hold_run = P->S.hold_q = -1;
  P->fn = kp_pick(prec, f32 ? cat : 0);
  P->smem = sm;
  cudaError_t e = cudaFuncSetAttribute(P->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0, dev = 0, nsm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P->fn, kPThreads, sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  P->grid = per_sm * nsm;
  P->runs = nullptr;
  P->ctr = nullptr;
  const size_t nctr = (size_t)kCtrWords + 1;
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&P->runs), n * sizeof(PRun), st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&P->ctr), nctr * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->runs, R.data(), n * sizeof(PRun), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->ctr, 0, nctr * sizeof(unsigned), st);
  if (e != cudaSuccess) {
    if (P->runs) cudaFreeAsync(P->runs, st);
    if (P->ctr) cudaFreeAsync(P->ctr, st);
    delete P;
    return e;
  }
  P->S.runs = P->runs;
  P->S.ctr = P->ctr;
  P->S.sticky = P->ctr + nctr - 1;
  *out = P;
  return cudaSuccess;
}

// One launch of nsub[r] (0 .. kMaxSub) substeps of each run r, each from its own RK3 substep
// (hs[r]->nsub).
cudaError_t persist_launch(PersistPlan* P, chan_s* const* hs, const int* nsub, cudaStream_t st) {
  PSched S = P->S;
  int items = 0;
  for (int r = 0; r < P->n; ++r) {
    if (nsub[r] < 0 || nsub[r] > kMaxSub) return cudaErrorInvalidValue;
    S.nq[r] = nsub[r] * PH_N;
    S.s0[r] = (int)(hs[r]->nsub % 3);
    for (int p = 0; p < PH_N; ++p) items += nsub[r] * S.nb[r][p];
  }
  if (items == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(P->ctr, 0, (size_t)kCtrWords * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int grid = P->grid < items ? P->grid : items;
  void* args[] = {&S};
  return cudaLaunchKernel(P->fn, dim3(grid), dim3(kPThreads), args, P->smem, st);
}

int persist_max_substeps() { return kMaxSub; }

// 1 if a wait of a launch gave up since the last call (the stream is synchronised first).
cudaError_t persist_status(PersistPlan* P, cudaStream_t st, int* timed_out) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, P->S.sticky, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && v) e = cudaMemsetAsync(P->S.sticky, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *timed_out = v != 0;
  return e;
}

void persist_set_wait(PersistPlan* P, long long spins, int hold_run, int hold_stage) {
  P->S.spin_limit = spins;
  P->S.hold_run = hold_run;
  P->S.hold_q = hold_stage;
}

int persist_grid(const PersistPlan* P) { return P->grid; }

void persist_free(PersistPlan* P, cudaStream_t st) {
  if (!P) return;
  if (P->runs) cudaFreeAsync(P->runs, st);
  if (P->ctr) cudaFreeAsync(P->ctr, st);
  delete P;
}
