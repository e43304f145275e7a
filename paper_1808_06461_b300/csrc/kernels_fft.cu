// Dealiased Fourier passes of the channel substep (Sec. 2.1 of
// arXiv:1808.06461: 3/2-rule zero padding in x and z; Appendix C: the
// non-linear terms H = u x omega are formed in physical space).
//
// One x-z plane at a time never leaves the device: a z-pass transforms the
// columns of a plane (zero-padding kz from Nz to 3Nz/2), an x-pass turns two
// physical z-rows at once into real space (two real rows packed into one
// complex FFT), forms the products there and transforms them back, and a
// final z-pass truncates to the stored modes.  All transforms are in-CTA,
// in-place mixed-radix (3, 4, 2) shared-memory FFTs with natural-order spectra
// and digit-reversed physical samples: Cooley-Tukey stages with FMA twiddle
// steps in FP64 and FP32, decimation in frequency (inverse) and in time
// (forward) for the double-float pairs.
#include <cstring>
#include <type_traits>

#include "chan_internal.cuh"
#include "df.cuh"
#include "fft_bodies.cuh"

namespace {

// The FP32 stage-transform z passes are held to 32 registers (eight CTAs of 256 threads per
// SM): they issue on most of their cycles, and their column loads want every warp the SM holds.
template <typename T, int CAT>
constexpr int kZMinBlocks = std::is_same<T, float>::value && CAT == 0 ? 6 : 1;

template <typename T, int CAT>
__global__ void __launch_bounds__(256, kZMinBlocks<T, CAT>) k_zinv(ZArgs A, const typename V2<T>::t* __restrict__ tw) {
  zinv_body<T, CAT>(A, tw, blockIdx.x, blockIdx.y, blockIdx.z);
}



template <typename T, int CAT>
__global__ void __launch_bounds__(256, kZMinBlocks<T, CAT>) k_zfwd(ZArgs A, const typename V2<T>::t* __restrict__ tw) {
  zfwd_body<T, CAT>(A, tw, blockIdx.x, blockIdx.y, blockIdx.z);
}



// (category-3 register transforms need more registers than 512 threads leave)
template <typename T, int MODE, int CAT>
__global__ void __launch_bounds__(CAT == 3 ? 256 : 512) k_xpass(XArgs A, const typename V2<T>::t* __restrict__ tw) {
  xpass_body<T, MODE, CAT>(A, tw, blockIdx.x, blockIdx.y);
}
// The same for CTAs of at most 128 threads, with registers held to what six CTAs per SM allow
// (the FP32 register transforms otherwise take 86, five CTAs)
template <typename T, int MODE, int CAT>
__global__ void __launch_bounds__(128, 6) k_xpass128(XArgs A, const typename V2<T>::t* __restrict__ tw) {
  xpass_body<T, MODE, CAT>(A, tw, blockIdx.x, blockIdx.y);
}



// Packed launches: one grid over several runs (same precision, any sizes).
struct ZBatch {
  ZArgs a[CHAN_MAXBATCH];
  const void* tw[CHAN_MAXBATCH];
  int gx[CHAN_MAXBATCH], gy[CHAN_MAXBATCH];
  int begin[CHAN_MAXBATCH + 1];
  int n;
};
struct XBatch {
  XArgs a[CHAN_MAXBATCH];
  const void* tw[CHAN_MAXBATCH];
  int gx[CHAN_MAXBATCH];
  int begin[CHAN_MAXBATCH + 1];
  int n;
};
__device__ __forceinline__ int run_of(const int* begin, int n, int b) {
  int r = 0;
  while (r + 1 < n && b >= begin[r + 1]) ++r;
  return r;
}
template <typename T, bool INV, int CAT>
__global__ void __launch_bounds__(256) kb_z(ZBatch B) {
  typedef typename V2<T>::t T2;
  const int r = run_of(B.begin, B.n, blockIdx.x);
  const int l = blockIdx.x - B.begin[r];
  const int bx = l % B.gx[r], t = l / B.gx[r];
  const int by = t % B.gy[r], bz = t / B.gy[r];
  if (INV) zinv_body<T, CAT>(B.a[r], (const T2*)B.tw[r], bx, by, bz);
  else zfwd_body<T, CAT>(B.a[r], (const T2*)B.tw[r], bx, by, bz);
}
template <typename T, int CAT>
__global__ void __launch_bounds__(256) kb_xpass(XBatch B) {
  typedef typename V2<T>::t T2;
  const int r = run_of(B.begin, B.n, blockIdx.x);
  const int l = blockIdx.x - B.begin[r];
  xpass_body<T, 0, CAT>(B.a[r], (const T2*)B.tw[r], l % B.gx[r], l / B.gx[r]);
}

template <typename T> size_t esize() { return sizeof(typename V2<T>::t); }

// Columns per z-pass CTA: as many as fit 56 KB of shared memory (4 CTAs per SM), at most 16.
}  // namespace

// Row stride (elements) of a transform buffer: one slot more than the row, so rows start in
// different banks; FP32 rows (swizzled in 16-slot groups) hold whole groups.
int fft_ld(int L, size_t es) { return (es == sizeof(float2) ? 16 * ((L + 15) / 16) : L) + 1; }

// x-pass rows: with FP32 two-pass transforms, r2 (r1 + 1) elements, the stride congruent to r1
// mod 16 so that a warp's column sweep that runs into the next row keeps to distinct banks.
int fft_ld_x(int L, size_t es) {
  int r1, r2;
  if (es == sizeof(float2) && fft_split(L, &r1, &r2)) {
    int ld = r2 * (r1 + 1);
    while ((ld - r1) % 16) ++ld;
    return ld;
  }
  return fft_ld(L, es);
}

bool fft_split(int L, int* r1, int* r2) {
#define CHAN_FFT2P_HOST(A, B) \
  if (L == (A) * (B)) {       \
    *r1 = A;                  \
    *r2 = B;                  \
    return true;              \
  }
  CHAN_FFT2P_SPLITS(CHAN_FFT2P_HOST)
#undef CHAN_FFT2P_HOST
  *r1 = *r2 = 0;
  return false;
}

int pick_kb(int nxh, int L3, size_t es) {
  int kb = 1;
  while (kb * 2 <= nxh && kb * 2 <= 16 && (size_t)(kb * 2) * fft_ld(L3, es) * es <= 56 * 1024) kb *= 2;
  return kb;
}

// Allow the transform kernels the full 227 KB of shared memory (per process; the handle
// is not needed).
cudaError_t fft_configure(chan_s*) {
  const void* fns[] = {(const void*)k_zinv<double, 0>,
                       (const void*)k_zfwd<double, 0>,
                       (const void*)k_xpass<double, 0, 0>,
                       (const void*)k_xpass<double, 1, 0>,
                       (const void*)k_xpass<double, 2, 0>,
                       (const void*)kb_z<double, true, 0>,
                       (const void*)kb_z<double, false, 0>,
                       (const void*)kb_xpass<double, 0>,
                       (const void*)k_zinv<dfr, 0>,
                       (const void*)k_zfwd<dfr, 0>,
                       (const void*)k_xpass<dfr, 0, 0>,
                       (const void*)k_xpass<dfr, 1, 0>,
                       (const void*)k_xpass<dfr, 2, 0>,
                       (const void*)kb_z<dfr, true, 0>,
                       (const void*)kb_z<dfr, false, 0>,
                       (const void*)kb_xpass<dfr, 0>,
                       (const void*)k_zinv<float, 0>,
                       (const void*)k_zfwd<float, 0>,
                       (const void*)k_xpass<float, 0, 0>,
                       (const void*)k_xpass128<float, 0, 0>,
                       (const void*)k_xpass128<float, 0, 1>,
                       (const void*)k_xpass128<float, 0, 2>,
                       (const void*)k_xpass128<float, 0, 3>,
                       (const void*)k_xpass<float, 1, 0>,
                       (const void*)k_xpass<float, 2, 0>,
                       (const void*)kb_z<float, true, 0>,
                       (const void*)kb_z<float, false, 0>,
                       (const void*)kb_xpass<float, 0>,
                       (const void*)k_zinv<float, 1>,
                       (const void*)k_zfwd<float, 1>,
                       (const void*)k_xpass<float, 0, 1>,
                       (const void*)k_xpass<float, 1, 1>,
                       (const void*)k_xpass<float, 2, 1>,
                       (const void*)kb_z<float, true, 1>,
                       (const void*)kb_z<float, false, 1>,
                       (const void*)kb_xpass<float, 1>,
                       (const void*)k_zinv<float, 2>,
                       (const void*)k_zfwd<float, 2>,
                       (const void*)k_xpass<float, 0, 2>,
                       (const void*)k_xpass<float, 1, 2>,
                       (const void*)k_xpass<float, 2, 2>,
                       (const void*)kb_z<float, true, 2>,
                       (const void*)kb_z<float, false, 2>,
                       (const void*)kb_xpass<float, 2>,
                       (const void*)k_zinv<float, 3>,
                       (const void*)k_zfwd<float, 3>,
                       (const void*)k_xpass<float, 0, 3>,
                       (const void*)k_xpass<float, 1, 3>,
                       (const void*)k_xpass<float, 2, 3>,
                       (const void*)kb_z<float, true, 3>,
                       (const void*)kb_z<float, false, 3>,
                       (const void*)kb_xpass<float, 3>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int fft_plan_category(const FftPlan& pl) { return plan_cat(pl); }

cudaError_t launch_zinv(chan_s* h, const double2* const* in, const int* apply_G, void* const* out, int nf, int ny,
                        int f32_mask, int skip00) {
  const size_t es = fft_esize(h);
  ZArgs A = zargs(h, es);
  A.f32_mask = prec_t32(h->prec) ? f32_mask : 0;
  A.skip00 = skip00;
  for (int f = 0; f < nf; ++f) { A.in[f] = in[f]; A.out[f] = out[f]; A.applyG[f] = apply_G ? apply_G[f] : 0; }
  dim3 grid((h->nxh + A.KB - 1) / A.KB, ny, nf);
  size_t sm = (size_t)A.KB * A.ld * es + tw2p_bytes(h->p3);
  if (h->prec == CHAN_PREC_FP64) k_zinv<double, 0><<<grid, 256, sm, h->stream>>>(A, (const double2*)h->tw3);
  else if (prec_t32(h->prec)) {
    const float2* tw = (const float2*)h->tw3;
    switch (plan_cat(h->p3)) {
      case 0: k_zinv<float, 0><<<grid, 256, sm, h->stream>>>(A, tw); break;
      case 1: k_zinv<float, 1><<<grid, 256, sm, h->stream>>>(A, tw); break;
      case 2: k_zinv<float, 2><<<grid, 256, sm, h->stream>>>(A, tw); break;
      default: k_zinv<float, 3><<<grid, 256, sm, h->stream>>>(A, tw); break;
    }
  } else k_zinv<dfr, 0><<<grid, 256, sm, h->stream>>>(A, (const dfc*)h->tw3);
  return cudaGetLastError();
}

cudaError_t launch_zfwd(chan_s* h, void* const* in, double2* const* out, int nf, int ny, int pair_out) {
  const size_t es = fft_esize(h);
  ZArgs A = zargs(h, es);
  A.pair_out = pair_out && prec_pairs(h->prec);
  for (int f = 0; f < nf; ++f) { A.out[f] = in[f]; A.outd[f] = out[f]; }
  dim3 grid((h->nxh + A.KB - 1) / A.KB, ny, nf);
  size_t sm = (size_t)A.KB * A.ld * es + tw2p_bytes(h->p3);
  if (h->prec == CHAN_PREC_FP64) k_zfwd<double, 0><<<grid, 256, sm, h->stream>>>(A, (const double2*)h->tw3);
  else if (prec_t32(h->prec)) {
    const float2* tw = (const float2*)h->tw3;
    switch (plan_cat(h->p3)) {
      case 0: k_zfwd<float, 0><<<grid, 256, sm, h->stream>>>(A, tw); break;
      case 1: k_zfwd<float, 1><<<grid, 256, sm, h->stream>>>(A, tw); break;
      case 2: k_zfwd<float, 2><<<grid, 256, sm, h->stream>>>(A, tw); break;
      default: k_zfwd<float, 3><<<grid, 256, sm, h->stream>>>(A, tw); break;
    }
  } else k_zfwd<dfr, 0><<<grid, 256, sm, h->stream>>>(A, (const dfc*)h->tw3);
  return cudaGetLastError();
}

cudaError_t launch_xpass(chan_s* h, int mode, void* const* in, void* const* out, int ny) {
  const size_t es = fft_esize(h);
  XArgs A;
  memset(&A, 0, sizeof(A));
  const int nin = mode == 0 ? 6 : 3, nout = mode == 0 ? 3 : (mode == 1 ? 6 : 1);
  for (int f = 0; f < nin; ++f) A.in[f] = in[f];
  for (int f = 0; f < nout; ++f) A.out[f] = out[f];
  A.nxh = h->nxh; A.L1 = h->L1; A.L3 = h->L3; A.ld = fft_ld_x(h->L1, fft_esize(h));
  A.mag_nxh = h->nxh == 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + h->nxh - 1) / h->nxh);
  A.scale = 1.0 / ((double)h->L1 * (double)h->L3);
  A.pl = h->p1;
  dim3 grid(h->L3 / 2, ny);
  size_t sm = 6 * (size_t)A.ld * es + tw2p_bytes(h->p1);
  const int nt = h->xthreads > 0 ? h->xthreads : 256;
  if (h->prec == CHAN_PREC_FP64) {
    const double2* tw = (const double2*)h->tw1;
    if (mode == 0) k_xpass<double, 0, 0><<<grid, nt, sm, h->stream>>>(A, tw);
    else if (mode == 1) k_xpass<double, 1, 0><<<grid, nt, sm, h->stream>>>(A, tw);
    else k_xpass<double, 2, 0><<<grid, nt, sm, h->stream>>>(A, tw);
  } else if (prec_t32(h->prec)) {
    const float2* tw = (const float2*)h->tw1;
    const int c = plan_cat(h->p1);
    const int ntc = c == 3 && nt > 256 ? 256 : nt;   // category-3 instances take at most 256 threads
#define CHAN_XPASS_CAT(C)                                                       \
  if (mode == 0 && ntc <= 128) k_xpass128<float, 0, C><<<grid, ntc, sm, h->stream>>>(A, tw); \
  else if (mode == 0) k_xpass<float, 0, C><<<grid, ntc, sm, h->stream>>>(A, tw); \
  else if (mode == 1) k_xpass<float, 1, C><<<grid, ntc, sm, h->stream>>>(A, tw); \
  else k_xpass<float, 2, C><<<grid, ntc, sm, h->stream>>>(A, tw);
    switch (c) {
      case 0: CHAN_XPASS_CAT(0) break;
      case 1: CHAN_XPASS_CAT(1) break;
      case 2: CHAN_XPASS_CAT(2) break;
      default: CHAN_XPASS_CAT(3) break;
    }
#undef CHAN_XPASS_CAT
  } else {
    const dfc* tw = (const dfc*)h->tw1;
    if (mode == 0) k_xpass<dfr, 0, 0><<<grid, nt, sm, h->stream>>>(A, tw);
    else if (mode == 1) k_xpass<dfr, 1, 0><<<grid, nt, sm, h->stream>>>(A, tw);
    else k_xpass<dfr, 2, 0><<<grid, nt, sm, h->stream>>>(A, tw);
  }
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Packed FFT launchers (see launch_pre_batch)
// ---------------------------------------------------------------------------
cudaError_t launch_zinv_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  ZBatch B;
  memset(&B, 0, sizeof(B));
  B.n = n;
  size_t sm = 0;
  int acc = 0;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    ZArgs A = zargs(h, fft_esize(h));
    const double2* in[6];
    A.f32_mask = substep_inputs(h, w[r].u1, w[r].u3, w[r].om1, w[r].om3, 0, in);
    for (int f = 0; f < 6; ++f) { A.in[f] = in[f]; A.out[f] = w[r].mixed[f]; A.applyG[f] = 0; }
    B.a[r] = A;
    B.tw[r] = h->tw3;
    B.gx[r] = (h->nxh + A.KB - 1) / A.KB;
    B.gy[r] = h->Ny;
    B.begin[r] = acc;
    acc += B.gx[r] * B.gy[r] * 6;
    const size_t smr = (size_t)A.KB * A.ld * fft_esize(h) + tw2p_bytes(h->p3);
    sm = smr > sm ? smr : sm;
  }
  B.begin[n] = acc;
  const int prec = hs[0]->prec;
  int c = 0;   // the largest register-transform category of the runs
  for (int r = 0; r < n; ++r) c = plan_cat(hs[r]->p3) > c ? plan_cat(hs[r]->p3) : c;
  if (prec == CHAN_PREC_FP64) kb_z<double, true, 0><<<acc, 256, sm, st>>>(B);
  else if (prec_t32(prec)) {
    switch (c) {
      case 0: kb_z<float, true, 0><<<acc, 256, sm, st>>>(B); break;
      case 1: kb_z<float, true, 1><<<acc, 256, sm, st>>>(B); break;
      case 2: kb_z<float, true, 2><<<acc, 256, sm, st>>>(B); break;
      default: kb_z<float, true, 3><<<acc, 256, sm, st>>>(B); break;
    }
  } else kb_z<dfr, true, 0><<<acc, 256, sm, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_zfwd_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  ZBatch B;
  memset(&B, 0, sizeof(B));
  B.n = n;
  size_t sm = 0;
  int acc = 0;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    ZArgs A = zargs(h, fft_esize(h));
    double2* outs[3] = {w[r].H1, w[r].H2, w[r].H3};
    for (int f = 0; f < 3; ++f) { A.out[f] = w[r].mixed[f]; A.outd[f] = outs[f]; }
    A.pair_out = prec_pairs(h->prec);   // H of the substep
    B.a[r] = A;
    B.tw[r] = h->tw3;
    B.gx[r] = (h->nxh + A.KB - 1) / A.KB;
    B.gy[r] = h->Ny;
    B.begin[r] = acc;
    acc += B.gx[r] * B.gy[r] * 3;
    const size_t smr = (size_t)A.KB * A.ld * fft_esize(h) + tw2p_bytes(h->p3);
    sm = smr > sm ? smr : sm;
  }
  B.begin[n] = acc;
  const int prec = hs[0]->prec;
  int c = 0;
  for (int r = 0; r < n; ++r) c = plan_cat(hs[r]->p3) > c ? plan_cat(hs[r]->p3) : c;
  if (prec == CHAN_PREC_FP64) kb_z<double, false, 0><<<acc, 256, sm, st>>>(B);
  else if (prec_t32(prec)) {
    switch (c) {
      case 0: kb_z<float, false, 0><<<acc, 256, sm, st>>>(B); break;
      case 1: kb_z<float, false, 1><<<acc, 256, sm, st>>>(B); break;
      case 2: kb_z<float, false, 2><<<acc, 256, sm, st>>>(B); break;
      default: kb_z<float, false, 3><<<acc, 256, sm, st>>>(B); break;
    }
  } else kb_z<dfr, false, 0><<<acc, 256, sm, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_xpass_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  XBatch B;
  memset(&B, 0, sizeof(B));
  B.n = n;
  size_t sm = 0;
  int acc = 0;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    XArgs A;
    memset(&A, 0, sizeof(A));
    for (int f = 0; f < 6; ++f) A.in[f] = w[r].mixed[f];
    for (int f = 0; f < 3; ++f) A.out[f] = w[r].mixed[f];
    A.nxh = h->nxh; A.L1 = h->L1; A.L3 = h->L3; A.ld = fft_ld_x(h->L1, fft_esize(h));
  A.mag_nxh = h->nxh == 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + h->nxh - 1) / h->nxh);
    A.scale = 1.0 / ((double)h->L1 * (double)h->L3);
    A.pl = h->p1;
    B.a[r] = A;
    B.tw[r] = h->tw1;
    B.gx[r] = h->L3 / 2;   // packed launches use 256 threads whatever a run's tuned shape
    B.begin[r] = acc;
    acc += B.gx[r] * h->Ny;
    const size_t smr = 6 * (size_t)A.ld * fft_esize(h) + tw2p_bytes(h->p1);
    sm = smr > sm ? smr : sm;
  }
  B.begin[n] = acc;
  const int prec = hs[0]->prec;
  int c = 0;
  for (int r = 0; r < n; ++r) c = plan_cat(hs[r]->p1) > c ? plan_cat(hs[r]->p1) : c;
  if (prec == CHAN_PREC_FP64) kb_xpass<double, 0><<<acc, 256, sm, st>>>(B);
  else if (prec_t32(prec)) {
    switch (c) {
      case 0: kb_xpass<float, 0><<<acc, 256, sm, st>>>(B); break;
      case 1: kb_xpass<float, 1><<<acc, 256, sm, st>>>(B); break;
      case 2: kb_xpass<float, 2><<<acc, 256, sm, st>>>(B); break;
      default: kb_xpass<float, 3><<<acc, 256, sm, st>>>(B); break;
    }
  } else kb_xpass<dfr, 0><<<acc, 256, sm, st>>>(B);
  return cudaGetLastError();
}
