// Filter epilogue and plane statistics of the channel substep.
//   tau_ij = G P(u_i u_j) - P(ubar_i ubar_j), ubar_i = G u_i   (Sec. 3.1, arXiv:1808.06461)
//   <u_i u_j>(y) by Parseval over the stored modes, U_i, u_tau   (Sec. 3.3)
#include <cstring>

#include "chan_internal.cuh"

namespace {

struct FiltArgs {
  const double2* u[3];
  double2* puu[6];        // in: P(u'_i u'_j); out: P(u_i u_j)
  const double2* pbb[6];  // P(ubar'_i ubar'_j)
  double2* ubar[3];
  double2* tau[6];
  const double* G;
  const double *U1, *U3;  // mean profiles, indexed by plane
  size_t n;        // planes * M
  int M;
  int y0;          // first plane
  int pair;        // u_i stored as FP32 pairs (double-float mode)
};

// The products of the filter pass are formed from the fluctuations u'_i = u_i - U_i(y) (the
// transforms take the (0,0) mode as zero).  The filter acts in x and z only and G(0) = 1, so
// filt(U_i u'_j) = U_i ubar'_j and, u'_j being band-limited, P(U_i u'_j) = U_i u'_j; hence
//   tau_ij = G P(u'_i u'_j) - P(ubar'_i ubar'_j)   (the same tau_ij, without the large mean
//   parts that cancel in G P(u_i u_j) - P(ubar_i ubar_j)), and
//   P(u_i u_j) = P(u'_i u'_j) + U_i u'_j + U_j u'_i, plus U_i U_j in the (0,0) mode.
__global__ void k_filter_out(FiltArgs A) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.n) return;
  const int m = (int)(e % A.M);
  const int y = A.y0 + (int)(e / A.M);
  const double g = A.G[m];
  double2 x[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    x[f] = load_c(A.u[f], e, A.pair);
    A.ubar[f][e] = make_double2(g * x[f].x, g * x[f].y);
  }
  const double U[3] = {A.U1[y], 0.0, A.U3[y]};
  const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    double2 a = A.puu[p][e];
    const double2 b = A.pbb[p][e];
    A.tau[p][e] = make_double2(fma(g, a.x, -b.x), fma(g, a.y, -b.y));
    const int i = pi[p], j = pj[p];
    if (m == 0) {
      a.x += U[i] * U[j];
    } else {
      a.x += fma(U[i], x[j].x, U[j] * x[i].x);
      a.y += fma(U[i], x[j].y, U[j] * x[i].y);
    }
    A.puu[p][e] = a;
  }
}

__global__ void k_apply_G(const double2* __restrict__ in, const double* __restrict__ G, double2* out, size_t n,
                          int M) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double g = G[e % M];
  const double2 x = in[e];
  out[e] = make_double2(g * x.x, g * x.y);
}

// Retained modes of the sharp filter in a compact [Ny][M3][M1] block: kx < M1,
// kz = 0..K3 then -K3..-1 (M3 = 2 K3 + 1).
__global__ void k_gather_retained(const double2* __restrict__ src, double2* dst, int Ny, int Nz, int nxh, int M1,
                                  int M3) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)Ny * M3 * M1;
  if (e >= n) return;
  const int j1 = (int)(e % M1);
  const size_t t = e / M1;
  const int j3 = (int)(t % M3);
  const int y = (int)(t / M3);
  const int K3 = (M3 - 1) / 2;
  const int jz = j3 <= K3 ? j3 : Nz - (M3 - j3);
  dst[e] = src[((size_t)y * Nz + jz) * nxh + j1];
}

// E_i(k1, y, k3) = w |u_i|^2 (w = 2 for kx > 0 counts the conjugate), mean mode excluded.
__global__ void k_spectra(const double2* __restrict__ u1, const double2* __restrict__ v,
                          const double2* __restrict__ u3, double* E, size_t n, int M, int nxh, int pair) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int m = (int)(e % M);
  const double w = m == 0 ? 0.0 : ((m % nxh) == 0 ? 1.0 : 2.0);
  const double2 a = load_c(u1, e, pair), b = load_c(v, e, pair), c = load_c(u3, e, pair);
  E[e] = w * (a.x * a.x + a.y * a.y);
  E[n + e] = w * (b.x * b.x + b.y * b.y);
  E[2 * n + e] = w * (c.x * c.x + c.y * c.y);
}

struct StatArgs {
  const double2* u[3];   // full fields, rows y0 + j (what & 1)
  const double2* ub[3];  // filtered velocities of the slab, plane j (what & 2)
  const double2* tau[6]; // filtered stresses of the slab, plane j (what & 2)
  const double *U1, *U3, *d0, *dN, *wq;
  double* out;          // [CHAN_NSTAT][Ny] + utau, ubulk
  double nu;
  int Ny, M, nxh;
  int y0, nplanes;      // planes y0 .. y0 + nplanes - 1
  int what;             // 1: U_i, <u_i u_j>, u_tau, U_b (rows 0-7); 2: <ubar_i ubar_j>, <tau_ij> (rows 8-19)
  int zero_filtered;    // with what 1: rows 8-19 set to zero (no filter output since the last step)
  int pair;             // u_i stored as FP32 pairs (double-float mode)
};

// Block j < nplanes reduces plane y0 + j in a fixed order (thread-strided partial sums,
// then a fixed shared-memory tree), so results do not depend on scheduling.
__global__ void __launch_bounds__(256) k_stats(StatArgs A) {
  __shared__ double red[6][256];
  const int j = blockIdx.x;
  const int Ny = A.Ny;
  if (j == A.nplanes) {
    if ((A.what & 1) && threadIdx.x == 0) {
      double a = 0.0, b = 0.0, q = 0.0;
      for (int i = 0; i < Ny; ++i) { a += A.d0[i] * A.U1[i]; b += A.dN[i] * A.U1[i]; q += A.wq[i] * A.U1[i]; }
      A.out[CHAN_NSTAT * Ny] = sqrt(A.nu * 0.5 * (fabs(a) + fabs(b)));
      A.out[CHAN_NSTAT * Ny + 1] = 0.5 * q;
    }
    return;
  }
  const int y = A.y0 + j;
  const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
  double acc[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) acc[p] = 0.0;
  const bool filt = A.what == 2;
  const size_t base = (size_t)(filt ? j : y) * A.M;
  for (int m = threadIdx.x; m < A.M; m += blockDim.x) {
    const double w = (m % A.nxh) == 0 ? 1.0 : 2.0;
    double2 q[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) q[f] = filt ? A.ub[f][base + m] : load_c(A.u[f], base + m, A.pair);
#pragma unroll
    for (int p = 0; p < 6; ++p) acc[p] += w * (q[pi[p]].x * q[pj[p]].x + q[pi[p]].y * q[pj[p]].y);
  }
#pragma unroll
  for (int p = 0; p < 6; ++p) red[p][threadIdx.x] = acc[p];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int p = 0; p < 6; ++p) red[p][threadIdx.x] += red[p][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!filt) {
      A.out[0 * Ny + y] = A.U1[y];
      A.out[1 * Ny + y] = A.U3[y];
      for (int p = 0; p < 6; ++p) A.out[(2 + p) * Ny + y] = red[p][0];
      if (A.zero_filtered)
        for (int p = 0; p < 12; ++p) A.out[(8 + p) * Ny + y] = 0.0;
    } else {
      for (int p = 0; p < 6; ++p) {
        A.out[(8 + p) * Ny + y] = red[p][0];
        A.out[(14 + p) * Ny + y] = A.tau[p][base].x;
      }
    }
  }
}

// Double-float storage: FP64 values to (hi, lo) float pairs in place, and back.
__global__ void k_to_pairs(double2* p, size_t n) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double2 v = p[e];
  const dfr a = df_split(v.x), b = df_split(v.y);
  reinterpret_cast<float4*>(p)[e] = make_float4(a.h, a.l, b.h, b.l);
}
__global__ void k_from_pairs(const double2* src, double2* dst, size_t n) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  dst[e] = load_c(src, e, 1);
}

}  // namespace

cudaError_t launch_to_pairs(chan_s* h, double2* p, size_t n) {
  if (n) k_to_pairs<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_from_pairs(chan_s* h, const double2* src, double2* dst, size_t n) {
  if (n) k_from_pairs<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_filter_out(chan_s* h, const double2* const* u, double2* const* puu, const double2* const* pbb,
                              double2* const* ubar, double2* const* tau, int y0, int ny) {
  FiltArgs A;
  A.U1 = h->U1;
  A.U3 = h->U3;
  A.y0 = y0;
  for (int f = 0; f < 3; ++f) { A.u[f] = u[f]; A.ubar[f] = ubar[f]; }
  for (int p = 0; p < 6; ++p) { A.puu[p] = puu[p]; A.pbb[p] = pbb[p]; A.tau[p] = tau[p]; }
  A.G = h->G;
  A.n = (size_t)ny * h->M;
  A.pair = prec_pairs(h->prec);
  A.M = h->M;
  k_filter_out<<<(unsigned)((A.n + 255) / 256), 256, 0, h->stream>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_apply_G(chan_s* h, const double2* in, double2* out) {
  const size_t n = (size_t)h->Ny * h->M;
  k_apply_G<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(in, h->G, out, n, h->M);
  return cudaGetLastError();
}

cudaError_t launch_gather_retained(chan_s* h, const double2* src, double2* dst, int M1, int M3, int ny) {
  const size_t n = (size_t)ny * M3 * M1;
  k_gather_retained<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(src, dst, ny, h->Nz, h->nxh, M1, M3);
  return cudaGetLastError();
}

cudaError_t launch_spectra(chan_s* h, const double2* u1, const double2* u3, double* E) {
  const size_t n = (size_t)h->Ny * h->M;
  k_spectra<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(u1, h->v, u3, E, n, h->M, h->nxh,
                                                                 prec_pairs(h->prec));
  return cudaGetLastError();
}

cudaError_t launch_stats(chan_s* h, const double2* u1, const double2* u3, int zero_filtered) {
  StatArgs A;
  memset(&A, 0, sizeof(A));
  A.u[0] = u1; A.u[1] = h->v; A.u[2] = u3;
  A.U1 = h->U1; A.U3 = h->U3; A.d0 = h->tab_d0; A.dN = h->tab_dN; A.wq = h->tab_wq;
  A.out = h->stat; A.nu = h->nu;
  A.Ny = h->Ny; A.M = h->M; A.nxh = h->nxh;
  A.y0 = 0; A.nplanes = h->Ny; A.what = 1; A.zero_filtered = zero_filtered;
  A.pair = prec_pairs(h->prec);
  k_stats<<<h->Ny + 1, 256, 0, h->stream>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_stats_filtered(chan_s* h, const double2* const* ubar, const double2* const* tau, int y0, int ny) {
  StatArgs A;
  memset(&A, 0, sizeof(A));
  for (int f = 0; f < 3; ++f) A.ub[f] = ubar[f];
  for (int p = 0; p < 6; ++p) A.tau[p] = tau[p];
  A.out = h->stat; A.nu = h->nu;
  A.Ny = h->Ny; A.M = h->M; A.nxh = h->nxh;
  A.y0 = y0; A.nplanes = ny; A.what = 2;
  k_stats<<<ny, 256, 0, h->stream>>>(A);
  return cudaGetLastError();
}
