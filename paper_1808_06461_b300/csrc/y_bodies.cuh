// Device bodies of the wall-normal (y) kernels and the host helpers that build their
// arguments.  Included by the single-run and packed kernels (kernels_y.cu) and by the
// persistent work-list kernel (kernels_fft.cu).  CHAN_RO qualifies the pointers a body only
// reads; a translation unit whose kernels read data that the same launch writes defines it
// empty before the include, so that no such load takes the read-only (non-coherent) path.
#pragma once
#include <cstdint>

#include "chan_internal.cuh"
#include "df.cuh"

#ifndef CHAN_RO
#define CHAN_RO __restrict__
#endif

namespace {

// Spalart-Moser-Rogers low-storage RK3: (gamma, zeta, alpha, beta) per substep.
__constant__ double c_rk3[3][4] = {{8.0 / 15.0, 0.0, 29.0 / 96.0, 37.0 / 160.0},
                                   {5.0 / 12.0, -17.0 / 60.0, -3.0 / 40.0, 5.0 / 24.0},
                                   {3.0 / 4.0, -5.0 / 12.0, 1.0 / 6.0, 1.0 / 6.0}};
const double h_rk3[3][4] = {{8.0 / 15.0, 0.0, 29.0 / 96.0, 37.0 / 160.0},
                            {5.0 / 12.0, -17.0 / 60.0, -3.0 / 40.0, 5.0 / 24.0},
                            {3.0 / 4.0, -5.0 / 12.0, 1.0 / 6.0, 1.0 / 6.0}};

__device__ __forceinline__ double2 z2() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 axpy(double a, double2 x, double2 y) {  // y + a x
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ double2 scl(double a, double2 x) { return make_double2(a * x.x, a * x.y); }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <int N>
__device__ __forceinline__ void push(double2 (&w)[N], double2 x) {
#pragma unroll
  for (int d = 0; d < N - 1; ++d) w[d] = w[d + 1];
  w[N - 1] = x;
}

// Banded row times window: sum_d c[d] w[d] (columns i-3..i+3).
__device__ __forceinline__ double2 band7(const double* c, const double2 (&w)[7]) {
  double2 r = z2();
#pragma unroll
  for (int d = 0; d < 7; ++d) r = axpy(c[d], w[d], r);
  return r;
}

// Forward substitution of row i: z_i = r - sum_d l[d] z_{i-3+d}; hist = (z_{i-3}, z_{i-2}, z_{i-1}).
__device__ __forceinline__ double2 fwd(double2 r, double l0, double l1, double l2, double2 (&hist)[3]) {
  r = axpy(-l0, hist[0], r);
  r = axpy(-l1, hist[1], r);
  r = axpy(-l2, hist[2], r);
  push(hist, r);
  return r;
}

// Back substitution of row i: x_i = (z_i - sum_d u[d] x_{i+1+d}) dinv; nxt = (x_{i+1}, x_{i+2}, x_{i+3}).
__device__ __forceinline__ double2 bwd(double2 z, double u0, double u1, double u2, double dinv, double2 (&nxt)[3]) {
  z = axpy(-u0, nxt[0], z);
  z = axpy(-u1, nxt[1], z);
  z = axpy(-u2, nxt[2], z);
  double2 x = scl(dinv, z);
  nxt[2] = nxt[1];
  nxt[1] = nxt[0];
  nxt[0] = x;
  return x;
}

__device__ __forceinline__ void load_tab(double* dst, const double* src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// ---------------------------------------------------------------------------
// Row prefetch ring.  Each sweep reads the rows of its pencil once, in order, and its
// serial recurrence would otherwise wait on every row's loads.  cp.async copies the
// values of the row kRing - 1 rows ahead into this thread's own shared-memory slots while
// the current row is computed.  A slot is written and read by one thread only, so the
// thread's own cp.async.wait_group is all the synchronisation there is (no barrier, no
// spin).  Layout per CTA: [kRing][K16][blockDim] slots of 16 bytes, then
// [kRing][K8][blockDim] slots of 8 bytes; a warp's 32 slots are contiguous.
// ---------------------------------------------------------------------------
constexpr int kRing = 4;   // rows in flight per sweep (a power of two)

__device__ __forceinline__ void cp16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int K16, int K8>
struct Ring {
  unsigned char* b;
  __device__ __forceinline__ explicit Ring(void* base) : b(static_cast<unsigned char*>(base)) {}
  __device__ __forceinline__ unsigned char* f(int st, int k) const {
    return b + ((size_t)(st * K16 + k) * blockDim.x + threadIdx.x) * 16;
  }
  __device__ __forceinline__ unsigned char* t(int st, int k) const {
    return b + (size_t)kRing * K16 * blockDim.x * 16 + ((size_t)(st * K8 + k) * blockDim.x + threadIdx.x) * 8;
  }
  static constexpr size_t per_thread = (size_t)kRing * (K16 * 16 + K8 * 8);
};

// Runs fn(t) for t = 0 .. n-1 with issue(t) called kRing - 1 rows ahead: on return from
// the wait, the copies of row t are in this thread's slots of stage t & (kRing - 1).
template <class Issue, class Body>
__device__ __forceinline__ void pipelined(int n, Issue issue, Body body) {
#pragma unroll 1
  for (int q = 0; q < kRing - 1; ++q) {
    if (q < n) issue(q, q & (kRing - 1));
    cp_commit();
  }
#pragma unroll 1
  for (int t = 0; t < n; ++t) {
    const int tn = t + kRing - 1;
    if (tn < n) issue(tn, tn & (kRing - 1));
    cp_commit();
    cp_wait<kRing - 1>();
    body(t, t & (kRing - 1));
  }
  cp_wait<0>();
}

// Shared-memory ring base after the staged tables (16-byte aligned).
__device__ __forceinline__ void* ring_base(void* p) {
  return reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
}


// Arithmetic and storage of the four substep y-kernels, chosen per precision
// mode: FP64, or double-float (FP32 pairs, about 2^-47) in the double-float mode,
// where every Fourier field holds (hi, lo) float pairs in the 16 bytes of a
// complex double (ld / st move them as one 128-bit access).
struct YF64 {
  typedef double R;
  typedef double2 C;
  __device__ static __forceinline__ R r(double x) { return x; }
  __device__ static __forceinline__ C c(double2 x) { return x; }
  __device__ static __forceinline__ C zero() { return make_double2(0.0, 0.0); }
  __device__ static __forceinline__ C axpy(R a, C x, C y) { return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y)); }
  __device__ static __forceinline__ C scl(R a, C x) { return make_double2(a * x.x, a * x.y); }
  __device__ static __forceinline__ C sub(C a, C b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ static __forceinline__ C itimes(C a) { return make_double2(-a.y, a.x); }
  __device__ static __forceinline__ R neg(R a) { return -a; }
  __device__ static __forceinline__ void st(double2* p, size_t o, C x) { p[o] = x; }
  // a value copied into a shared-memory ring slot
  __device__ static __forceinline__ C lds(const unsigned char* q) { return *reinterpret_cast<const double2*>(q); }
  __device__ static __forceinline__ R ldr(const unsigned char* q) { return *reinterpret_cast<const double*>(q); }
  __device__ static __forceinline__ float2 ldsf(const unsigned char* q) { return f(lds(q)); }
  // rounded to FP32 (a transform input of the mixed modes), on the integer pipe
  __device__ static __forceinline__ float2 f(C x) { return make_float2(d2f_int(x.x), d2f_int(x.y)); }
  __device__ static __forceinline__ const R* A2(const YTabs& t) { return t.A2; }
  __device__ static __forceinline__ const R* B2(const YTabs& t) { return t.B2; }
  __device__ static __forceinline__ const R* B1(const YTabs& t) { return t.B1; }
  __device__ static __forceinline__ const R* LU1(const YTabs& t) { return t.lu1; }
  __device__ static __forceinline__ const R* D0(const YTabs& t) { return t.d0; }
  __device__ static __forceinline__ const R* DN(const YTabs& t) { return t.dN; }
  // sums of products (band rows, substitution steps): plain FMA accumulation
  typedef double2 Acc;
  __device__ static __forceinline__ Acc acc(C x) { return x; }
  __device__ static __forceinline__ void acc_add(Acc& s, R a, C x) { s = axpy(a, x, s); }
  __device__ static __forceinline__ C acc_done(const Acc& s) { return s; }
};
// Double-float sum of products with one normalisation: the high parts are summed exactly
// (Knuth's two-sum) and every low-order part (each product's FMA residual and cross terms,
// each two-sum's error) goes into one float, renormalised once at the end (fast two-sum).
// The value is the one the per-term pair arithmetic gives, to a few units of 2^-48 of the
// largest partial sum, at 12 instead of 15 FP32 operations a term.
struct DfAcc {
  float h, l;
};
__device__ __forceinline__ DfAcc dfacc(dfr x) { return DfAcc{x.h, x.l}; }
__device__ __forceinline__ void dfacc_add(DfAcc& s, dfr a, dfr x) {
  const float p = __fmul_rn(a.h, x.h);
  float e = __fmaf_rn(a.h, x.h, -p);
  e = __fmaf_rn(a.h, x.l, e);
  e = __fmaf_rn(a.l, x.h, e);
  const float t = __fadd_rn(s.h, p);
  const float bb = __fsub_rn(t, s.h);
  const float er = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(er, e));
}
__device__ __forceinline__ dfr dfacc_done(DfAcc s) {
  const float t = __fadd_rn(s.h, s.l);
  return dfr{t, __fsub_rn(s.l, __fsub_rn(t, s.h))};
}
struct YDF {
  typedef dfr R;
  typedef dfc C;
  __device__ static __forceinline__ R r(double x) { return df_split(x); }
  __device__ static __forceinline__ C c(double2 x) { return dfc{df_split(x.x), df_split(x.y)}; }
  __device__ static __forceinline__ C zero() { return dfc{dfr{0.f, 0.f}, dfr{0.f, 0.f}}; }
  __device__ static __forceinline__ C axpy(R a, C x, C y) { return dfc{y.x + mul_u(a, x.x), y.y + mul_u(a, x.y)}; }
  __device__ static __forceinline__ C scl(R a, C x) { return dfc{a * x.x, a * x.y}; }
  __device__ static __forceinline__ C sub(C a, C b) { return dfc{a.x - b.x, a.y - b.y}; }
  __device__ static __forceinline__ C itimes(C a) { return dfc{-a.y, a.x}; }
  __device__ static __forceinline__ R neg(R a) { return -a; }
  __device__ static __forceinline__ void st(double2* p, size_t o, C x) {
    reinterpret_cast<float4*>(p)[o] = make_float4(x.x.h, x.x.l, x.y.h, x.y.l);
  }
  __device__ static __forceinline__ C lds(const unsigned char* p) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    return dfc{dfr{q.x, q.y}, dfr{q.z, q.w}};
  }
  __device__ static __forceinline__ R ldr(const unsigned char* p) { return *reinterpret_cast<const dfr*>(p); }
  __device__ static __forceinline__ float2 ldsf(const unsigned char* p) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    return make_float2(q.x + q.y, q.z + q.w);
  }
  __device__ static __forceinline__ float2 f(C x) { return make_float2(x.x.h + x.x.l, x.y.h + x.y.l); }
  __device__ static __forceinline__ const R* A2(const YTabs& t) { return t.A2p; }
  __device__ static __forceinline__ const R* B2(const YTabs& t) { return t.B2p; }
  __device__ static __forceinline__ const R* B1(const YTabs& t) { return t.B1p; }
  __device__ static __forceinline__ const R* LU1(const YTabs& t) { return t.lu1p; }
  __device__ static __forceinline__ const R* D0(const YTabs& t) { return t.d0p; }
  __device__ static __forceinline__ const R* DN(const YTabs& t) { return t.dNp; }
  struct Acc {
    DfAcc x, y;
  };
  __device__ static __forceinline__ Acc acc(C v) { return Acc{dfacc(v.x), dfacc(v.y)}; }
  __device__ static __forceinline__ void acc_add(Acc& s, R a, C v) { dfacc_add(s.x, a, v.x); dfacc_add(s.y, a, v.y); }
  __device__ static __forceinline__ C acc_done(const Acc& s) { return dfc{dfacc_done(s.x), dfacc_done(s.y)}; }
};

template <class Y, int N>
__device__ __forceinline__ void ypush(typename Y::C (&w)[N], typename Y::C x) {
#pragma unroll
  for (int d = 0; d < N - 1; ++d) w[d] = w[d + 1];
  w[N - 1] = x;
}
template <class Y>
__device__ __forceinline__ typename Y::C yband7(const typename Y::R* c, const typename Y::C (&w)[7]) {
  typename Y::Acc r = Y::acc(Y::zero());
#pragma unroll
  for (int d = 0; d < 7; ++d) Y::acc_add(r, c[d], w[d]);
  return Y::acc_done(r);
}
template <class Y>
__device__ __forceinline__ typename Y::C yfwd(typename Y::C r, typename Y::R l0, typename Y::R l1, typename Y::R l2,
                                              typename Y::C (&hist)[3]) {
  typename Y::Acc s = Y::acc(r);
  Y::acc_add(s, Y::neg(l0), hist[0]);
  Y::acc_add(s, Y::neg(l1), hist[1]);
  Y::acc_add(s, Y::neg(l2), hist[2]);
  r = Y::acc_done(s);
  ypush<Y>(hist, r);
  return r;
}
template <class Y>
__device__ __forceinline__ typename Y::C ybwd(typename Y::C z, typename Y::R u0, typename Y::R u1, typename Y::R u2,
                                              typename Y::R dinv, typename Y::C (&nxt)[3]) {
  typename Y::Acc s = Y::acc(z);
  Y::acc_add(s, Y::neg(u0), nxt[0]);
  Y::acc_add(s, Y::neg(u1), nxt[1]);
  Y::acc_add(s, Y::neg(u2), nxt[2]);
  z = Y::acc_done(s);
  typename Y::C x = Y::scl(dinv, z);
  nxt[2] = nxt[1];
  nxt[1] = nxt[0];
  nxt[0] = x;
  return x;
}
// A mode-independent y table: staged in shared memory (when stage), else read in place
// from global memory (every thread of a warp reads the same row: L1 broadcasts).
template <class Y>
__device__ __forceinline__ const typename Y::R* ystage(typename Y::R*& dst, const typename Y::R* src, int n,
                                                       bool stage) {
  if (!stage) return src;
  typename Y::R* d = dst;
  for (int k = threadIdx.x; k < n; k += blockDim.x) d[k] = src[k];
  dst += n;
  return d;
}

struct ModeInfo {
  int jz, kx, c;
  bool nyq;
  double k1, k3, k2;
};

__device__ __forceinline__ ModeInfo mode_info(const Geo& g, int m) {
  ModeInfo mi;
  mi.jz = m / g.nxh;
  mi.kx = m - mi.jz * g.nxh;
  const int hz = g.Nz / 2;
  mi.nyq = (mi.jz == hz);
  int kza = mi.jz < hz ? mi.jz : g.Nz - mi.jz;
  mi.c = mi.nyq ? 0 : kza * g.nxh + mi.kx;
  mi.k1 = g.k1[mi.kx];
  mi.k3 = g.k3[mi.jz];
  mi.k2 = mi.k1 * mi.k1 + mi.k3 * mi.k3;
  return mi;
}

// ---------------------------------------------------------------------------
// a1: u_1, u_3, omega_1, omega_3 from (v, omega_2, dv/dy); two D1 sweeps.
// dv/dy is part of the state (it is D1 v of the last Poisson solve).
// ---------------------------------------------------------------------------
// F32OUT (mixed modes, substep path): the two D1 sweeps stay in the sweep precision (FP64
// or pairs); u_1, u_3, omega_1, omega_3, which only feed the FP32 transforms, are formed in
// FP32 from those values and stored as float2: u_1, u_3 in the omega_1 slot ([2][Ny][M]
// float2), omega_1, omega_3 in the omega_3 slot; the u_1, u_3 slots keep the forward sweep.

// One mode's two D1 sweeps and outputs; MEAN: the (0,0) mode, whose inputs are the mean
// profiles (a separate instantiation, so no per-row branch on it is issued elsewhere).
template <class Y, bool F32OUT, bool MEAN>
__device__ __forceinline__ void pre_sweep(const Geo& g, const typename Y::R* sB1, const typename Y::R* sLU,
                                          const ModeInfo& mi, int m, const double2* CHAN_RO v,
                                          const double2* CHAN_RO om, const double2* CHAN_RO dv,
                                          const double* CHAN_RO U1, const double* CHAN_RO U3,
                                          double2* u1o, double2* u3o, double2* om1o, double2* om3o, void* ring) {
  typedef typename Y::R R;
  typedef typename Y::C C;
  const int Ny = g.Ny;
  const size_t M = g.M;
  const size_t nf = (size_t)Ny * M;
  float2* fu = reinterpret_cast<float2*>(om1o);   // F32OUT: u_1 [0, nf), u_3 [nf, 2 nf)
  float2* fw = reinterpret_cast<float2*>(om3o);   //         omega_1, omega_3
  Ring<5, 0> rg(ring);
  C wx[7], ww[7], hx[3], hw[3];
#pragma unroll
  for (int d = 0; d < 7; ++d) { wx[d] = Y::zero(); ww[d] = Y::zero(); }
#pragma unroll
  for (int d = 0; d < 3; ++d) { hx[d] = Y::zero(); hw[d] = Y::zero(); }
  // forward sweep of D1 = A1^-1 B1 on x = dv/dy (U1 for the mean) and w = omega_2 (U3),
  // parked in the u_1, u_3 outputs
  pipelined(
      Ny + 3,
      [&](int t, int st) {
        if (!MEAN && t < Ny) {
          const size_t o = (size_t)t * M + m;
          cp16(rg.f(st, 0), dv + o);
          cp16(rg.f(st, 1), om + o);
        }
      },
      [&](int t, int st) {
        C nx = Y::zero(), nw = Y::zero();
        if (t < Ny) {
          if (MEAN) { nx = Y::c(make_double2(U1[t], 0.0)); nw = Y::c(make_double2(U3[t], 0.0)); }
          else { nx = Y::lds(rg.f(st, 0)); nw = Y::lds(rg.f(st, 1)); }
        }
        ypush<Y>(wx, nx);
        ypush<Y>(ww, nw);
        const int i = t - 3;
        if (i < 0) return;
        const R* b = sB1 + 7 * i;
        const R* l = sLU + 7 * i;
        Y::st(u1o, (size_t)i * M + m, yfwd<Y>(yband7<Y>(b, wx), l[0], l[1], l[2], hx));
        Y::st(u3o, (size_t)i * M + m, yfwd<Y>(yband7<Y>(b, ww), l[0], l[1], l[2], hw));
      });
  C px[3] = {Y::zero(), Y::zero(), Y::zero()}, pw[3] = {Y::zero(), Y::zero(), Y::zero()};
  const R q1 = Y::r(MEAN ? 0.0 : mi.k1 / mi.k2), q3 = Y::r(MEAN ? 0.0 : mi.k3 / mi.k2);
  const R k1 = Y::r(mi.k1), k3 = Y::r(mi.k3);
  const float q1f = MEAN ? 0.f : (float)(mi.k1 / mi.k2), q3f = MEAN ? 0.f : (float)(mi.k3 / mi.k2);
  const float k1f = (float)mi.k1, k3f = (float)mi.k3;
  pipelined(
      Ny,
      [&](int q, int st) {
        const size_t o = (size_t)(Ny - 1 - q) * M + m;
        cp16(rg.f(st, 0), u1o + o);
        cp16(rg.f(st, 1), u3o + o);
        if (!MEAN) {
          cp16(rg.f(st, 2), dv + o);
          cp16(rg.f(st, 3), om + o);
          cp16(rg.f(st, 4), v + o);
        }
      },
      [&](int q, int st) {
        const int i = Ny - 1 - q;
        const size_t o = (size_t)i * M + m;
        const R* lu = sLU + 7 * i;
        const C P = ybwd<Y>(Y::lds(rg.f(st, 0)), lu[3], lu[4], lu[5], lu[6], px);   // D1 of dv/dy
        const C Q = ybwd<Y>(Y::lds(rg.f(st, 1)), lu[3], lu[4], lu[5], lu[6], pw);   // D1 omega_2
        if constexpr (F32OUT) {
          const float2 fP = Y::f(P), fQ = Y::f(Q);
          float2 a1, a3, d1, d3, fv = make_float2(0.f, 0.f);
          if (MEAN) {
            a1 = make_float2(d2f_int(U1[i]), 0.f);
            a3 = make_float2(d2f_int(U3[i]), 0.f);
            d1 = fP;
            d3 = fQ;
          } else {
            const float2 fd = Y::ldsf(rg.f(st, 2)), fo = Y::ldsf(rg.f(st, 3));
            fv = Y::ldsf(rg.f(st, 4));
            // u_1 = i (q1 dv - q3 om), u_3 = i (q3 dv + q1 om), likewise d/dy from (P, Q)
            a1 = make_float2(-(q1f * fd.y - q3f * fo.y), q1f * fd.x - q3f * fo.x);
            a3 = make_float2(-(q3f * fd.y + q1f * fo.y), q3f * fd.x + q1f * fo.x);
            d1 = make_float2(-(q1f * fP.y - q3f * fQ.y), q1f * fP.x - q3f * fQ.x);
            d3 = make_float2(-(q3f * fP.y + q1f * fQ.y), q3f * fP.x + q1f * fQ.x);
          }
          fu[o] = a1;
          fu[nf + o] = a3;
          fw[o] = make_float2(d3.x + k3f * fv.y, d3.y - k3f * fv.x);        // du3/dy - i k3 v
          fw[nf + o] = make_float2(-k1f * fv.y - d1.x, k1f * fv.x - d1.y);  // i k1 v - du1/dy
          return;
        }
        C u1, u3, du1, du3, vi = Y::zero();
        if (MEAN) {
          u1 = Y::c(make_double2(U1[i], 0.0));
          u3 = Y::c(make_double2(U3[i], 0.0));
          du1 = P;
          du3 = Q;
        } else {
          const C dvi = Y::lds(rg.f(st, 2)), omi = Y::lds(rg.f(st, 3));
          vi = Y::lds(rg.f(st, 4));
          u1 = Y::itimes(Y::axpy(Y::neg(q3), omi, Y::scl(q1, dvi)));
          u3 = Y::itimes(Y::axpy(q1, omi, Y::scl(q3, dvi)));
          du1 = Y::itimes(Y::axpy(Y::neg(q3), Q, Y::scl(q1, P)));
          du3 = Y::itimes(Y::axpy(q1, Q, Y::scl(q3, P)));
        }
        // omega_1 = du3/dy - i k3 v, omega_3 = i k1 v - du1/dy
        Y::st(u1o, o, u1);
        Y::st(u3o, o, u3);
        Y::st(om1o, o, Y::sub(du3, Y::itimes(Y::scl(k3, vi))));
        Y::st(om3o, o, Y::sub(Y::itimes(Y::scl(k1, vi)), du1));
      });
}

template <class Y, bool F32OUT = false>
__device__ __forceinline__ void pre_body(Geo g, YTabs t, const double2* CHAN_RO v,
                                         const double2* CHAN_RO om, const double2* CHAN_RO dv,
                                         const double* CHAN_RO U1, const double* CHAN_RO U3,
                                         double2* u1o, double2* u3o, double2* om1o, double2* om3o, int bid) {
  typedef typename Y::R R;
  extern __shared__ double sm[];
  const int Ny = g.Ny;
  R* sp = reinterpret_cast<R*>(sm);
  const R* sB1 = ystage<Y>(sp, Y::B1(t), 7 * Ny, !g.gtab);
  const R* sLU = ystage<Y>(sp, Y::LU1(t), 7 * Ny, !g.gtab);
  if (!g.gtab) __syncthreads();
  void* ring = ring_base(sp);
  // The (0,0) mode runs its own instantiation of the sweeps in a block of its own (the one
  // after the mode blocks), so no warp holds both code paths.
  const int nblk = (g.M + blockDim.x - 1) / blockDim.x;
  if (bid == nblk) {
    if (threadIdx.x == 0)
      pre_sweep<Y, F32OUT, true>(g, sB1, sLU, mode_info(g, 0), 0, v, om, dv, U1, U3, u1o, u3o, om1o, om3o, ring);
    return;
  }
  const int m = bid * blockDim.x + threadIdx.x;
  if (m >= g.M || m == 0) return;
  const size_t M = g.M;
  ModeInfo mi = mode_info(g, m);
  const size_t nf = (size_t)Ny * M;
  float2* fu = reinterpret_cast<float2*>(om1o);
  float2* fw = reinterpret_cast<float2*>(om3o);
  if (mi.nyq) {
    for (int i = 0; i < Ny; ++i) {
      size_t o = (size_t)i * M + m;
      if (F32OUT) {
        const float2 z = make_float2(0.f, 0.f);
        fu[o] = z; fu[nf + o] = z; fw[o] = z; fw[nf + o] = z;
      } else {
        u1o[o] = z2(); u3o[o] = z2(); om1o[o] = z2(); om3o[o] = z2();
      }
    }
    return;
  }
  pre_sweep<Y, F32OUT, false>(g, sB1, sLU, mi, m, v, om, dv, U1, U3, u1o, u3o, om1o, om3o, ring);
}

// ---------------------------------------------------------------------------
// a5: N_omega2 = i k3 H1 - i k1 H3, N_chi = -D1(i k1 H1 + i k3 H3) - k^2 H2.
// ---------------------------------------------------------------------------
template <class Y>
__device__ __forceinline__ void nonlin_body(Geo g, YTabs t, const double2* CHAN_RO H1,
                                            const double2* CHAN_RO H2, const double2* CHAN_RO H3,
                                            double2* Nchi, double2* Nom, double2* scr_, int bid) {
  typedef typename Y::R R;
  typedef typename Y::C C;
  extern __shared__ double sm[];
  const int Ny = g.Ny;
  R* sp = reinterpret_cast<R*>(sm);
  const R* sB1 = ystage<Y>(sp, Y::B1(t), 7 * Ny, !g.gtab);
  const R* sLU = ystage<Y>(sp, Y::LU1(t), 7 * Ny, !g.gtab);
  if (!g.gtab) __syncthreads();
  void* ring = ring_base(sp);
  const int m = bid * blockDim.x + threadIdx.x;
  if (m >= g.M) return;
  const size_t M = g.M;
  ModeInfo mi = mode_info(g, m);
  if (mi.nyq || m == 0) {
    for (int i = 0; i < Ny; ++i) { Nchi[(size_t)i * M + m] = z2(); Nom[(size_t)i * M + m] = z2(); }
    return;
  }
  double2* scr = scr_;
  const R k1 = Y::r(mi.k1), k3 = Y::r(mi.k3), mk2 = Y::r(-mi.k2);
  Ring<4, 0> rg(ring);
  C w[7], hz[3];
#pragma unroll
  for (int d = 0; d < 7; ++d) w[d] = Y::zero();
#pragma unroll
  for (int d = 0; d < 3; ++d) hz[d] = Y::zero();
  pipelined(
      Ny + 3,
      [&](int t, int st) {
        if (t < Ny) {
          const size_t o = (size_t)t * M + m;
          cp16(rg.f(st, 0), H1 + o);
          cp16(rg.f(st, 1), H3 + o);
        }
      },
      [&](int t, int st) {
        C f = Y::zero();
        if (t < Ny) f = Y::itimes(Y::axpy(k3, Y::lds(rg.f(st, 1)), Y::scl(k1, Y::lds(rg.f(st, 0)))));   // i k1 H1 + i k3 H3
        ypush<Y>(w, f);
        const int i = t - 3;
        if (i < 0) return;
        const R* l = sLU + 7 * i;
        Y::st(scr, (size_t)i * M + m, yfwd<Y>(yband7<Y>(sB1 + 7 * i, w), l[0], l[1], l[2], hz));
      });
  C nx[3] = {Y::zero(), Y::zero(), Y::zero()};
  pipelined(
      Ny,
      [&](int q, int st) {
        const size_t o = (size_t)(Ny - 1 - q) * M + m;
        cp16(rg.f(st, 0), scr + o);
        cp16(rg.f(st, 1), H2 + o);
        cp16(rg.f(st, 2), H1 + o);
        cp16(rg.f(st, 3), H3 + o);
      },
      [&](int q, int st) {
        const int i = Ny - 1 - q;
        const size_t o = (size_t)i * M + m;
        const R* lu = sLU + 7 * i;
        const C d = ybwd<Y>(Y::lds(rg.f(st, 0)), lu[3], lu[4], lu[5], lu[6], nx);
        const C h2 = Y::lds(rg.f(st, 1)), h1 = Y::lds(rg.f(st, 2)), h3 = Y::lds(rg.f(st, 3));
        Y::st(Nchi, o, Y::axpy(mk2, h2, Y::sub(Y::zero(), d)));                 // -D1 f - k^2 H2
        Y::st(Nom, o, Y::itimes(Y::axpy(Y::neg(k1), h3, Y::scl(k3, h1))));      // i k3 H1 - i k1 H3
      });
}

// ---------------------------------------------------------------------------
// a6 + first half of a7: implicit RK3 Helmholtz steps of omega_2 and chi
// (Eqs. (psi), (chi1)) multiplied through by A:
//   [(1 + b dt nu k^2) A - b dt nu B] X+ = A[(1 - a dt nu k^2) X + dt(g N + z Nprev)] + a dt nu B X,
// wall rows X+ = 0 (chi's are the particular solution).  Nprev <- N.
// The interior right-hand side R of each solve is kept; in the next substep
// (coefficients b' of the previous one) B X follows from it, since
// [(1 + b' dt nu k^2) A - b' dt nu B] X = R' on interior rows (the wall
// corrections of chi leave interior rows unchanged), and the right-hand side
// becomes A[(1 + a/b') X + dt(g N + z Nprev)] - (a/b') R' with no B product.
// The first substep after a state upload (flag scal[2] = 0) uses B X directly.
// ---------------------------------------------------------------------------
// One field (omega_2 or chi) of one mode: right-hand side, forward and backward sweeps.
template <class Y, bool PREV>
__device__ __forceinline__ void helm_one(int Ny, size_t M, size_t NC, int m, const typename Y::R* sA,
                                         const typename Y::R* sB, const typename Y::R* CHAN_RO H, double2* X,
                                         const double2* CHAN_RO N, double2* Np, double2* Rf, double2* scr,
                                         typename Y::R c1, typename Y::R cg, typename Y::R cz,
                                         typename Y::R ca, typename Y::R qp, void* ring) {
  typedef typename Y::R R;
  typedef typename Y::C C;
  Ring<4, 4> rg(ring);
  C wa[7], wx[7], hz[3];
#pragma unroll
  for (int d = 0; d < 7; ++d) { wa[d] = Y::zero(); wx[d] = Y::zero(); }
#pragma unroll
  for (int d = 0; d < 3; ++d) hz[d] = Y::zero();
  // forward: row t of N, X, Nprev and, three rows behind, the kept right-hand side and the
  // L factors of row t - 3
  pipelined(
      Ny + 3,
      [&](int t, int st) {
        if (t < Ny) {
          const size_t o = (size_t)t * M + m;
          cp16(rg.f(st, 0), N + o);
          cp16(rg.f(st, 1), X + o);
          cp16(rg.f(st, 2), Np + o);
        }
        const int i = t - 3;
        if (i >= 0) {
          if (PREV && i > 0 && i < Ny - 1) cp16(rg.f(st, 3), Rf + (size_t)i * M + m);
          const R* Hi = H + (size_t)i * 11 * NC;
          cp8(rg.t(st, 0), Hi);
          cp8(rg.t(st, 1), Hi + NC);
          cp8(rg.t(st, 2), Hi + 2 * NC);
        }
      },
      [&](int t, int st) {
        C a = Y::zero(), x = Y::zero();
        if (t < Ny) {
          const C n = Y::lds(rg.f(st, 0));
          x = Y::lds(rg.f(st, 1));
          a = Y::axpy(cz, Y::lds(rg.f(st, 2)), Y::axpy(cg, n, Y::scl(c1, x)));
          Y::st(Np, (size_t)t * M + m, n);
        }
        ypush<Y>(wa, a);
        ypush<Y>(wx, x);
        const int i = t - 3;
        if (i < 0) return;
        C r = Y::zero();
        if (i > 0 && i < Ny - 1) {
          if constexpr (PREV) r = Y::axpy(qp, Y::lds(rg.f(st, 3)), yband7<Y>(sA + 7 * i, wa));
          else r = Y::axpy(ca, yband7<Y>(sB + 7 * i, wx), yband7<Y>(sA + 7 * i, wa));
          if (Rf) Y::st(Rf, (size_t)i * M + m, r);   // kept unless the handle keeps none (lean boxes)
        }
        Y::st(scr, (size_t)i * M + m,
              yfwd<Y>(r, Y::ldr(rg.t(st, 0)), Y::ldr(rg.t(st, 1)), Y::ldr(rg.t(st, 2)), hz));
      });
  C nx[3] = {Y::zero(), Y::zero(), Y::zero()};
  pipelined(
      Ny,
      [&](int q, int st) {
        const int i = Ny - 1 - q;
        cp16(rg.f(st, 0), scr + (size_t)i * M + m);
        const R* Hi = H + (size_t)i * 11 * NC;
        cp8(rg.t(st, 0), Hi + 3 * NC);
        cp8(rg.t(st, 1), Hi + 4 * NC);
        cp8(rg.t(st, 2), Hi + 5 * NC);
        cp8(rg.t(st, 3), Hi + 6 * NC);
      },
      [&](int q, int st) {
        const int i = Ny - 1 - q;
        Y::st(X, (size_t)i * M + m,
              ybwd<Y>(Y::lds(rg.f(st, 0)), Y::ldr(rg.t(st, 0)), Y::ldr(rg.t(st, 1)), Y::ldr(rg.t(st, 2)),
                      Y::ldr(rg.t(st, 3)), nx));
      });
}

// FS: 0 omega_2 only, 1 chi only, 2 both (one after the other).  Each field's arithmetic
// is the same in every form, so one thread per (mode, field) and one per mode agree bitwise.
template <class Y, int FS>
__device__ __forceinline__ void helm_body(Geo g, YTabs t, const typename Y::R* CHAN_RO helm,
                                          double2* om, double2* chi, const double2* CHAN_RO Nchi,
                                          const double2* CHAN_RO Nom, double2* Nchi_p, double2* Nom_p,
                                          double2* Rom, double2* Rchi, const double* CHAN_RO scal,
                                          double2* scr_, int s, int bid) {
  typedef typename Y::R R;
  extern __shared__ double sm[];
  const int Ny = g.Ny;
  R* sp = reinterpret_cast<R*>(sm);
  const R* sA = ystage<Y>(sp, Y::A2(t), 7 * Ny, !g.gtab);
  const R* sB = ystage<Y>(sp, Y::B2(t), 7 * Ny, !g.gtab);
  if (!g.gtab) __syncthreads();
  void* ring = ring_base(sp);
  const int m = bid * blockDim.x + threadIdx.x;
  if (m >= g.M) return;
  const size_t M = g.M;
  const size_t NC = g.C;
  ModeInfo mi = mode_info(g, m);
  if (mi.nyq) {
    for (int i = 0; i < Ny; ++i) {
      size_t o = (size_t)i * M + m;
      if (FS != 1) { om[o] = z2(); Nom_p[o] = z2(); }
      if (FS != 0) { chi[o] = z2(); Nchi_p[o] = z2(); }
    }
    return;
  }
  const double gm = c_rk3[s][0], zt = c_rk3[s][1], al = c_rk3[s][2];
  const double dt = g.dt, nu = g.nu;
  // the previous substep's right-hand sides are valid (a lean box keeps none: Rom = NULL)
  const bool prev = Rom != nullptr && scal[2] != 0.0;
  const double bp = c_rk3[(s + 2) % 3][3];
  const R c1 = Y::r(prev ? 1.0 + al / bp : 1.0 - al * dt * nu * mi.k2), cg = Y::r(dt * gm), cz = Y::r(dt * zt);
  const R ca = Y::r(al * dt * nu), qp = Y::r(-al / bp);
  const R* H = helm + mi.c;   // the substep's slot
  // separate instantiations: the B product of the first substep is not issued under a predicate
  double2* scr2 = scr_ + (size_t)Ny * M;
  if (prev) {
    if (FS != 1) helm_one<Y, true>(Ny, M, NC, m, sA, sB, H, om, Nom, Nom_p, Rom, scr_, c1, cg, cz, ca, qp, ring);
    if (FS != 0) helm_one<Y, true>(Ny, M, NC, m, sA, sB, H, chi, Nchi, Nchi_p, Rchi, scr2, c1, cg, cz, ca, qp, ring);
  } else {
    if (FS != 1) helm_one<Y, false>(Ny, M, NC, m, sA, sB, H, om, Nom, Nom_p, Rom, scr_, c1, cg, cz, ca, qp, ring);
    if (FS != 0) helm_one<Y, false>(Ny, M, NC, m, sA, sB, H, chi, Nchi, Nchi_p, Rchi, scr2, c1, cg, cz, ca, qp, ring);
  }
}

// ---------------------------------------------------------------------------
// Second half of a7: (B - k^2 A) v_p = A chi_p, v_p(+-1) = 0 (Eq. (chi2));
// v = v_p + c_a v_a + c_b v_b and chi likewise, with (c_a, c_b) making
// dv/dy(+-1) = 0 through the precomputed influence matrix; then dv/dy = D1 v.
// ---------------------------------------------------------------------------
template <class Y>
__device__ __forceinline__ void poisson_body(Geo g, YTabs t, const typename Y::R* CHAN_RO helm,
                                             const typename Y::R* CHAN_RO pois,
                                             const typename Y::R* CHAN_RO infl, double2* v, double2* chi,
                                             double2* dv, double2* scr_, double* scal, int s, int bid) {
  // the Helmholtz right-hand sides of this substep are in place for the next one (the
  // Helmholtz kernel of this substep, which reads the flag, is complete)
  if (bid == 0 && threadIdx.x == 0) scal[2] = 1.0;
  typedef typename Y::R R;
  typedef typename Y::C C;
  extern __shared__ double sm[];
  const int Ny = g.Ny;
  R* sp = reinterpret_cast<R*>(sm);
  const R* sA = ystage<Y>(sp, Y::A2(t), 7 * Ny, !g.gtab);
  const R* sB1 = ystage<Y>(sp, Y::B1(t), 7 * Ny, !g.gtab);
  const R* sLU = ystage<Y>(sp, Y::LU1(t), 7 * Ny, !g.gtab);
  const R* sd0 = ystage<Y>(sp, Y::D0(t), Ny, !g.gtab);
  const R* sdN = ystage<Y>(sp, Y::DN(t), Ny, !g.gtab);
  if (!g.gtab) __syncthreads();
  void* ring = ring_base(sp);
  const int m = bid * blockDim.x + threadIdx.x;
  if (m >= g.M) return;
  const size_t M = g.M;
  const size_t NC = g.C;
  ModeInfo mi = mode_info(g, m);
  if (mi.nyq) {
    for (int i = 0; i < Ny; ++i) { size_t o = (size_t)i * M + m; v[o] = z2(); dv[o] = z2(); }
    return;
  }
  const R* P = pois + mi.c;
  const R* H = helm + mi.c;   // the substep's slot
  double2* scr = scr_;
  Ring<2, 4> rg(ring);
  C w[7], hz[3];
#pragma unroll
  for (int d = 0; d < 7; ++d) w[d] = Y::zero();
#pragma unroll
  for (int d = 0; d < 3; ++d) hz[d] = Y::zero();
  // particular solution: forward sweep of (B - k^2 A) v_p = A chi_p (interior rows)
  pipelined(
      Ny + 3,
      [&](int t, int st) {
        if (t < Ny) cp16(rg.f(st, 0), chi + (size_t)t * M + m);
        const int i = t - 3;
        if (i >= 0) {
          const R* Pi = P + (size_t)i * 7 * NC;
          cp8(rg.t(st, 0), Pi);
          cp8(rg.t(st, 1), Pi + NC);
          cp8(rg.t(st, 2), Pi + 2 * NC);
        }
      },
      [&](int t, int st) {
        ypush<Y>(w, t < Ny ? Y::lds(rg.f(st, 0)) : Y::zero());
        const int i = t - 3;
        if (i < 0) return;
        C r = (i > 0 && i < Ny - 1) ? yband7<Y>(sA + 7 * i, w) : Y::zero();
        Y::st(scr, (size_t)i * M + m,
              yfwd<Y>(r, Y::ldr(rg.t(st, 0)), Y::ldr(rg.t(st, 1)), Y::ldr(rg.t(st, 2)), hz));
      });
  C nx[3] = {Y::zero(), Y::zero(), Y::zero()};
  C s0 = Y::zero(), sN = Y::zero();
  pipelined(
      Ny,
      [&](int q, int st) {
        const int i = Ny - 1 - q;
        cp16(rg.f(st, 0), scr + (size_t)i * M + m);
        const R* Pi = P + (size_t)i * 7 * NC;
        cp8(rg.t(st, 0), Pi + 3 * NC);
        cp8(rg.t(st, 1), Pi + 4 * NC);
        cp8(rg.t(st, 2), Pi + 5 * NC);
        cp8(rg.t(st, 3), Pi + 6 * NC);
      },
      [&](int q, int st) {
        const int i = Ny - 1 - q;
        const C vp = ybwd<Y>(Y::lds(rg.f(st, 0)), Y::ldr(rg.t(st, 0)), Y::ldr(rg.t(st, 1)), Y::ldr(rg.t(st, 2)),
                             Y::ldr(rg.t(st, 3)), nx);
        Y::st(scr, (size_t)i * M + m, vp);   // v_p parked in the scratch until the wall correction is known
        s0 = Y::axpy(sd0[i], vp, s0);
        sN = Y::axpy(sdN[i], vp, sN);
      });
  const R* Gi = infl + mi.c;
  const R g11 = Gi[0], g12 = Gi[NC], g21 = Gi[2 * NC], g22 = Gi[3 * NC];  // inverse influence matrix
  const C cA = Y::sub(Y::zero(), Y::axpy(g12, sN, Y::scl(g11, s0)));
  const C cB = Y::sub(Y::zero(), Y::axpy(g22, sN, Y::scl(g21, s0)));
  double2* scr2 = scr + (size_t)Ny * M;
#pragma unroll
  for (int d = 0; d < 7; ++d) w[d] = Y::zero();
#pragma unroll
  for (int d = 0; d < 3; ++d) hz[d] = Y::zero();
  // v = v_p + c_a v_a + c_b v_b, chi likewise; forward sweep of dv/dy = D1 v
  pipelined(
      Ny + 3,
      [&](int t, int st) {
        if (t < Ny) {
          const size_t o = (size_t)t * M + m;
          cp16(rg.f(st, 0), scr + o);
          cp16(rg.f(st, 1), chi + o);
          const R* Hj = H + (size_t)t * 11 * NC;
          cp8(rg.t(st, 0), Hj + 7 * NC);
          cp8(rg.t(st, 1), Hj + 8 * NC);
          cp8(rg.t(st, 2), Hj + 9 * NC);
          cp8(rg.t(st, 3), Hj + 10 * NC);
        }
      },
      [&](int t, int st) {
        C vj = Y::zero();
        if (t < Ny) {
          const size_t o = (size_t)t * M + m;
          const R xa = Y::ldr(rg.t(st, 0)), xb = Y::ldr(rg.t(st, 1)), va = Y::ldr(rg.t(st, 2)),
                  vb = Y::ldr(rg.t(st, 3));
          vj = Y::axpy(vb, cB, Y::axpy(va, cA, Y::lds(rg.f(st, 0))));
          Y::st(v, o, vj);
          Y::st(chi, o, Y::axpy(xb, cB, Y::axpy(xa, cA, Y::lds(rg.f(st, 1)))));
        }
        ypush<Y>(w, vj);
        const int i = t - 3;
        if (i < 0) return;
        const R* l = sLU + 7 * i;
        Y::st(scr2, (size_t)i * M + m, yfwd<Y>(yband7<Y>(sB1 + 7 * i, w), l[0], l[1], l[2], hz));
      });
  for (int d = 0; d < 3; ++d) nx[d] = Y::zero();
  pipelined(
      Ny,
      [&](int q, int st) { cp16(rg.f(st, 0), scr2 + (size_t)(Ny - 1 - q) * M + m); },
      [&](int q, int st) {
        const int i = Ny - 1 - q;
        const R* lu = sLU + 7 * i;
        Y::st(dv, (size_t)i * M + m, ybwd<Y>(Y::lds(rg.f(st, 0)), lu[3], lu[4], lu[5], lu[6], nx));
      });
}

// ---------------------------------------------------------------------------
// a8: mean profiles.  The (0,0) Helmholtz factors (k = 0) of substep s serve
//   (A - b dt nu B) U+ = A[U + dt(g <H> + z <H>prev)] + a dt nu B U,  U+(+-1) = 0.
// U_1 gets c U_h with U_h = (A - b dt nu B)^-1 A 1 (precomputed per substep)
// so the trapezoid flux stays Q0; f = c / ((a + b) dt).  One block: the
// right-hand sides and the flux sums are row-parallel, the two banded
// sweeps (U_1, U_3) run on two warps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mean_body(Geo g, YTabs t, const double* CHAN_RO helm,
                                              const double* CHAN_RO meanh, const double2* CHAN_RO H1,
                                              const double2* CHAN_RO H3, double* U1, double* U3, double* H1p,
                                              double* H3p, double* scal, int s, int bid) {
  extern __shared__ double sm[];
  const int Ny = g.Ny;
  const size_t M = g.M, C = g.C;
  double* r1 = sm;            // right-hand sides, then the solutions
  double* r3 = sm + Ny;
  double* red = sm + 2 * Ny;  // [256]
  double* sH = red + 256;     // [Ny][7] the k = 0 factors, staged by all threads for the serial sweeps
  const double gm = c_rk3[s][0], zt = c_rk3[s][1], al = c_rk3[s][2], be = c_rk3[s][3];
  const double dt = g.dt, nu = g.nu;
  for (int k = threadIdx.x; k < 7 * Ny; k += blockDim.x) {
    const int i = k / 7, q = k - 7 * i;
    sH[k] = helm[((size_t)i * 11 + q) * C];
  }
  for (int i = threadIdx.x; i < Ny; i += blockDim.x) {
    double a1 = 0.0, a3 = 0.0;
    if (i > 0 && i < Ny - 1) {
      for (int d = 0; d < 7; ++d) {
        const int j = i - 3 + d;
        if (j < 0 || j >= Ny) continue;
        const double A = t.A2[7 * i + d], B = t.B2[7 * i + d];
        const double u1 = U1[j], u3 = U3[j];
        a1 += A * (u1 + dt * (gm * load_re(H1, (size_t)j * M, g.pair) + zt * H1p[j])) + al * dt * nu * B * u1;
        a3 += A * (u3 + dt * (gm * load_re(H3, (size_t)j * M, g.pair) + zt * H3p[j])) + al * dt * nu * B * u3;
      }
    }
    r1[i] = a1;
    r3[i] = a3;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
    double* r = threadIdx.x == 0 ? r1 : r3;
    double h[3] = {0, 0, 0};
    for (int i = 0; i < Ny; ++i) {
      const double* Hi = sH + 7 * i;
      double x = r[i] - Hi[0] * h[0] - Hi[1] * h[1] - Hi[2] * h[2];
      h[0] = h[1]; h[1] = h[2]; h[2] = x;
      r[i] = x;
    }
    double nx[3] = {0, 0, 0};
    for (int i = Ny - 1; i >= 0; --i) {
      const double* Hi = sH + 7 * i;
      double x = (r[i] - Hi[3] * nx[0] - Hi[4] * nx[1] - Hi[5] * nx[2]) * Hi[6];
      nx[2] = nx[1]; nx[1] = nx[0]; nx[0] = x;
      r[i] = x;
    }
  }
  __syncthreads();
  // flux of U_1* (fixed-order block reduction)
  double q = 0.0;
  for (int i = threadIdx.x; i < Ny; i += blockDim.x) q += t.wq[i] * r1[i];
  red[threadIdx.x] = q;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double* uh = meanh + (size_t)s * (Ny + 1);
  const double c = (scal[1] - red[0]) / uh[Ny];
  for (int i = threadIdx.x; i < Ny; i += blockDim.x) {
    H1p[i] = load_re(H1, (size_t)i * M, g.pair);
    H3p[i] = load_re(H3, (size_t)i * M, g.pair);
    U1[i] = r1[i] + c * uh[i];
    U3[i] = r3[i];
  }
  if (threadIdx.x == 0) scal[0] = c / ((al + be) * dt);
}

// Arguments of each body for one run (the packed and persistent launches).
struct PreP { Geo g; YTabs t; const double2 *v, *om, *dv; const double *U1, *U3; double2 *u1o, *u3o, *om1o, *om3o; };
struct NonlinP { Geo g; YTabs t; const double2 *H1, *H2, *H3; double2 *Nchi, *Nom, *scr; };
struct HelmP { Geo g; YTabs t; const void* helm; double2 *om, *chi; const double2 *Nchi, *Nom; double2 *Nchi_p, *Nom_p, *Rom, *Rchi; const double* scal; double2* scr; int s; };
struct PoisP { Geo g; YTabs t; const void *helm, *pois, *infl; double2 *v, *chi, *dv, *scr; double* scal; int s; };
struct MeanP { Geo g; YTabs t; const double *helm, *meanh; const double2 *H1, *H3; double *U1, *U3, *H1p, *H3p, *scal; int s; };

// ---------------------------------------------------------------------------
// Host helpers: the arguments of a run
// ---------------------------------------------------------------------------
static Geo geo(const chan_s* h) {
  Geo g;
  g.Nx = h->Nx; g.Ny = h->Ny; g.Nz = h->Nz; g.nxh = h->nxh; g.M = h->M; g.C = h->C;
  g.L1 = h->L1; g.L3 = h->L3; g.dt = h->dt; g.nu = h->nu; g.k1 = h->k1; g.k3 = h->k3;
  g.pair = prec_pairs(h->prec);
  g.gtab = ytab_in_place(h->ytab, h->Ny);
  return g;
}
static YTabs ytabs(const chan_s* h) {
  YTabs t;
  t.A2 = h->tab_A2; t.B2 = h->tab_B2; t.B1 = h->tab_B1; t.lu1 = h->tab_lu1; t.lu2f = h->tab_lu2f;
  t.d0 = h->tab_d0; t.dN = h->tab_dN; t.wq = h->tab_wq;
  const dfr* p = h->tab_pairs;
  const size_t r7 = 7 * (size_t)h->Ny;
  t.A2p = p; t.B2p = p ? p + r7 : nullptr; t.B1p = p ? p + 2 * r7 : nullptr; t.lu1p = p ? p + 3 * r7 : nullptr;
  t.d0p = p ? p + 4 * r7 : nullptr; t.dNp = p ? p + 4 * r7 + h->Ny : nullptr;
  return t;
}
// Tables of substep s: slot s, or the single slot refilled per substep (lean tables).
static double* helm_slot(const chan_s* h, int s) {
  return h->helm + (h->lean ? 0 : (size_t)s * h->Ny * 11 * h->C);
}
static const void* helm_slot_y(const chan_s* h, int s) {
  const size_t o = h->lean ? 0 : (size_t)s * h->Ny * 11 * h->C;
  return prec_pairs(h->prec) ? (const void*)(h->helm_df + o) : (const void*)(h->helm + o);
}
static const void* infl_slot_y(const chan_s* h, int s) {
  const size_t o = h->lean ? 0 : (size_t)s * 4 * h->C;
  return prec_pairs(h->prec) ? (const void*)(h->infl_df + o) : (const void*)(h->infl + o);
}
static const void* pois_y(const chan_s* h) {
  return prec_pairs(h->prec) ? (const void*)h->pois_df : (const void*)h->pois;
}
static const int kYThreads = 128;
// Shared memory of a sweep kernel of nt threads: the staged tables (per_y values per y point,
// none when the tables are read in place) and the kernel's row prefetch ring.
static size_t ysm_n(const chan_s* h, int per_y, size_t ring, int nt) {
  return (geo(h).gtab ? 0 : sizeof(double) * per_y * (size_t)h->Ny) + 16 + ring * nt;
}
static size_t ysm(const chan_s* h, int per_y, size_t ring) { return ysm_n(h, per_y, ring, kYThreads); }
static size_t ysm_batch(chan_s* const* hs, int n, int per_y, size_t ring) {
  size_t m = 0;
  for (int r = 0; r < n; ++r) m = ysm(hs[r], per_y, ring) > m ? ysm(hs[r], per_y, ring) : m;
  return m;
}
// Prefetch ring bytes per thread of each sweep kernel.
static const size_t kRingPre = Ring<5, 0>::per_thread, kRingNonlin = Ring<4, 0>::per_thread,
                    kRingHelm = Ring<4, 4>::per_thread, kRingPois = Ring<2, 4>::per_thread;
static dim3 ygrid(const chan_s* h) { return dim3((h->M + kYThreads - 1) / kYThreads); }

}  // namespace
