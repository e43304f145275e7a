// Device bodies of the transform passes (inverse z, fused x, forward z) and the host
// helpers that build their arguments.  Included by the transform kernels (kernels_fft.cu)
// and by the persistent work-list kernel (kernels_persist.cu).  CHAN_RO as in y_bodies.cuh.
#pragma once
#include <cstring>
#include <type_traits>

#include "chan_internal.cuh"
#include "df.cuh"

#ifndef CHAN_RO
#define CHAN_RO __restrict__
#endif

namespace {

template <typename T> struct V2;
template <> struct V2<double> { typedef double2 t; };
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<dfr> { typedef dfc t; };

template <typename T2> struct Scal;
template <> struct Scal<double2> { typedef double t; };
template <> struct Scal<float2> { typedef float t; };
template <> struct Scal<dfc> { typedef dfr t; };

// scalar helpers: conversion from / to double, halving, sqrt(3)/2
template <typename T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ dfr from_d<dfr>(double x) {
  const float h = __double2float_rn(x);
  return dfr{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(dfr x) { return (double)x.h + (double)x.l; }
__device__ __forceinline__ double half_of(double x) { return 0.5 * x; }
__device__ __forceinline__ float half_of(float x) { return 0.5f * x; }
__device__ __forceinline__ dfr half_of(dfr x) { return dfr{0.5f * x.h, 0.5f * x.l}; }
template <typename T> __device__ __forceinline__ T sqrt3_2();
template <> __device__ __forceinline__ double sqrt3_2<double>() { return 0.86602540378443864676; }
template <> __device__ __forceinline__ float sqrt3_2<float>() { return 0.86602540378443864676f; }
template <> __device__ __forceinline__ dfr sqrt3_2<dfr>() { return dfr{0x1.bb67aep-1f, 0x1.0b0996p-26f}; }

template <typename T2> __device__ __forceinline__ T2 zero2() {
  T2 r;
  memset(&r, 0, sizeof(T2));
  return r;
}

// Shared-memory slot of element i of a transform buffer row.  FP32 rows are swizzled
// within each 16-slot (128-byte) group: slot = i ^ 5 ((i >> 4) & 3).  The unit-span and
// span-4 stages of a radix-4 transform then hit 16 different bank pairs per half warp
// (unswizzled: 4-way conflicts, half of the FP32 passes' shared-memory wavefronts), and
// contiguous runs stay contiguous.  Rows hold whole groups (row stride a multiple of 16
// slots, plus one).  FP64 and pair transforms, bound by their arithmetic, keep i.
template <typename T2> struct Swz { static constexpr bool v = false; };
template <> struct Swz<float2> { static constexpr bool v = true; };
template <typename T2> __device__ __forceinline__ int sw(int i) {
  return Swz<T2>::v ? i ^ (((i >> 4) & 3) * 5) : i;
}

template <typename T2> __device__ __forceinline__ T2 mk(double x, double y) {
  typedef typename Scal<T2>::t T;
  T2 r;
  r.x = from_d<T>(x);
  r.y = from_d<T>(y);
  return r;
}

// A stored Fourier value in the transform type, optionally times the real filter
// factor g.  FP64 storage is converted (g applied in FP64); in the double-float
// mode the fields hold (hi, lo) float pairs, taken as they are (g as a pair).
template <typename T2> __device__ __forceinline__ T2 ld_fourier(const double2* p, size_t o, bool useg, double g) {
  double2 v = p[o];
  if (useg) { v.x *= g; v.y *= g; }
  return mk<T2>(v.x, v.y);
}
template <> __device__ __forceinline__ float2 ld_fourier<float2>(const double2* p, size_t o, bool useg, double g) {
  double2 v = p[o];
  if (useg) { v.x *= g; v.y *= g; }
  return make_float2(d2f_int(v.x), d2f_int(v.y));
}
template <> __device__ __forceinline__ dfc ld_fourier<dfc>(const double2* p, size_t o, bool useg, double g) {
  const float4 q = reinterpret_cast<const float4*>(p)[o];
  dfc v{dfr{q.x, q.y}, dfr{q.z, q.w}};
  if (useg) {
    const dfr gg = from_d<dfr>(g);
    v.x = v.x * gg;
    v.y = v.y * gg;
  }
  return v;
}
// Store a transform value as a Fourier value: FP64, or (pair) the raw (hi, lo) pairs.
template <typename T2> __device__ __forceinline__ void st_fourier(double2* p, size_t o, T2 x, int pair) {
  (void)pair;
  p[o] = make_double2(to_d(x.x), to_d(x.y));
}
template <> __device__ __forceinline__ void st_fourier<float2>(double2* p, size_t o, float2 x, int pair) {
  if (pair) reinterpret_cast<float4*>(p)[o] = make_float4(x.x, 0.f, x.y, 0.f);   // (hi, lo = 0) pairs
  else p[o] = make_double2(f2d_int(x.x), f2d_int(x.y));
}
// A pair-stored Fourier value rounded to FP32 (hi + lo), optionally times g.
__device__ __forceinline__ float2 ld_pair_f32(const double2* p, size_t o, bool useg, double g) {
  const float4 q = reinterpret_cast<const float4*>(p)[o];
  float2 v = make_float2(q.x + q.y, q.z + q.w);
  if (useg) {
    const float gf = d2f_int(g);
    v.x *= gf;
    v.y *= gf;
  }
  return v;
}
template <> __device__ __forceinline__ void st_fourier<dfc>(double2* p, size_t o, dfc x, int pair) {
  if (pair) reinterpret_cast<float4*>(p)[o] = make_float4(x.x.h, x.x.l, x.y.h, x.y.l);
  else p[o] = make_double2(to_d(x.x), to_d(x.y));
}

// A product that feeds an addition: plain for double and float, unnormalised pairs for dfr.
__device__ __forceinline__ double mulu(double a, double b) { return a * b; }
__device__ __forceinline__ float mulu(float a, float b) { return a * b; }
__device__ __forceinline__ dfr mulu(dfr a, dfr b) { return mul_u(a, b); }

// A sum that feeds another operation inside the butterfly: plain, or unnormalised pairs.
__device__ __forceinline__ double addu(double a, double b) { return a + b; }
__device__ __forceinline__ float addu(float a, float b) { return a + b; }
__device__ __forceinline__ dfr addu(dfr a, dfr b) { return add_u(a, b); }

template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {   // feeds the butterfly
  T2 r;
  r.x = addu(mulu(a.x, b.x), -mulu(a.y, b.y));
  r.y = addu(mulu(a.x, b.y), mulu(a.y, b.x));
  return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { T2 r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { T2 r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// inner sums of a butterfly (the outputs are formed with cadd / csub)
template <typename T2> __device__ __forceinline__ T2 caddu(T2 a, T2 b) { T2 r; r.x = addu(a.x, b.x); r.y = addu(a.y, b.y); return r; }
template <typename T2> __device__ __forceinline__ T2 csubu(T2 a, T2 b) { T2 r; r.x = addu(a.x, -b.x); r.y = addu(a.y, -b.y); return r; }

// Radix-R DFT in registers.  DIR = -1: exp(-2 pi i jk/R) (forward); +1: inverse.
template <int DIR, typename T2> __device__ __forceinline__ void dft2(T2* v) {
  T2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <int DIR, typename T2> __device__ __forceinline__ void dft4(T2* v) {
  T2 t0 = caddu(v[0], v[2]), t1 = csubu(v[0], v[2]);
  T2 t2 = caddu(v[1], v[3]), d = csubu(v[1], v[3]);
  T2 t3;  // DIR * i * d
  if (DIR < 0) { t3.x = d.y; t3.y = -d.x; } else { t3.x = -d.y; t3.y = d.x; }
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}
template <int DIR, typename T2> __device__ __forceinline__ void dft3(T2* v) {
  typedef typename Scal<T2>::t T;
  const T h = sqrt3_2<T>();
  T2 s = caddu(v[1], v[2]), d = csubu(v[1], v[2]);
  T2 y0 = cadd(v[0], s);
  T2 mm;
  mm.x = addu(v[0].x, -half_of(s.x));
  mm.y = addu(v[0].y, -half_of(s.y));
  // y1 = m + DIR * i * h * d, y2 = m - DIR * i * h * d
  T2 r;
  if (DIR < 0) { r.x = mulu(h, d.y); r.y = -mulu(h, d.x); } else { r.x = -mulu(h, d.y); r.y = mulu(h, d.x); }
  v[0] = y0;
  v[1] = cadd(mm, r);
  v[2] = csub(mm, r);
}
// Radix 3 with v[1] = 0: y0 = v0 + v2, y1 = v0 + w^2 v2, y2 = v0 + w v2 (w = exp(DIR 2 pi i / 3)).
template <int DIR, typename T2> __device__ __forceinline__ void dft3_zmid(T2* v) {
  typedef typename Scal<T2>::t T;
  const T h = sqrt3_2<T>();
  T2 c = v[2];
  T2 mm;
  mm.x = addu(v[0].x, -half_of(c.x));
  mm.y = addu(v[0].y, -half_of(c.y));
  T2 r;  // DIR * i * h * (v1 - v2) with v1 = 0
  if (DIR < 0) { r.x = -mulu(h, c.y); r.y = mulu(h, c.x); } else { r.x = mulu(h, c.y); r.y = -mulu(h, c.x); }
  v[0] = cadd(v[0], c);
  v[1] = cadd(mm, r);
  v[2] = csub(mm, r);
}
// Radix 3 without the middle output.
template <int DIR, typename T2> __device__ __forceinline__ void dft3_nomid(T2* v) {
  typedef typename Scal<T2>::t T;
  const T h = sqrt3_2<T>();
  T2 s = caddu(v[1], v[2]), d = csubu(v[1], v[2]);
  T2 mm;
  mm.x = addu(v[0].x, -half_of(s.x));
  mm.y = addu(v[0].y, -half_of(s.y));
  T2 r;
  if (DIR < 0) { r.x = mulu(h, d.y); r.y = -mulu(h, d.x); } else { r.x = -mulu(h, d.y); r.y = mulu(h, d.x); }
  v[0] = cadd(v[0], s);
  v[2] = csub(mm, r);
}

// In-place mixed-radix FFT stages of the double-float transforms (the FP64 and
// FP32 ones use the Cooley-Tukey stages further down, with the same slots).
// The inverse transforms (spectral -> physical) are decimation in frequency
// (DIF): natural-order input, digit-reversed output.  The forward transforms are decimation in time
// (DIT) with the radices in reverse order: digit-reversed input, natural
// output.  Physical-space data (the z rows of the mixed buffer, the x
// samples of the x-pass) therefore stay in digit-reversed order, which the
// pointwise products do not care about.  Every butterfly reads and writes the
// same R slots, so a stage needs one buffer and one barrier.
//
// The DIF plan starts with radix 3 and the DIT plan ends with it: with 3/2
// zero padding the middle third of a DIF input is zero (the first stage skips
// those loads and their additions) and the middle third of a DIT output is
// discarded by the truncation (the last stage does not form it).

// DIF stage of radix R on blocks of size Ls: butterfly j of block b reads
// x[b Ls + j + r m] (m = Ls/R), forms y_q = sum_r x_r w_R^(DIR r q), scales
// y_q by w_Ls^(DIR q j) and writes it back to slot q.  TW = false is the stage
// with m = 1 (every j is 0).  With m > 1 the butterflies with j = 0 multiply by
// tw[0] = 1 (exact) rather than branch: a warp holding one of them would run the
// twiddles for the others anyway, and the compiler predicates a short branch,
// which still takes issue slots.
template <int R, int DIR, bool ZMID, bool TW, typename T2>
__device__ __forceinline__ void dif_loop(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, int Ls,
                                         unsigned mag_nbf, unsigned mag_m) {
  const int m = Ls / R;
  const int nbf = L / R;
  const int tmul = L / Ls;
  const int total = nb * nbf;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = mag_nbf ? (int)__umulhi((unsigned)t, mag_nbf) : t;   // t / nbf (exact while t nbf < 2^32)
    const int u = t - bi * nbf;
    const int blk = TW ? (int)__umulhi((unsigned)u, mag_m) : u;   // u / m
    const int j = u - blk * m;
    T2* x = a + bi * ld + blk * Ls + j;
    T2 v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = (ZMID && q == 1) ? zero2<T2>() : x[q * m];
    if (R == 4) dft4<DIR>(v);
    else if (R == 2) dft2<DIR>(v);
    else if (ZMID) dft3_zmid<DIR>(v);
    else dft3<DIR>(v);
    if (TW) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        T2 w = tw[q * j * tmul];
        if (DIR > 0) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) x[q * m] = v[q];
  }
}
template <int R, int DIR, bool ZMID, typename T2>
__device__ __forceinline__ void dif_stage(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, int Ls,
                                          unsigned mag_nbf, unsigned mag_m) {
  if (mag_m) dif_loop<R, DIR, ZMID, true>(a, L, nb, ld, tw, Ls, mag_nbf, mag_m);   // mag 0: m = 1
  else dif_loop<R, DIR, ZMID, false>(a, L, nb, ld, tw, Ls, mag_nbf, mag_m);
  __syncthreads();
}

// DIT stage of radix R on blocks of size Ls: input r of butterfly j is scaled
// by w_Ls^(DIR r j), then y_q = sum_r x_r w_R^(DIR r q) goes to slot q.  With
// ZMID the middle output (q = 1) is neither formed nor stored.  TW as in the DIF
// stage.
template <int R, int DIR, bool ZMID, bool TW, typename T2>
__device__ __forceinline__ void dit_loop(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, int Ls,
                                         unsigned mag_nbf, unsigned mag_m) {
  const int m = Ls / R;
  const int nbf = L / R;
  const int tmul = L / Ls;
  const int total = nb * nbf;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = mag_nbf ? (int)__umulhi((unsigned)t, mag_nbf) : t;   // t / nbf (exact while t nbf < 2^32)
    const int u = t - bi * nbf;
    const int blk = TW ? (int)__umulhi((unsigned)u, mag_m) : u;   // u / m
    const int j = u - blk * m;
    T2* x = a + bi * ld + blk * Ls + j;
    T2 v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = x[q * m];
    if (TW) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        T2 w = tw[q * j * tmul];
        if (DIR > 0) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    if (R == 4) dft4<DIR>(v);
    else if (R == 2) dft2<DIR>(v);
    else if (ZMID) dft3_nomid<DIR>(v);
    else dft3<DIR>(v);
#pragma unroll
    for (int q = 0; q < R; ++q)
      if (!(ZMID && q == 1)) x[q * m] = v[q];
  }
}
template <int R, int DIR, bool ZMID, typename T2>
__device__ __forceinline__ void dit_stage(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, int Ls,
                                          unsigned mag_nbf, unsigned mag_m) {
  if (mag_m) dit_loop<R, DIR, ZMID, true>(a, L, nb, ld, tw, Ls, mag_nbf, mag_m);   // mag 0: m = 1
  else dit_loop<R, DIR, ZMID, false>(a, L, nb, ld, tw, Ls, mag_nbf, mag_m);
  __syncthreads();
}

// Inverse (DIR = +1) transform of nb sequences: natural in, digit-reversed out.
// pl.radix holds the DIF order (first radix 3); zmid: middle third of the input is zero.
template <int DIR, typename T2>
__device__ void fft_dif(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, const FftPlan& pl, bool zmid) {
  int Ls = L;
  for (int s = 0; s < pl.np; ++s) {
    const int R = pl.radix[s];
    const unsigned mn = pl.mag_nbf[s], mm = pl.mag_mdif[s];
    if (R == 4) dif_stage<4, DIR, false>(a, L, nb, ld, tw, Ls, mn, mm);
    else if (R == 2) dif_stage<2, DIR, false>(a, L, nb, ld, tw, Ls, mn, mm);
    else if (s == 0 && zmid) dif_stage<3, DIR, true>(a, L, nb, ld, tw, Ls, mn, mm);
    else dif_stage<3, DIR, false>(a, L, nb, ld, tw, Ls, mn, mm);
    Ls /= R;
  }
}

// Forward (DIR = -1) transform: digit-reversed in (as fft_dif left it), natural
// out.  Runs the DIF radices backwards; zmid: the middle third of the output is
// not needed.
template <int DIR, typename T2>
__device__ void fft_dit(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, const FftPlan& pl, bool zmid) {
  int Ls = 1;
  for (int s = pl.np - 1; s >= 0; --s) {
    const int R = pl.radix[s];
    Ls *= R;
    const unsigned mn = pl.mag_nbf[s], mm = pl.mag_mdit[s];
    if (R == 4) dit_stage<4, DIR, false>(a, L, nb, ld, tw, Ls, mn, mm);
    else if (R == 2) dit_stage<2, DIR, false>(a, L, nb, ld, tw, Ls, mn, mm);
    else if (s == 0 && zmid) dit_stage<3, DIR, true>(a, L, nb, ld, tw, Ls, mn, mm);
    else dit_stage<3, DIR, false>(a, L, nb, ld, tw, Ls, mn, mm);
  }
}

// Cooley-Tukey stages for FP64 and FP32: the twiddles scale the INPUTS of each
// butterfly, so every radix-2 step is a +- w b, and a - w b = 2a - (a + w b) takes
// the FMA form (six fused operations per radix-2 step instead of a complex multiply
// and four additions).  A twiddled radix-4 butterfly is two levels of such steps
// (24 FP64 operations instead of 28), a twiddled radix 3 shares one product between
// its sum and difference (18 instead of 20).  FP64 throughput is what bounds these
// transforms on this GPU, so the operation count is the time.
//
// The forward transforms (digit-reversed in, natural out) are the decimation-in-time
// stages above with these butterflies.  The inverse transforms keep natural input
// and digit-reversed output, with the same digit order as the DIF stages: stage s
// splits each block of size Ls (the residue of the spectrum modulo z^Ls - c) into R
// blocks of size m = Ls/R.  Input r of block b is scaled by w_L^(DIR r K m), where K
// is the digit reversal of b over the radices already applied (K = 0 for the single
// block of the first stage, which therefore has no twiddles); then the radix-R DFT.
// K m is read from a per-plan table built at set-up (FftPlan::revK).
// Double-float transforms keep the DIF / DIT stages: a pair product is not one fused
// operation, so the rewrite would save nothing there.

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// a <- a + w b, b <- a - w b
template <typename T2> __device__ __forceinline__ void ct2(T2& a, T2& b, T2 w) {
  typedef typename Scal<T2>::t T;
  T2 p;
  p.x = fmaT(w.x, b.x, fmaT(-w.y, b.y, a.x));
  p.y = fmaT(w.x, b.y, fmaT(w.y, b.x, a.y));
  b.x = fmaT(T(2), a.x, -p.x);
  b.y = fmaT(T(2), a.y, -p.y);
  a = p;
}
// y_q = sum_r v_r w^r i^(DIR r q), with w2 = w^2: (v0, v2) and (v1, v3) with w^2, then
// (e0, o0) with w and (e1, o1) with DIR i w.
template <int DIR, typename T2> __device__ __forceinline__ void ct4(T2* v, T2 w, T2 w2) {
  ct2(v[0], v[2], w2);
  ct2(v[1], v[3], w2);
  T2 wi;   // DIR i w
  if (DIR < 0) { wi.x = w.y; wi.y = -w.x; } else { wi.x = -w.y; wi.y = w.x; }
  ct2(v[0], v[1], w);    // y0, y2
  ct2(v[2], v[3], wi);   // y1, y3
  T2 t = v[1]; v[1] = v[2]; v[2] = t;
}
// y_q = sum_r v_r w^r w_3^(DIR r q): p = w v1, s = p + w^2 v2, d = p - w^2 v2 = 2p - s.
// NOMID: the middle output is not formed.
template <int DIR, bool NOMID, typename T2> __device__ __forceinline__ void ct3(T2* v, T2 w, T2 w2) {
  typedef typename Scal<T2>::t T;
  const T h = sqrt3_2<T>();
  T2 p, sm, d, mm;
  p.x = fmaT(w.x, v[1].x, -w.y * v[1].y);
  p.y = fmaT(w.x, v[1].y, w.y * v[1].x);
  sm.x = fmaT(w2.x, v[2].x, fmaT(-w2.y, v[2].y, p.x));
  sm.y = fmaT(w2.x, v[2].y, fmaT(w2.y, v[2].x, p.y));
  d.x = fmaT(T(2), p.x, -sm.x);
  d.y = fmaT(T(2), p.y, -sm.y);
  mm.x = fmaT(T(-0.5), sm.x, v[0].x);
  mm.y = fmaT(T(-0.5), sm.y, v[0].y);
  v[0].x += sm.x;
  v[0].y += sm.y;
  // y1 = mm + DIR i h d, y2 = mm - DIR i h d
  const T g = DIR < 0 ? h : -h;
  if (!NOMID) {
    v[1].x = fmaT(g, d.y, mm.x);
    v[1].y = fmaT(-g, d.x, mm.y);
  }
  v[2].x = fmaT(-g, d.y, mm.x);
  v[2].y = fmaT(g, d.x, mm.y);
}

// One Cooley-Tukey stage.  NR: inverse (block twiddles, block size Ls shrinking); else
// forward (twiddle of butterfly j is w_Ls^(DIR j)).  Z = 1: the middle input is zero
// (first inverse stage of a padded transform); Z = 2: the middle output is dropped
// (last forward stage before the truncation).  TW = false: every twiddle is 1.
// G (divides nb): a thread takes butterfly u of G rows (cg, cg + nb/G, ...), so its
// indices, swizzled slots and twiddles are formed once for the G of them; each butterfly's
// arithmetic is the same whatever G.
template <int R, int DIR, int Z, bool TW, bool NR, int G, typename T2>
__device__ __forceinline__ void ct_loop(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, int Ls,
                                        unsigned mag_nbf, unsigned mag_m, const FftPlan& pl, int s) {
  const int m = Ls / R;
  const int nbf = L / R;
  const int tmul = L / Ls;
  const int ng = G == 1 ? nb : nb / G;
  const int total = ng * nbf;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int cg = mag_nbf ? (int)__umulhi((unsigned)t, mag_nbf) : t;   // t / nbf (exact while t nbf < 2^32)
    const int u = t - cg * nbf;
    const int blk = mag_m ? (int)__umulhi((unsigned)u, mag_m) : u;      // u / m (mag 0: m = 1)
    const int j = u - blk * m;
    const int ib = blk * Ls + j;
    int o[R];
#pragma unroll
    for (int q = 0; q < R; ++q) o[q] = sw<T2>(ib + q * m);
    T2 w, w2;
    if (TW) {
      const int e = NR ? pl.revK[pl.revoff[s] + blk] : j * tmul;
      w = tw[e];
      w2 = R == 2 ? w : tw[2 * e];
      if (DIR > 0) { w.y = -w.y; w2.y = -w2.y; }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      T2* row = a + (cg + g * ng) * ld;
      T2 v[R];
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = (Z == 1 && q == 1) ? zero2<T2>() : row[o[q]];
      if (TW) {
        if (R == 4) ct4<DIR>(v, w, w2);
        else if (R == 2) ct2(v[0], v[1], w);
        else ct3<DIR, Z == 2>(v, w, w2);
      } else {
        if (R == 4) dft4<DIR>(v);
        else if (R == 2) dft2<DIR>(v);
        else if (Z == 1) dft3_zmid<DIR>(v);
        else if (Z == 2) dft3_nomid<DIR>(v);
        else dft3<DIR>(v);
      }
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (!(Z == 2 && q == 1)) row[o[q]] = v[q];
    }
  }
  __syncthreads();
}

// The Cooley-Tukey stages of a whole transform, G rows per butterfly item (see ct_loop).
// Inverse: natural in, digit-reversed out, block size shrinking; the first stage has one
// block (no twiddles) and, when zmid, a zero middle input.
template <int DIR, int G, typename T2>
__device__ __forceinline__ void ct_inv_stages(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, const FftPlan& pl,
                                              bool zmid) {
  int Ls = L;
  for (int s = 0; s < pl.np; ++s) {
    const int R = pl.radix[s];
    const unsigned mn = pl.mag_nbf[s], mm = pl.mag_mdif[s];
    if (s == 0) {   // one block, K = 0
      if (R == 4) ct_loop<4, DIR, 0, false, true, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else if (R == 2) ct_loop<2, DIR, 0, false, true, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else if (zmid) ct_loop<3, DIR, 1, false, true, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else ct_loop<3, DIR, 0, false, true, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
    } else {
      if (R == 4) ct_loop<4, DIR, 0, true, true, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else if (R == 2) ct_loop<2, DIR, 0, true, true, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else ct_loop<3, DIR, 0, true, true, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
    }
    Ls /= R;
  }
}
// Forward: digit-reversed in, natural out, the radices in reverse; when zmid the last
// stage does not form its middle output.
template <int DIR, int G, typename T2>
__device__ __forceinline__ void ct_fwd_stages(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, const FftPlan& pl,
                                              bool zmid) {
  int Ls = 1;
  for (int s = pl.np - 1; s >= 0; --s) {
    const int R = pl.radix[s];
    Ls *= R;
    const unsigned mn = pl.mag_nbf[s], mm = pl.mag_mdit[s];
    if (mm == 0) {   // m = 1: every twiddle is 1
      if (R == 4) ct_loop<4, DIR, 0, false, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else if (R == 2) ct_loop<2, DIR, 0, false, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else if (s == 0 && zmid) ct_loop<3, DIR, 2, false, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else ct_loop<3, DIR, 0, false, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
    } else {
      if (R == 4) ct_loop<4, DIR, 0, true, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else if (R == 2) ct_loop<2, DIR, 0, true, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else if (s == 0 && zmid) ct_loop<3, DIR, 2, true, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
      else ct_loop<3, DIR, 0, true, false, G>(a, L, nb, ld, tw, Ls, mn, mm, pl, s);
    }
  }
}

template <typename T2> struct IsPair { static constexpr bool v = false; };
template <> struct IsPair<dfc> { static constexpr bool v = true; };

// ---------------------------------------------------------------------------
// FP32 two-pass transforms.  For L = R1 R2 with both factors small (2^a 3^b <= 48), a
// transform is two sets of register-resident DFTs with one exchange through shared
// memory (Cooley-Tukey in "four-step" order, w_N = exp(2 pi i / N)):
//   inverse  x[R2 n1 + n2] = sum_k1 w_R1^(n1 k1) [ w_L^(n2 k1) sum_k2 X[k1 + R1 k2] w_R2^(n2 k2) ]
//   forward  X[k1 + R1 k2] = sum_n2 w_R2^(-n2 k2) [ w_L^(-n2 k1) sum_n1 x[R2 n1 + n2] w_R1^(-n1 k1) ]
// Every index inside a register DFT is a compile-time constant, and so is every twiddle
// (template arguments), so a DFT is straight-line arithmetic on registers; the stage
// transforms instead spend most of their instructions on shared-memory traffic and index
// arithmetic.  Slot s = c + R1 r of a row lives at element r (R1 + 1) + c (rows of R1
// padded by one, R1 even): the column sweeps (stride R1) and the row sweeps (unit
// stride) of a warp both fall in distinct banks.  In place: the inverse takes spectrum
// entry k from slot k and leaves sample x[R2 n1 + n2] in slot n1 + R1 n2; the forward
// reads that order and returns the spectrum to natural slots.  Each sweep reads and
// writes only its own slots, so one barrier separates the two.
// ---------------------------------------------------------------------------
constexpr double kPiD = 3.14159265358979323846264338327950288;
// sin and cos of 2 pi e / n (integers; e may be negative) by their Taylor series on the
// angle reduced to [-pi, pi]: evaluated by the compiler for the twiddles below.
__host__ __device__ constexpr double red_angle(int e, int n) {
  int r = ((e % n) + n) % n;
  if (2 * r > n) r -= n;
  return 2.0 * kPiD * r / n;
}
__host__ __device__ constexpr double taylor_sin(double x) {
  double t = x, sum = x;
  for (int i = 1; i < 30; ++i) { t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0)); sum += t; }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double t = 1.0, sum = 1.0;
  for (int i = 1; i < 30; ++i) { t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i)); sum += t; }
  return sum;
}

// In-place DFT of N registers, natural order in and out: y_k = sum_n v_n w_N^(DIR n k).
// Decimation in time by P = 4 (else 3, else 2): P interleaved DFTs of N / P, then
// N / P radix-P butterflies with twiddles w_N^(DIR p K).
template <int N, int DIR> struct RDft;
template <int DIR> struct RDft<1, DIR> { __device__ static __forceinline__ void run(float2*) {} };
template <int DIR> struct RDft<2, DIR> { __device__ static __forceinline__ void run(float2* v) { dft2<DIR>(v); } };
template <int DIR> struct RDft<3, DIR> { __device__ static __forceinline__ void run(float2* v) { dft3<DIR>(v); } };
template <int DIR> struct RDft<4, DIR> { __device__ static __forceinline__ void run(float2* v) { dft4<DIR>(v); } };
template <int N, int DIR> struct RDft {
  static constexpr int P = N % 4 == 0 ? 4 : (N % 3 == 0 ? 3 : 2);
  static constexpr int Q = N / P;
  static_assert(P * Q == N && Q > 1, "N must be 2^a 3^b");
  template <int p, int K>
  __device__ static __forceinline__ void twiddle(float2 (&t)[P], float2 (&s)[P][Q]) {
    if constexpr (p < P) {
      constexpr int q4 = (((4 * DIR * p * K) / N) % 4 + 4) % 4;   // the twiddle is i^q4 when exact
      if constexpr (K == 0 || p == 0) {
        t[p] = s[p][K];
      } else if constexpr ((4 * p * K) % N == 0) {
        const float2 x = s[p][K];
        t[p] = q4 == 0 ? x : (q4 == 1 ? make_float2(-x.y, x.x) : (q4 == 2 ? make_float2(-x.x, -x.y) : make_float2(x.y, -x.x)));
      } else {
        constexpr float c = (float)taylor_cos(red_angle(DIR * p * K, N));
        constexpr float sn = (float)taylor_sin(red_angle(DIR * p * K, N));
        const float2 x = s[p][K];
        t[p] = make_float2(fmaf(c, x.x, -sn * x.y), fmaf(c, x.y, sn * x.x));
      }
      twiddle<p + 1, K>(t, s);
    }
  }
  template <int K>
  __device__ static __forceinline__ void combine(float2* v, float2 (&s)[P][Q]) {
    if constexpr (K < Q) {
      float2 t[P];
      twiddle<0, K>(t, s);
      if constexpr (P == 4) dft4<DIR>(t);
      else if constexpr (P == 3) dft3<DIR>(t);
      else dft2<DIR>(t);
#pragma unroll
      for (int j = 0; j < P; ++j) v[K + Q * j] = t[j];
      combine<K + 1>(v, s);
    }
  }
  __device__ static __forceinline__ void run(float2* v) {
    float2 s[P][Q];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int q = 0; q < Q; ++q) s[p][q] = v[P * q + p];
#pragma unroll
    for (int p = 0; p < P; ++p) RDft<Q, DIR>::run(s[p]);
    combine<0>(v, s);
  }
};

// Inverse of nb rows at a + b ld: spectrum entries with index in [zlo, zhi] are zero (the
// 3/2 padding) and not read.  ts: the CTA's shared copy of the plan's twiddles, w_L^(-n2 k1)
// at [k1 (R2 + 1) + n2] (the padding keeps both sweeps' reads in distinct banks).
template <int R1, int R2>
__device__ __forceinline__ void fft2p_inv(float2* a, int nb, int ld, const float2* ts, int zlo, int zhi) {
  constexpr int RS = R1 + 1;
  for (int it = threadIdx.x; it < nb * R1; it += blockDim.x) {
    const int b = it / R1, k1 = it - b * R1;
    float2* col = a + b * ld + k1;
    float2 v[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int k = k1 + R1 * k2;
      v[k2] = (k >= zlo && k <= zhi) ? make_float2(0.f, 0.f) : col[k2 * RS];
    }
    RDft<R2, +1>::run(v);
#pragma unroll
    for (int n2 = 1; n2 < R2; ++n2) {   // times w_L^(n2 k1), the conjugate of the table's entry
      const float2 w = ts[k1 * (R2 + 1) + n2];
      v[n2] = make_float2(fmaf(w.x, v[n2].x, w.y * v[n2].y), fmaf(w.x, v[n2].y, -w.y * v[n2].x));
    }
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) col[n2 * RS] = v[n2];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nb * R2; it += blockDim.x) {
    const int b = it / R2, n2 = it - b * R2;
    float2* row = a + b * ld + n2 * RS;
    float2 v[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = row[k1];
    RDft<R1, +1>::run(v);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) row[n1] = v[n1];
  }
  __syncthreads();
}

// Forward of nb rows in the inverse's output order; spectrum entries with index in
// [zlo, zhi] are not stored (the 3/2 truncation).
template <int R1, int R2>
__device__ __forceinline__ void fft2p_fwd(float2* a, int nb, int ld, const float2* ts, int zlo, int zhi) {
  constexpr int RS = R1 + 1;
  for (int it = threadIdx.x; it < nb * R2; it += blockDim.x) {
    const int b = it / R2, n2 = it - b * R2;
    float2* row = a + b * ld + n2 * RS;
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = row[n1];
    RDft<R1, -1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {   // times w_L^(-n2 k1)
      const float2 w = ts[k1 * (R2 + 1) + n2];
      v[k1] = make_float2(fmaf(w.x, v[k1].x, -w.y * v[k1].y), fmaf(w.x, v[k1].y, w.y * v[k1].x));
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) row[k1] = v[k1];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nb * R1; it += blockDim.x) {
    const int b = it / R1, k1 = it - b * R1;
    float2* col = a + b * ld + k1;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = col[n2 * RS];
    RDft<R2, -1>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int k = k1 + R1 * k2;
      if (!(k >= zlo && k <= zhi)) col[k2 * RS] = v[k2];
    }
  }
  __syncthreads();
}

// The splits the FP32 path runs as two passes (R1 even; the host's fft_split lists the
// same pairs).  Returns false for other lengths.
#define CHAN_FFT2P_SPLITS(X) \
  X(4, 3) X(6, 3) X(6, 4) X(6, 6) X(8, 6) X(6, 9) X(8, 9) X(8, 12) X(12, 12) X(16, 12) X(16, 18) X(16, 24) \
  X(24, 24) X(32, 24) X(32, 36) X(32, 48) X(48, 36) X(48, 48)

// Register-size category of a split: 1 (factors <= 16), 2 (<= 24), 3 (<= 48).  A kernel
// instance of category c holds the splits of categories 1 .. c, so its register allocation
// follows the largest register transform it may run.
__host__ __device__ constexpr int fft2p_cat(int a, int b) {
  return (a > b ? a : b) <= 16 ? 1 : ((a > b ? a : b) <= 24 ? 2 : 3);
}

template <int DIR, int CAT>
__device__ __forceinline__ bool fft2p(float2* a, int nb, int ld, const float2* ts, const FftPlan& pl, bool zmid) {
  const int L = pl.L, zlo = zmid ? L / 3 : 1, zhi = zmid ? 2 * L / 3 : 0;
#define CHAN_FFT2P_CASE(A, B)                                              \
  if constexpr (fft2p_cat(A, B) <= CAT) {                                  \
    if (pl.r1 == A && pl.r2 == B) {                                        \
      if (DIR > 0) fft2p_inv<A, B>(a, nb, ld, ts, zlo, zhi);               \
      else fft2p_fwd<A, B>(a, nb, ld, ts, zlo, zhi);                       \
      return true;                                                         \
    }                                                                      \
  }
  CHAN_FFT2P_SPLITS(CHAN_FFT2P_CASE)
#undef CHAN_FFT2P_CASE
  return false;
}

// A CTA's shared copy of the two-pass twiddles, placed at `end` (after its rows); null when
// the stage transforms run.  Read only after the CTA's next barrier.
template <typename T2>
__device__ __forceinline__ const float2* stage_tw2p(T2* end, const FftPlan& pl) {
  if constexpr (std::is_same<T2, float2>::value) {
    if (pl.r1) {
      const int n = pl.r1 * (pl.r2 + 1);
      for (int i = threadIdx.x; i < n; i += blockDim.x) end[i] = pl.tw2p[i];
      return end;
    }
  }
  return nullptr;
}

// Slot of element i of a transform row: the two-pass padded layout, the FP32 swizzle of
// the stage transforms, or i.
template <typename T2>
__device__ __forceinline__ int slot(int i, const FftPlan& pl) {
  if constexpr (std::is_same<T2, float2>::value) {
    if (pl.r1) return i + (int)__umulhi((unsigned)i, pl.mag_r1);
  }
  return sw<T2>(i);
}

// Inverse transform (spectral -> physical) of nb sequences: natural in, digit-reversed out.
// zmid: the middle third of the input is zero (3/2 padding).
template <int DIR, int CAT, typename T2>
__device__ void fft_inv(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, const FftPlan& pl, bool zmid,
                        const float2* ts) {
  if constexpr (std::is_same<T2, float2>::value && CAT > 0) {
    if (pl.r1 && fft2p<DIR, CAT>(a, nb, ld, ts, pl, zmid)) return;
  }
  if constexpr (IsPair<T2>::v) {
    fft_dif<DIR>(a, L, nb, ld, tw, pl, zmid);
  } else {
    // FP32 rows in even numbers: two rows per butterfly item (ct_loop G); FP64 is bound by
    // its FP64 arithmetic, not by the index work G shares
    if constexpr (std::is_same<T2, float2>::value) {
      if ((nb & 1) == 0) { ct_inv_stages<DIR, 2>(a, L, nb, ld, tw, pl, zmid); return; }
    }
    ct_inv_stages<DIR, 1>(a, L, nb, ld, tw, pl, zmid);
  }
}

// Forward transform (physical -> spectral): digit-reversed in (as fft_inv leaves it),
// natural out.  zmid: the middle third of the output is not needed (3/2 truncation).
template <int DIR, int CAT, typename T2>
__device__ void fft_fwd(T2* a, int L, int nb, int ld, const T2* CHAN_RO tw, const FftPlan& pl, bool zmid,
                        const float2* ts) {
  if constexpr (std::is_same<T2, float2>::value && CAT > 0) {
    if (pl.r1 && fft2p<DIR, CAT>(a, nb, ld, ts, pl, zmid)) return;
  }
  if constexpr (IsPair<T2>::v) {
    fft_dit<DIR>(a, L, nb, ld, tw, pl, zmid);
  } else {
    if constexpr (std::is_same<T2, float2>::value) {
      if ((nb & 1) == 0) { ct_fwd_stages<DIR, 2>(a, L, nb, ld, tw, pl, zmid); return; }
    }
    ct_fwd_stages<DIR, 1>(a, L, nb, ld, tw, pl, zmid);
  }
}

struct ZArgs {
  const double2* in[CHAN_MAXFIELDS];
  double2* outd[CHAN_MAXFIELDS];
  void* out[CHAN_MAXFIELDS];
  int applyG[CHAN_MAXFIELDS];
  const double* G;
  int Ny, Nz, nxh, M, L3, KB, ld;
  int lgKB;       // KB = 2^lgKB columns per CTA
  int pair_out;   // double-float mode: the forward pass writes (hi, lo) pairs
  int f32_mask;   // inverse pass: bit f set = field f is stored as float2 (mixed modes)
  int pair_in;    // FP32 transforms of Fourier fields stored as pairs (mixed mode with pair sweeps)
  int skip00;     // inverse pass: the (0,0) mode (the plane mean) is taken as zero
  FftPlan pl;
};

// FP32 column elements copied global -> shared without a register round trip (cp.async,
// 8 bytes each, zero-filled when !valid): all of a thread's copies of a column chunk are in
// flight at once.  The thread waits for its own copies (zc_wait) before the block barrier.
__device__ __forceinline__ void zc8(void* s, const void* g, bool valid = true) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void zc_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Inverse z-pass: Fourier [Ny][Nz][nxh] (double) -> mixed [Ny][L3][nxh] (T),
// kz zero-padded to 3Nz/2 (the kz Nyquist row is dropped), optional filter
// transfer G applied on load.
// Load a column chunk of one Fourier field into the padded transform buffer.  KIND 0: stored
// as the state is stored; 1: times the filter transfer G; 2: stored as float2 (mixed modes);
// 3, 4: stored as pairs, FP32 transforms (as 0, 1).
template <typename T2, int KIND>
__device__ __forceinline__ void zinv_load(const ZArgs& A, T2* a, const double2* in, const float2* in32, int kx0, int hz) {
  if constexpr (std::is_same<T2, float2>::value && KIND != 2) {
    // FP32 transforms of FP64 or pair-stored fields: the rounding to FP32 needs the value in
    // registers, so ZB elements' loads are issued before any is converted and stored
    constexpr int ZB = 4;
    for (int e0 = threadIdx.x; e0 < A.Nz * A.KB; e0 += ZB * blockDim.x) {
      float2 v[ZB];
      int dst[ZB];
#pragma unroll
      for (int b = 0; b < ZB; ++b) {
        const int e = e0 + b * blockDim.x;
        dst[b] = -1;
        if (e >= A.Nz * A.KB) continue;
        const int jz = e >> A.lgKB, kl = e & (A.KB - 1), kx = kx0 + kl;
        if (kx >= A.nxh || jz == hz) continue;
        const int q = jz * A.nxh + kx;
        const int pz = jz < hz ? jz : jz + (A.L3 - A.Nz);
        if constexpr (KIND >= 3) v[b] = ld_pair_f32(in, q, KIND == 4, KIND == 4 ? A.G[q] : 0.0);
        else v[b] = ld_fourier<T2>(in, q, KIND == 1, KIND == 1 ? A.G[q] : 0.0);
        dst[b] = kl * A.ld + slot<T2>(pz, A.pl);
      }
#pragma unroll
      for (int b = 0; b < ZB; ++b)
        if (dst[b] >= 0) a[dst[b]] = v[b];
    }
    return;
  }
  for (int e = threadIdx.x; e < A.Nz * A.KB; e += blockDim.x) {
    const int jz = e >> A.lgKB, kl = e & (A.KB - 1), kx = kx0 + kl;
    if (kx >= A.nxh || jz == hz) continue;
    const int q = jz * A.nxh + kx;
    const int pz = jz < hz ? jz : jz + (A.L3 - A.Nz);
    if constexpr (KIND == 2) {
      if constexpr (std::is_same<T2, float2>::value) zc8(&a[kl * A.ld + slot<T2>(pz, A.pl)], &in32[q]);
    } else if constexpr (KIND >= 3) {
      if constexpr (std::is_same<T2, float2>::value)
        a[kl * A.ld + slot<T2>(pz, A.pl)] = ld_pair_f32(in, q, KIND == 4, KIND == 4 ? A.G[q] : 0.0);
    } else {
      a[kl * A.ld + slot<T2>(pz, A.pl)] = ld_fourier<T2>(in, q, KIND == 1, KIND == 1 ? A.G[q] : 0.0);
    }
  }
}

template <typename T, int CAT>
__device__ __forceinline__ void zinv_body(const ZArgs& A, const typename V2<T>::t* CHAN_RO tw, int bx, int by,
                                          int bz) {
  typedef typename V2<T>::t T2;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* a = reinterpret_cast<T2*>(smraw);
  const int f = bz, y = by, kx0 = bx * A.KB;
  const int hz = A.Nz / 2;
  // The first stage skips the middle third of each padded column, and the load below
  // writes every other slot except the dropped kz Nyquist row at 2 L3/3: only that one
  // is zeroed (no conflict with the loads, so no barrier in between).
  for (int kl = threadIdx.x; kl < A.KB; kl += blockDim.x) a[kl * A.ld + slot<T2>(A.L3 - hz, A.pl)] = zero2<T2>();
  const bool f32 = (A.f32_mask >> f) & 1;
  const double2* in = A.in[f] + (size_t)y * A.M;
  const float2* in32 = reinterpret_cast<const float2*>(A.in[f]) + (size_t)y * A.M;
  // one loop per input kind, so that no branch of another kind is issued (predicated) per element
  if (f32) zinv_load<T2, 2>(A, a, in, in32, kx0, hz);   // (float2 inputs are never filtered)
  else if (A.pair_in) {
    if (A.applyG[f]) zinv_load<T2, 4>(A, a, in, in32, kx0, hz);
    else zinv_load<T2, 3>(A, a, in, in32, kx0, hz);
  } else if (A.applyG[f]) zinv_load<T2, 1>(A, a, in, in32, kx0, hz);
  else zinv_load<T2, 0>(A, a, in, in32, kx0, hz);
  if constexpr (std::is_same<T2, float2>::value) zc_wait();
  // the (0,0) mode is element 0 of the first column chunk, loaded by thread 0 above
  if (A.skip00 && bx == 0 && threadIdx.x == 0) a[slot<T2>(0, A.pl)] = zero2<T2>();
  const float2* ts = stage_tw2p<T2>(a + A.KB * A.ld, A.pl);
  __syncthreads();
  // the middle third of the padded column is zero: pruned first stage
  fft_inv<+1, CAT>(a, A.L3, A.KB, A.ld, tw, A.pl, true, ts);
  // physical rows leave in digit-reversed z order (slot = position in the column)
  T2* out = reinterpret_cast<T2*>(A.out[f]) + (size_t)y * A.L3 * A.nxh;
  for (int e = threadIdx.x; e < A.L3 * A.KB; e += blockDim.x) {
    const int z = e >> A.lgKB, kl = e & (A.KB - 1), kx = kx0 + kl;
    if (kx < A.nxh) out[z * A.nxh + kx] = a[kl * A.ld + slot<T2>(z, A.pl)];   // 32-bit index within the plane
  }
}

// Forward z-pass: mixed (T) -> Fourier (double), truncation to the stored kz.
template <typename T2, int PAIR>
__device__ __forceinline__ void zfwd_store(const ZArgs& A, const T2* r, double2* out, int kx0, int hz) {
  for (int e = threadIdx.x; e < A.Nz * A.KB; e += blockDim.x) {
    const int jz = e >> A.lgKB, kl = e & (A.KB - 1), kx = kx0 + kl;
    if (kx >= A.nxh) continue;
    if (jz != hz) {
      const int pz = jz < hz ? jz : jz + (A.L3 - A.Nz);
      st_fourier<T2>(out, jz * A.nxh + kx, r[kl * A.ld + slot<T2>(pz, A.pl)], PAIR);
    } else {
      out[jz * A.nxh + kx] = make_double2(0.0, 0.0);
    }
  }
}

template <typename T, int CAT>
__device__ __forceinline__ void zfwd_body(const ZArgs& A, const typename V2<T>::t* CHAN_RO tw, int bx, int by,
                                          int bz) {
  typedef typename V2<T>::t T2;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* a = reinterpret_cast<T2*>(smraw);
  const int f = bz, y = by, kx0 = bx * A.KB;
  const int hz = A.Nz / 2;
  const T2* in = reinterpret_cast<const T2*>(A.out[f]) + (size_t)y * A.L3 * A.nxh;
  for (int e = threadIdx.x; e < A.L3 * A.KB; e += blockDim.x) {
    const int z = e >> A.lgKB, kl = e & (A.KB - 1), kx = kx0 + kl;
    if constexpr (std::is_same<T2, float2>::value)
      zc8(&a[kl * A.ld + slot<T2>(z, A.pl)], &in[z * A.nxh + (kx < A.nxh ? kx : 0)], kx < A.nxh);
    else
      a[kl * A.ld + slot<T2>(z, A.pl)] = kx < A.nxh ? in[z * A.nxh + kx] : zero2<T2>();
  }
  if constexpr (std::is_same<T2, float2>::value) zc_wait();
  const float2* ts = stage_tw2p<T2>(a + A.KB * A.ld, A.pl);
  __syncthreads();
  // digit-reversed rows in, natural kz out; the middle third (truncated) is not formed
  fft_fwd<-1, CAT>(a, A.L3, A.KB, A.ld, tw, A.pl, true, ts);
  double2* out = A.outd[f] + (size_t)y * A.M;
  if (A.pair_out) zfwd_store<T2, 1>(A, a, out, kx0, hz);   // one store loop per output form
  else zfwd_store<T2, 0>(A, a, out, kx0, hz);
}

struct XArgs {
  void* in[CHAN_MAXFIELDS];
  void* out[CHAN_MAXFIELDS];
  int nxh, L1, L3, ld;
  double scale;  // 1 / (L1 L3): analysis normalisation of the padded grid
  unsigned mag_nxh;  // ceil(2^32 / nxh) for nxh >= 2 (exact below e nxh < 2^32), 0 for nxh = 1
  FftPlan pl;
};

// x-pass on the physical z-rows (z0, z0+1) of plane y.  MODE 0: inputs
// (u1, u2, u3, w1, w2, w3) -> H = u x omega (3 outputs).  MODE 1: inputs
// (u1, u2, u3) -> the six products u_i u_j (11, 22, 33, 12, 13, 23).
// MODE 2: inputs (w1, w2, w3) -> w_i w_i (1 output).
template <typename T, int MODE, int CAT>
__device__ __forceinline__ void xpass_body(const XArgs& A, const typename V2<T>::t* CHAN_RO tw, int bx, int by) {
  typedef typename V2<T>::t T2;
  constexpr int NIN = MODE == 0 ? 6 : 3;
  constexpr int NOUT = MODE == 0 ? 3 : (MODE == 1 ? 6 : 1);
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* a = reinterpret_cast<T2*>(smraw);
  const int z0 = 2 * bx, y = by;
  const int L1 = A.L1, nxh = A.nxh, ld = A.ld;
  const size_t rowoff = ((size_t)y * A.L3 + z0) * nxh;   // rows z0, z0 + 1 of plane y
  // The first stage skips the middle third [nxh, 2 nxh) and the packing below writes every
  // other slot except the dropped kx Nyquist slot 2 nxh: only that one is zeroed.
  for (int f = threadIdx.x; f < NIN; f += blockDim.x) a[f * ld + slot<T2>(2 * nxh, A.pl)] = zero2<T2>();
  // pack rows z0 (real part) and z0+1 (imaginary part) with Hermitian extension in kx
  auto pack = [&](int f, int k, T2 P, T2 Q) {
    T2* dstf = a + f * ld;
    if (k == 0) {
      T2 c0;
      c0.x = P.x;
      c0.y = Q.x;
      dstf[slot<T2>(0, A.pl)] = c0;
    } else {
      T2 c1, c2;
      c1.x = P.x - Q.y; c1.y = P.y + Q.x;      // P_k + i Q_k
      c2.x = P.x + Q.y; c2.y = -P.y + Q.x;     // conj(P_k) + i conj(Q_k) at -k
      dstf[slot<T2>(k, A.pl)] = c1;
      dstf[slot<T2>(L1 - k, A.pl)] = c2;
    }
  };
  if constexpr (std::is_same<T2, float2>::value) {
    // FP32 (bound by waiting on these loads): XB elements' loads issued before any is packed
    constexpr int XB = 4;
    for (int e0 = threadIdx.x; e0 < NIN * nxh; e0 += XB * blockDim.x) {
      T2 P[XB], Q[XB];
      int fk[XB];
#pragma unroll
      for (int b = 0; b < XB; ++b) {
        const int e = e0 + b * blockDim.x;
        fk[b] = -1;
        if (e < NIN * nxh) {
          const int f = A.mag_nxh ? (int)__umulhi((unsigned)e, A.mag_nxh) : e, k = e - f * nxh;   // e / nxh
          const T2* row = reinterpret_cast<const T2*>(A.in[f]) + rowoff;
          P[b] = row[k];
          Q[b] = row[nxh + k];
          fk[b] = f * nxh + k;
        }
      }
#pragma unroll
      for (int b = 0; b < XB; ++b)
        if (fk[b] >= 0) {
          const int f = A.mag_nxh ? (int)__umulhi((unsigned)fk[b], A.mag_nxh) : fk[b];
          pack(f, fk[b] - f * nxh, P[b], Q[b]);
        }
    }
  } else {
    for (int e = threadIdx.x; e < NIN * nxh; e += blockDim.x) {
      const int f = A.mag_nxh ? (int)__umulhi((unsigned)e, A.mag_nxh) : e, k = e - f * nxh;   // e / nxh
      const T2* row = reinterpret_cast<const T2*>(A.in[f]) + rowoff;
      pack(f, k, row[k], row[nxh + k]);
    }
  }
  const float2* ts = stage_tw2p<T2>(a + 6 * ld, A.pl);
  __syncthreads();
  // kx in [nxh, 2 nxh] is zero padding: pruned first stage; x samples leave digit-reversed
  fft_inv<+1, CAT>(a, L1, NIN, ld, tw, A.pl, true, ts);
  T2* r = a;
  T2* o = a;   // products overwrite their own sample slot (all fields share the order)
  for (int x = threadIdx.x; x < L1; x += blockDim.x) {
    T2 q[NIN];
    const int xs = slot<T2>(x, A.pl);
#pragma unroll
    for (int f = 0; f < NIN; ++f) q[f] = r[f * ld + xs];
    if (MODE == 0) {
      // H1 = u2 w3 - u3 w2, H2 = u3 w1 - u1 w3, H3 = u1 w2 - u2 w1 (both rows at once)
      T2 h1, h2, h3;
      h1.x = mulu(q[1].x, q[5].x) - mulu(q[2].x, q[4].x); h1.y = mulu(q[1].y, q[5].y) - mulu(q[2].y, q[4].y);
      h2.x = mulu(q[2].x, q[3].x) - mulu(q[0].x, q[5].x); h2.y = mulu(q[2].y, q[3].y) - mulu(q[0].y, q[5].y);
      h3.x = mulu(q[0].x, q[4].x) - mulu(q[1].x, q[3].x); h3.y = mulu(q[0].y, q[4].y) - mulu(q[1].y, q[3].y);
      o[0 * ld + xs] = h1;
      o[1 * ld + xs] = h2;
      o[2 * ld + xs] = h3;
    } else if (MODE == 2) {
      T2 w;
      w.x = q[0].x * q[0].x + q[1].x * q[1].x + q[2].x * q[2].x;
      w.y = q[0].y * q[0].y + q[1].y * q[1].y + q[2].y * q[2].y;
      o[xs] = w;
    } else {
      const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        T2 w;
        w.x = q[pi[p]].x * q[pj[p]].x;
        w.y = q[pi[p]].y * q[pj[p]].y;
        o[p * ld + xs] = w;
      }
    }
  }
  __syncthreads();
  // back to natural kx order; the middle third of the spectrum is discarded, so not formed
  fft_fwd<-1, CAT>(a, L1, NOUT, ld, tw, A.pl, true, ts);
  const T2* s = a;
  const T half = from_d<T>(0.5 * A.scale);
  for (int e = threadIdx.x; e < NOUT * nxh; e += blockDim.x) {
    const int gq = A.mag_nxh ? (int)__umulhi((unsigned)e, A.mag_nxh) : e, k = e - gq * nxh;   // e / nxh
    const T2 c = s[gq * ld + slot<T2>(k, A.pl)];
    const T2 cm = s[gq * ld + slot<T2>(k == 0 ? 0 : L1 - k, A.pl)];
    T2 F, G;
    F.x = half * (c.x + cm.x); F.y = half * (c.y - cm.y);      // (C_k + conj C_-k) / 2
    G.x = half * (c.y + cm.y); G.y = -half * (c.x - cm.x);     // (C_k - conj C_-k) / 2i
    T2* row = reinterpret_cast<T2*>(A.out[gq]) + rowoff;
    row[k] = F;
    row[nxh + k] = G;
  }
}

// ---------------------------------------------------------------------------
// Host helpers: the arguments of a run's transform passes
// ---------------------------------------------------------------------------
// Register-transform category of a plan's FP32 two-pass split (0: the stage transforms).
static int plan_cat(const FftPlan& pl) { return pl.r1 ? fft2p_cat(pl.r1, pl.r2) : 0; }
// Shared bytes of a CTA's copy of the two-pass twiddles.
static size_t tw2p_bytes(const FftPlan& pl) { return pl.r1 ? (size_t)pl.r1 * (pl.r2 + 1) * sizeof(float2) : 0; }

static ZArgs zargs(chan_s* h, size_t es) {
  ZArgs A;
  memset(&A, 0, sizeof(A));
  A.Ny = h->Ny; A.Nz = h->Nz; A.nxh = h->nxh; A.M = h->M; A.L3 = h->L3;
  A.KB = h->kb_z > 0 ? h->kb_z : pick_kb(h->nxh, h->L3, es);
  A.lgKB = 0;
  while ((1 << A.lgKB) < A.KB) ++A.lgKB;
  A.ld = fft_ld(h->L3, es);
  A.pl = h->p3;
  A.G = h->G;
  A.pair_in = h->prec == CHAN_PREC_MIXED_DF;
  return A;
}

static size_t fft_esize(const chan_s* h) { return prec_t32(h->prec) ? sizeof(float2) : sizeof(double2); }

}  // namespace
