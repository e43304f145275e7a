// Wall-normal (y) kernels of the channel substep: one thread per Fourier
// mode sweeps its y-pencil through (3,3)-banded compact operators.  The
// Fourier layout [Ny][M] puts consecutive modes at consecutive addresses,
// so each sweep step is a coalesced row load/store across a warp.
//
// Appendix A of arXiv:1808.06461: u_1, u_3 from continuity and omega_2;
// N_chi, N_omega2 of Eq. (hghv); the semi-implicit RK3 steps (chi1), (psi);
// the Poisson problem (chi2) with the influence-matrix wall correction; the
// mean profiles with a constant mass flux (Sec. 2.1).
#include <cstdint>

#include "chan_internal.cuh"
#include "df.cuh"
#include "y_bodies.cuh"

namespace {

__global__ void __launch_bounds__(128) k_pre(Geo g, YTabs t, const double2* __restrict__ v,
                                             const double2* __restrict__ om, const double2* __restrict__ dv,
                                             const double* __restrict__ U1, const double* __restrict__ U3,
                                             double2* u1o, double2* u3o, double2* om1o, double2* om3o) { pre_body<YF64>(g, t, v, om, dv, U1, U3, u1o, u3o, om1o, om3o, blockIdx.x); }
__global__ void __launch_bounds__(128) k_pre_f32(Geo g, YTabs t, const double2* __restrict__ v,
                                                 const double2* __restrict__ om, const double2* __restrict__ dv,
                                                 const double* __restrict__ U1, const double* __restrict__ U3,
                                                 double2* u1o, double2* u3o, double2* om1o, double2* om3o) { pre_body<YF64, true>(g, t, v, om, dv, U1, U3, u1o, u3o, om1o, om3o, blockIdx.x); }
__global__ void __launch_bounds__(128) k_pre_df(Geo g, YTabs t, const double2* __restrict__ v,
                                                const double2* __restrict__ om, const double2* __restrict__ dv,
                                                const double* __restrict__ U1, const double* __restrict__ U3,
                                                double2* u1o, double2* u3o, double2* om1o, double2* om3o) { pre_body<YDF>(g, t, v, om, dv, U1, U3, u1o, u3o, om1o, om3o, blockIdx.x); }
__global__ void __launch_bounds__(128) k_pre_df_f32(Geo g, YTabs t, const double2* __restrict__ v,
                                                    const double2* __restrict__ om, const double2* __restrict__ dv,
                                                    const double* __restrict__ U1, const double* __restrict__ U3,
                                                    double2* u1o, double2* u3o, double2* om1o, double2* om3o) { pre_body<YDF, true>(g, t, v, om, dv, U1, U3, u1o, u3o, om1o, om3o, blockIdx.x); }


__global__ void __launch_bounds__(128) k_nonlin(Geo g, YTabs t, const double2* __restrict__ H1,
                                                const double2* __restrict__ H2, const double2* __restrict__ H3,
                                                double2* Nchi, double2* Nom, double2* scr) { nonlin_body<YF64>(g, t, H1, H2, H3, Nchi, Nom, scr, blockIdx.x); }
__global__ void __launch_bounds__(128) k_nonlin_df(Geo g, YTabs t, const double2* __restrict__ H1,
                                                   const double2* __restrict__ H2, const double2* __restrict__ H3,
                                                   double2* Nchi, double2* Nom, double2* scr) { nonlin_body<YDF>(g, t, H1, H2, H3, Nchi, Nom, scr, blockIdx.x); }


// One thread per (mode, field): blockIdx.y = 0 omega_2, 1 chi.
template <class Y>
__global__ void __launch_bounds__(128) k_helm(Geo g, YTabs t, const typename Y::R* __restrict__ helm,
                                              double2* om, double2* chi, const double2* __restrict__ Nchi,
                                              const double2* __restrict__ Nom, double2* Nchi_p, double2* Nom_p,
                                              double2* Rom, double2* Rchi, const double* __restrict__ scal,
                                              double2* scr, int s) {
  if (blockIdx.y == 0) helm_body<Y, 0>(g, t, helm, om, chi, Nchi, Nom, Nchi_p, Nom_p, Rom, Rchi, scal, scr, s, blockIdx.x);
  else helm_body<Y, 1>(g, t, helm, om, chi, Nchi, Nom, Nchi_p, Nom_p, Rom, Rchi, scal, scr, s, blockIdx.x);
}



template <class Y>
__global__ void __launch_bounds__(128) k_poisson(Geo g, YTabs t, const typename Y::R* __restrict__ helm,
                                                 const typename Y::R* __restrict__ pois,
                                                 const typename Y::R* __restrict__ infl, double2* v, double2* chi,
                                                 double2* dv, double2* scr, double* scal, int s) {
  poisson_body<Y>(g, t, helm, pois, infl, v, chi, dv, scr, scal, s, blockIdx.x);
}



__global__ void __launch_bounds__(256) k_mean(Geo g, YTabs t, const double* __restrict__ helm,
                                              const double* __restrict__ meanh, const double2* __restrict__ H1,
                                              const double2* __restrict__ H3, double* U1, double* U3, double* H1p,
                                              double* H3p, double* scal, int s) { mean_body(g, t, helm, meanh, H1, H3, U1, U3, H1p, H3p, scal, s, blockIdx.x); }

// Tables in the work slots: the mean-flow solve runs beside the kernels that overwrite
// those slots, so it reads compact copies of what it needs from them.
// dst[i] = src[i * stride], i < n (the (0,0) class of a Helmholtz table slot).
__global__ void k_gather_class0(const double* __restrict__ src, size_t stride, int n, double* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[(size_t)i * stride];
}
// dst[y] = H1[y M], dst[Ny + y] = H3[y M]: the (0,0) modes of H_1, H_3 on every plane.
__global__ void k_copy_mean_modes(const double2* __restrict__ H1, const double2* __restrict__ H3, size_t M, int Ny,
                                  double2* dst) {
  for (int i = threadIdx.x; i < Ny; i += blockDim.x) {
    dst[i] = H1[(size_t)i * M];
    dst[Ny + i] = H3[(size_t)i * M];
  }
}


// U_h(s) = (A - b_s dt nu B)^-1 A 1 with zero wall values, and its trapezoid flux, from the
// substep's Helmholtz factors (helm at its slot) into out[Ny + 1].
__global__ void k_setup_mean(Geo g, YTabs t, const double* __restrict__ helm, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int Ny = g.Ny;
  const size_t C = g.C;
  const double* H = helm;
  double h[3] = {0, 0, 0};
  for (int i = 0; i < Ny; ++i) {
    double r = 0.0;
    if (i > 0 && i < Ny - 1)
      for (int d = 0; d < 7; ++d) {
        const int j = i - 3 + d;
        if (j >= 0 && j < Ny) r += t.A2[7 * i + d];
      }
    const double* Hi = H + (size_t)i * 11 * C;
    r -= Hi[0] * h[0] + Hi[C] * h[1] + Hi[2 * C] * h[2];
    h[0] = h[1]; h[1] = h[2]; h[2] = r;
    out[i] = r;
  }
  double nx[3] = {0, 0, 0}, q = 0.0;
  for (int i = Ny - 1; i >= 0; --i) {
    const double* Hi = H + (size_t)i * 11 * C;
    double x = (out[i] - Hi[3 * C] * nx[0] - Hi[4 * C] * nx[1] - Hi[5 * C] * nx[2]) * Hi[6 * C];
    nx[2] = nx[1]; nx[1] = nx[0]; nx[0] = x;
    out[i] = x;
  }
  for (int i = 0; i < Ny; ++i) q += t.wq[i] * out[i];
  out[Ny] = q;
}

// ---------------------------------------------------------------------------
// State derivation after a set_state: chi = A2^-1 (B2 - k^2 A2) v over all
// rows, and dv/dy = D1 v.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_derive(Geo g, YTabs t, const double2* __restrict__ v, double2* chi,
                                                double2* dv, double2* scr) {
  extern __shared__ double sm[];
  const int Ny = g.Ny;
  double* sA = sm;
  double* sB = sm + 7 * Ny;
  double* sB1 = sm + 14 * Ny;
  double* sLU1 = sm + 21 * Ny;
  double* sLU2 = sm + 28 * Ny;
  load_tab(sA, t.A2, 7 * Ny);
  load_tab(sB, t.B2, 7 * Ny);
  load_tab(sB1, t.B1, 7 * Ny);
  load_tab(sLU1, t.lu1, 7 * Ny);
  load_tab(sLU2, t.lu2f, 7 * Ny);
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.M) return;
  const size_t M = g.M;
  ModeInfo mi = mode_info(g, m);
  double2 w[7], h2[3], h1[3];
#pragma unroll
  for (int d = 0; d < 7; ++d) w[d] = z2();
#pragma unroll
  for (int d = 0; d < 3; ++d) { h2[d] = z2(); h1[d] = z2(); }
  double2* scr2 = scr + (size_t)Ny * M;
  const bool zero = mi.nyq || m == 0;
  for (int j = 0; j < Ny + 3; ++j) {
    push(w, (j < Ny && !zero) ? v[(size_t)j * M + m] : z2());
    const int i = j - 3;
    if (i < 0) continue;
    const double* a = sA + 7 * i;
    const double* b = sB + 7 * i;
    double2 r = z2();
#pragma unroll
    for (int d = 0; d < 7; ++d) r = axpy(b[d] - mi.k2 * a[d], w[d], r);
    const double* l2 = sLU2 + 7 * i;
    const double* l1 = sLU1 + 7 * i;
    scr[(size_t)i * M + m] = fwd(r, l2[0], l2[1], l2[2], h2);
    scr2[(size_t)i * M + m] = fwd(band7(sB1 + 7 * i, w), l1[0], l1[1], l1[2], h1);
  }
  double2 n2[3] = {z2(), z2(), z2()}, n1[3] = {z2(), z2(), z2()};
  for (int i = Ny - 1; i >= 0; --i) {
    const size_t o = (size_t)i * M + m;
    const double* l2 = sLU2 + 7 * i;
    const double* l1 = sLU1 + 7 * i;
    chi[o] = bwd(scr[o], l2[3], l2[4], l2[5], l2[6], n2);
    dv[o] = bwd(scr2[o], l1[3], l1[4], l1[5], l1[6], n1);
  }
}

// ---------------------------------------------------------------------------
// Set-up: LU factors (no pivoting) of the Poisson operator B - k^2 A per class
// and of the RK3 Helmholtz operator per (class, substep), homogeneous
// solutions chi_a, chi_b, v_a, v_b and the inverse influence matrix.
// ---------------------------------------------------------------------------

// One row of a (3,3)-banded Doolittle LU.  row[d]: column i-3+d.  Up[r][e] =
// u(k, k+e) of the previous rows k = i-3+r.  Returns l (cols i-3..i-1) and
// u (cols i..i+3).
__device__ void lu_row(int i, const double row[7], const double Up[3][4], double l[3], double u[4]) {
  for (int d = 0; d < 3; ++d) {
    l[d] = 0.0;
    const int j = i - 3 + d;
    if (j < 0) continue;
    double s = row[d];
    for (int k = i - 3; k < j; ++k) {
      if (k < 0) continue;
      const int e = j - k;  // <= 3
      s -= l[k - (i - 3)] * Up[k - (i - 3)][e];
    }
    l[d] = s / Up[d][0];
  }
  for (int e = 0; e < 4; ++e) {
    const int j = i + e;
    double s = row[3 + e];
    for (int k = i - 3; k < i; ++k) {
      if (k < 0) continue;
      const int ee = j - k;
      if (ee > 3) continue;
      s -= l[k - (i - 3)] * Up[k - (i - 3)][ee];
    }
    u[e] = s;
  }
}

// Factor rows of op(i, d) and store l, u, 1/u_ii at tab[(i*stride + q) * C].
template <typename RowFn>
__device__ void factor(int Ny, RowFn rowfn, double* tab, size_t stride, size_t C) {
  double Up[3][4] = {{0}};
  for (int i = 0; i < Ny; ++i) {
    double row[7], l[3], u[4];
    rowfn(i, row);
    lu_row(i, row, Up, l, u);
    double* o = tab + (size_t)i * stride * C;
    o[0] = l[0]; o[C] = l[1]; o[2 * C] = l[2];
    o[3 * C] = u[1]; o[4 * C] = u[2]; o[5 * C] = u[3];
    o[6 * C] = 1.0 / u[0];
    for (int e = 0; e < 4; ++e) { Up[0][e] = Up[1][e]; Up[1][e] = Up[2][e]; Up[2][e] = u[e]; }
  }
}

__global__ void k_setup_pois(Geo g, YTabs t, double* pois) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.C) return;
  const int kx = c % g.nxh, kza = c / g.nxh;
  const double k2 = g.k1[kx] * g.k1[kx] + g.k3[kza] * g.k3[kza];
  const int Ny = g.Ny;
  factor(Ny, [&](int i, double* row) {
    for (int d = 0; d < 7; ++d) row[d] = (i == 0 || i == Ny - 1) ? (d == 3 ? 1.0 : 0.0)
                                                                 : t.B2[7 * i + d] - k2 * t.A2[7 * i + d];
  }, pois + c, 7, g.C);
}

// Substeps s0 .. s0 + ns - 1 into table slots 0 .. ns - 1.
__global__ void k_setup_helm(Geo g, YTabs t, const double* __restrict__ pois, double* helm, double* infl, int s0,
                             int ns) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ns * g.C) return;
  const int slot = idx / g.C, c = idx - slot * g.C, s = s0 + slot;
  const int kx = c % g.nxh, kza = c / g.nxh;
  const double k2 = g.k1[kx] * g.k1[kx] + g.k3[kza] * g.k3[kza];
  const int Ny = g.Ny;
  const size_t C = g.C;
  const double hb = c_rk3[s][3] * g.dt * g.nu;
  double* H = helm + (size_t)slot * Ny * 11 * C + c;
  factor(Ny, [&](int i, double* row) {
    for (int d = 0; d < 7; ++d) row[d] = (i == 0 || i == Ny - 1) ? (d == 3 ? 1.0 : 0.0)
                                                                 : (1.0 + hb * k2) * t.A2[7 * i + d] - hb * t.B2[7 * i + d];
  }, H, 11, C);
  // homogeneous chi_a (1 at y=-1), chi_b (1 at y=+1): forward sweeps park z in slots 9, 10
  for (int q = 0; q < 2; ++q) {
    double h[3] = {0, 0, 0};
    for (int i = 0; i < Ny; ++i) {
      const double* Hi = H + (size_t)i * 11 * C;
      double r = (q == 0 ? (i == 0) : (i == Ny - 1)) ? 1.0 : 0.0;
      r -= Hi[0] * h[0] + Hi[C] * h[1] + Hi[2 * C] * h[2];
      h[0] = h[1]; h[1] = h[2]; h[2] = r;
      H[((size_t)i * 11 + 9 + q) * C] = r;
    }
    double nx[3] = {0, 0, 0};
    for (int i = Ny - 1; i >= 0; --i) {
      const double* Hi = H + (size_t)i * 11 * C;
      double x = (Hi[(9 + q) * C] - Hi[3 * C] * nx[0] - Hi[4 * C] * nx[1] - Hi[5 * C] * nx[2]) * Hi[6 * C];
      nx[2] = nx[1]; nx[1] = nx[0]; nx[0] = x;
      H[((size_t)i * 11 + 7 + q) * C] = x;
    }
  }
  // v_a, v_b: (B - k^2 A) v = A chi, v(+-1) = 0
  const double* P = pois + c;
  double gm[2][2];
  for (int q = 0; q < 2; ++q) {
    double w[7] = {0, 0, 0, 0, 0, 0, 0}, h[3] = {0, 0, 0};
    for (int j = 0; j < Ny + 3; ++j) {
      for (int d = 0; d < 6; ++d) w[d] = w[d + 1];
      w[6] = j < Ny ? H[((size_t)j * 11 + 7 + q) * C] : 0.0;
      const int i = j - 3;
      if (i < 0) continue;
      double r = 0.0;
      if (i > 0 && i < Ny - 1)
        for (int d = 0; d < 7; ++d) r += t.A2[7 * i + d] * w[d];
      const double* Pi = P + (size_t)i * 7 * C;
      r -= Pi[0] * h[0] + Pi[C] * h[1] + Pi[2 * C] * h[2];
      h[0] = h[1]; h[1] = h[2]; h[2] = r;
      H[((size_t)i * 11 + 9 + q) * C] = r;
    }
    double nx[3] = {0, 0, 0}, s0 = 0.0, sN = 0.0;
    for (int i = Ny - 1; i >= 0; --i) {
      const double* Pi = P + (size_t)i * 7 * C;
      double x = (H[((size_t)i * 11 + 9 + q) * C] - Pi[3 * C] * nx[0] - Pi[4 * C] * nx[1] - Pi[5 * C] * nx[2]) * Pi[6 * C];
      nx[2] = nx[1]; nx[1] = nx[0]; nx[0] = x;
      H[((size_t)i * 11 + 9 + q) * C] = x;
      s0 += t.d0[i] * x;
      sN += t.dN[i] * x;
    }
    gm[0][q] = s0;   // row: wall (0: y=-1, 1: y=+1); column: solution a/b
    gm[1][q] = sN;
  }
  const double det = gm[0][0] * gm[1][1] - gm[0][1] * gm[1][0];
  double* G = infl + (size_t)slot * 4 * C + c;
  G[0] = gm[1][1] / det;
  G[C] = -gm[0][1] / det;
  G[2 * C] = -gm[1][0] / det;
  G[3 * C] = gm[0][0] / det;
}


// ---------------------------------------------------------------------------
// Filtered pressure (Sec. 3.1, Eq. (2)): interior rows
//   (B - k^2 A) p = A r - B F22,  r = k1^2 F11 + k3^2 F33 + 2 k1 k3 F13 - 2 i k1 D1 F12 - 2 i k3 D1 F23,
// wall rows dp/dy = nu G chi; F_ij = G P(u_i u_j).  Particular solution with
// p(+-1) = 0 (Poisson factors), then the homogeneous pair p_a, p_b meets the
// Neumann conditions through the inverse influence matrix.  Mean mode: P = -F22.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_pressure(Geo g, YTabs t, const double* __restrict__ pois,
                                                  const double* __restrict__ prs, const double* __restrict__ prsinv,
                                                  const double2* __restrict__ P11, const double2* __restrict__ P22,
                                                  const double2* __restrict__ P33, const double2* __restrict__ P12,
                                                  const double2* __restrict__ P13, const double2* __restrict__ P23,
                                                  const double* __restrict__ G, const double2* __restrict__ chi,
                                                  double2* pout, double2* scr) {
  extern __shared__ double sm[];
  const int Ny = g.Ny;
  double* sA = sm;
  double* sB = sm + 7 * Ny;
  double* sB1 = sm + 14 * Ny;
  double* sLU = sm + 21 * Ny;
  load_tab(sA, t.A2, 7 * Ny);
  load_tab(sB, t.B2, 7 * Ny);
  load_tab(sB1, t.B1, 7 * Ny);
  load_tab(sLU, t.lu1, 7 * Ny);
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.M) return;
  const size_t M = g.M, C = g.C;
  ModeInfo mi = mode_info(g, m);
  const double gm = G[m];
  if (mi.nyq) {
    for (int i = 0; i < Ny; ++i) pout[(size_t)i * M + m] = z2();
    return;
  }
  if (m == 0) {
    for (int i = 0; i < Ny; ++i) pout[(size_t)i * M] = scl(-gm, P22[(size_t)i * M]);
    return;
  }
  double2* s2 = scr + (size_t)Ny * M;
  double2 wa[7], wb[7], ha[3], hb[3];
#pragma unroll
  for (int d = 0; d < 7; ++d) { wa[d] = z2(); wb[d] = z2(); }
#pragma unroll
  for (int d = 0; d < 3; ++d) { ha[d] = z2(); hb[d] = z2(); }
  // D1 of F12 and F23: forward sweeps
  for (int j = 0; j < Ny + 3; ++j) {
    push(wa, j < Ny ? scl(gm, P12[(size_t)j * M + m]) : z2());
    push(wb, j < Ny ? scl(gm, P23[(size_t)j * M + m]) : z2());
    const int i = j - 3;
    if (i < 0) continue;
    const double* l = sLU + 7 * i;
    scr[(size_t)i * M + m] = fwd(band7(sB1 + 7 * i, wa), l[0], l[1], l[2], ha);
    s2[(size_t)i * M + m] = fwd(band7(sB1 + 7 * i, wb), l[0], l[1], l[2], hb);
  }
  // backward sweeps; assemble r in place of the first scratch field
  double2 na[3] = {z2(), z2(), z2()}, nb[3] = {z2(), z2(), z2()};
  const double k1 = mi.k1, k3 = mi.k3;
  for (int i = Ny - 1; i >= 0; --i) {
    const size_t o = (size_t)i * M + m;
    const double* lu = sLU + 7 * i;
    const double2 d12 = bwd(scr[o], lu[3], lu[4], lu[5], lu[6], na);
    const double2 d23 = bwd(s2[o], lu[3], lu[4], lu[5], lu[6], nb);
    double2 r = scl(gm * k1 * k1, P11[o]);
    r = axpy(gm * k3 * k3, P33[o], r);
    r = axpy(2.0 * gm * k1 * k3, P13[o], r);
    // - 2 i (k1 d12 + k3 d23)
    const double2 q = make_double2(k1 * d12.x + k3 * d23.x, k1 * d12.y + k3 * d23.y);
    r.x += 2.0 * q.y;
    r.y -= 2.0 * q.x;
    scr[o] = r;
  }
  // A r - B F22 and the Poisson forward sweep
  const double* P = pois + mi.c;
#pragma unroll
  for (int d = 0; d < 7; ++d) { wa[d] = z2(); wb[d] = z2(); }
#pragma unroll
  for (int d = 0; d < 3; ++d) ha[d] = z2();
  for (int j = 0; j < Ny + 3; ++j) {
    push(wa, j < Ny ? scr[(size_t)j * M + m] : z2());
    push(wb, j < Ny ? scl(gm, P22[(size_t)j * M + m]) : z2());
    const int i = j - 3;
    if (i < 0) continue;
    double2 rhs = z2();
    if (i > 0 && i < Ny - 1) rhs = sub(band7(sA + 7 * i, wa), band7(sB + 7 * i, wb));
    const double* Pi = P + (size_t)i * 7 * C;
    s2[(size_t)i * M + m] = fwd(rhs, Pi[0], Pi[C], Pi[2 * C], ha);
  }
  double2 nx[3] = {z2(), z2(), z2()}, s0 = z2(), sN = z2();
  for (int i = Ny - 1; i >= 0; --i) {
    const size_t o = (size_t)i * M + m;
    const double* Pi = P + (size_t)i * 7 * C;
    const double2 pp = bwd(s2[o], Pi[3 * C], Pi[4 * C], Pi[5 * C], Pi[6 * C], nx);
    pout[o] = pp;
    s0 = axpy(t.d0[i], pp, s0);
    sN = axpy(t.dN[i], pp, sN);
  }
  // Neumann conditions dp/dy(+-1) = nu G chi(+-1)
  const double2 b0 = sub(scl(g.nu * gm, load_c(chi, m, g.pair)), s0);
  const double2 bN = sub(scl(g.nu * gm, load_c(chi, (size_t)(Ny - 1) * M + m, g.pair)), sN);
  const double* Gi = prsinv + mi.c;
  const double g11 = Gi[0], g12 = Gi[C], g21 = Gi[2 * C], g22 = Gi[3 * C];
  const double2 cA = make_double2(g11 * b0.x + g12 * bN.x, g11 * b0.y + g12 * bN.y);
  const double2 cB = make_double2(g21 * b0.x + g22 * bN.x, g21 * b0.y + g22 * bN.y);
  for (int i = 0; i < Ny; ++i) {
    const size_t o = (size_t)i * M + m;
    const double pa = prs[((size_t)i * 2) * C + mi.c], pb = prs[((size_t)i * 2 + 1) * C + mi.c];
    pout[o] = axpy(pb, cB, axpy(pa, cA, pout[o]));
  }
}

// Homogeneous Dirichlet solutions of (B - k^2 A) p = 0 (p_a = 1 at y = -1, p_b = 1 at
// y = +1) per class, and the inverse of their wall-derivative matrix (class 0, whose
// Neumann problem is singular, is left at zero and never used).
__global__ void k_setup_pressure(Geo g, YTabs t, const double* __restrict__ pois, double* prs, double* prsinv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.C) return;
  const int Ny = g.Ny;
  const size_t C = g.C;
  const double* P = pois + c;
  double dm[2][2];
  for (int q = 0; q < 2; ++q) {
    double h[3] = {0, 0, 0};
    for (int i = 0; i < Ny; ++i) {
      const double* Pi = P + (size_t)i * 7 * C;
      double r = (q == 0 ? i == 0 : i == Ny - 1) ? 1.0 : 0.0;
      r -= Pi[0] * h[0] + Pi[C] * h[1] + Pi[2 * C] * h[2];
      h[0] = h[1]; h[1] = h[2]; h[2] = r;
      prs[((size_t)i * 2 + q) * C + c] = r;
    }
    double nx[3] = {0, 0, 0}, s0 = 0, sN = 0;
    for (int i = Ny - 1; i >= 0; --i) {
      const double* Pi = P + (size_t)i * 7 * C;
      double x = (prs[((size_t)i * 2 + q) * C + c] - Pi[3 * C] * nx[0] - Pi[4 * C] * nx[1] - Pi[5 * C] * nx[2]) * Pi[6 * C];
      nx[2] = nx[1]; nx[1] = nx[0]; nx[0] = x;
      prs[((size_t)i * 2 + q) * C + c] = x;
      s0 += t.d0[i] * x;
      sN += t.dN[i] * x;
    }
    dm[0][q] = s0;
    dm[1][q] = sN;
  }
  const double det = dm[0][0] * dm[1][1] - dm[0][1] * dm[1][0];
  const bool ok = c != 0 && det != 0.0;
  prsinv[c] = ok ? dm[1][1] / det : 0.0;
  prsinv[C + c] = ok ? -dm[0][1] / det : 0.0;
  prsinv[2 * C + c] = ok ? -dm[1][0] / det : 0.0;
  prsinv[3 * C + c] = ok ? dm[0][0] / det : 0.0;
}

// ---------------------------------------------------------------------------
// Packed launches over several channels: one grid covers the blocks of every
// run; a block finds its run from the per-run block offsets and executes the
// same body with its local block index.  Runs may differ in size and RK3 phase.
// ---------------------------------------------------------------------------

template <class P> struct YBatch {
  P p[CHAN_MAXBATCH];
  int begin[CHAN_MAXBATCH + 1];
  int n;
};

__device__ __forceinline__ int batch_run(const int* begin, int n, int b) {
  int r = 0;
  while (r + 1 < n && b >= begin[r + 1]) ++r;
  return r;
}

template <class Y, bool F32OUT = false>
__global__ void __launch_bounds__(128) kb_pre(YBatch<PreP> B) {
  const int r = batch_run(B.begin, B.n, blockIdx.x);
  const PreP& p = B.p[r];
  pre_body<Y, F32OUT>(p.g, p.t, p.v, p.om, p.dv, p.U1, p.U3, p.u1o, p.u3o, p.om1o, p.om3o, blockIdx.x - B.begin[r]);
}
template <class Y>
__global__ void __launch_bounds__(128) kb_nonlin(YBatch<NonlinP> B) {
  const int r = batch_run(B.begin, B.n, blockIdx.x);
  const NonlinP& p = B.p[r];
  nonlin_body<Y>(p.g, p.t, p.H1, p.H2, p.H3, p.Nchi, p.Nom, p.scr, blockIdx.x - B.begin[r]);
}
template <class Y>
__global__ void __launch_bounds__(128) kb_helm(YBatch<HelmP> B) {
  typedef typename Y::R R;
  const int r = batch_run(B.begin, B.n, blockIdx.x);
  const HelmP& p = B.p[r];
  helm_body<Y, 2>(p.g, p.t, static_cast<const R*>(p.helm), p.om, p.chi, p.Nchi, p.Nom, p.Nchi_p, p.Nom_p, p.Rom,
                  p.Rchi, p.scal, p.scr, p.s, blockIdx.x - B.begin[r]);
}
template <class Y>
__global__ void __launch_bounds__(128) kb_poisson(YBatch<PoisP> B) {
  typedef typename Y::R R;
  const int r = batch_run(B.begin, B.n, blockIdx.x);
  const PoisP& p = B.p[r];
  poisson_body<Y>(p.g, p.t, static_cast<const R*>(p.helm), static_cast<const R*>(p.pois),
                  static_cast<const R*>(p.infl), p.v, p.chi, p.dv, p.scr, p.scal, p.s, blockIdx.x - B.begin[r]);
}
__global__ void __launch_bounds__(256) kb_mean(YBatch<MeanP> B) {
  const MeanP& p = B.p[blockIdx.x];
  mean_body(p.g, p.t, p.helm, p.meanh, p.H1, p.H3, p.U1, p.U3, p.H1p, p.H3p, p.scal, p.s, 0);
}

// Pair copy of the per-class tables for the double-float y-kernels.
__global__ void k_split_tab(const double* __restrict__ src, dfr* dst, size_t n) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = df_split(src[e]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static cudaError_t smem_attr(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

static bool use_df(const chan_s* h) { return prec_pairs(h->prec); }

// Helmholtz factors, homogeneous solutions and influence matrices of substeps
// s0 .. s0+ns-1 into slots 0 .. ns-1 (and their pair copies in the double-float mode).
static cudaError_t setup_helm_slots(chan_s* h, int s0, int ns) {
  Geo g = geo(h);
  YTabs t = ytabs(h);
  k_setup_helm<<<(ns * h->C + 127) / 128, 128, 0, h->stream>>>(g, t, h->pois, h->helm, h->infl, s0, ns);
  if (use_df(h)) {
    const size_t nh = (size_t)ns * h->Ny * 11 * h->C, ni = (size_t)ns * 4 * h->C;
    k_split_tab<<<(unsigned)((nh + 255) / 256), 256, 0, h->stream>>>(h->helm, h->helm_df, nh);
    k_split_tab<<<(unsigned)((ni + 255) / 256), 256, 0, h->stream>>>(h->infl, h->infl_df, ni);
  }
  return cudaGetLastError();
}

cudaError_t launch_setup_tables(chan_s* h) {
  Geo g = geo(h);
  YTabs t = ytabs(h);
  k_setup_pois<<<(h->C + 127) / 128, 128, 0, h->stream>>>(g, t, h->pois);
  if (use_df(h)) {
    const size_t np = (size_t)h->Ny * 7 * h->C;
    k_split_tab<<<(unsigned)((np + 255) / 256), 256, 0, h->stream>>>(h->pois, h->pois_df, np);
    const double* src[6] = {h->tab_A2, h->tab_B2, h->tab_B1, h->tab_lu1, h->tab_d0, h->tab_dN};
    const size_t cnt[6] = {7 * (size_t)h->Ny, 7 * (size_t)h->Ny, 7 * (size_t)h->Ny, 7 * (size_t)h->Ny,
                           (size_t)h->Ny, (size_t)h->Ny};
    dfr* dst = h->tab_pairs;
    for (int k = 0; k < 6; ++k) {
      k_split_tab<<<(unsigned)((cnt[k] + 255) / 256), 256, 0, h->stream>>>(src[k], dst, cnt[k]);
      dst += cnt[k];
    }
  }
  cudaError_t e;
  if (!h->lean) {
    if ((e = setup_helm_slots(h, 0, 3)) != cudaSuccess) return e;
    for (int s = 0; s < 3; ++s)
      k_setup_mean<<<1, 32, 0, h->stream>>>(g, t, helm_slot(h, s), h->meanh + (size_t)s * (h->Ny + 1));
  } else {   // one slot: U_h of each substep from its factors, then the slot is refilled per substep
    for (int s = 0; s < 3; ++s) {
      if ((e = setup_helm_slots(h, s, 1)) != cudaSuccess) return e;
      k_setup_mean<<<1, 32, 0, h->stream>>>(g, t, h->helm, h->meanh + (size_t)s * (h->Ny + 1));
      if (h->lean == 2)
        k_gather_class0<<<(11 * h->Ny + 255) / 256, 256, 0, h->stream>>>(h->helm, (size_t)h->C, 11 * h->Ny,
                                                                           h->mean_tab + (size_t)s * 11 * h->Ny);
    }
    h->lean_slot = 2;
  }
  return cudaGetLastError();
}

cudaError_t launch_setup_pois(chan_s* h, double* dst) {
  k_setup_pois<<<(h->C + 127) / 128, 128, 0, h->stream>>>(geo(h), ytabs(h), dst);
  return cudaGetLastError();
}

cudaError_t launch_copy_mean_modes(chan_s* h, const double2* H1, const double2* H3) {
  k_copy_mean_modes<<<1, 256, 0, h->stream>>>(H1, H3, (size_t)h->M, h->Ny, h->h00);
  return cudaGetLastError();
}

cudaError_t launch_setup_substep(chan_s* h, int s) {
  if (!h->lean) return cudaSuccess;
  const cudaError_t e = setup_helm_slots(h, s, 1);
  h->lean_slot = s;
  return e;
}



cudaError_t launch_derive(chan_s* h) {
  size_t sm = sizeof(double) * 35 * h->Ny;
  cudaError_t e = smem_attr((const void*)k_derive, sm);
  if (e != cudaSuccess) return e;
  k_derive<<<ygrid(h), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), h->v, h->chi, h->dv, h->scr);
  return cudaGetLastError();
}

cudaError_t launch_pre(chan_s* h, double2* u1, double2* u3, double2* om1, double2* om3, bool f32) {
  size_t sm = ysm(h, 14, kRingPre);
  f32 = f32 && prec_t32(h->prec);
  const bool df = use_df(h);
  const void* fn = df ? (f32 ? (const void*)k_pre_df_f32 : (const void*)k_pre_df)
                      : (f32 ? (const void*)k_pre_f32 : (const void*)k_pre);
  cudaError_t e = smem_attr(fn, sm);
  if (e != cudaSuccess) return e;
  if (df && f32)
    k_pre_df_f32<<<ygrid(h).x + 1, kYThreads, sm, h->stream>>>(geo(h), ytabs(h), h->v, h->om, h->dv, h->U1, h->U3, u1, u3, om1, om3);
  else if (df)
    k_pre_df<<<ygrid(h).x + 1, kYThreads, sm, h->stream>>>(geo(h), ytabs(h), h->v, h->om, h->dv, h->U1, h->U3, u1, u3, om1, om3);
  else if (f32)
    k_pre_f32<<<ygrid(h).x + 1, kYThreads, sm, h->stream>>>(geo(h), ytabs(h), h->v, h->om, h->dv, h->U1, h->U3, u1, u3, om1, om3);
  else
    k_pre<<<ygrid(h).x + 1, kYThreads, sm, h->stream>>>(geo(h), ytabs(h), h->v, h->om, h->dv, h->U1, h->U3, u1, u3, om1, om3);
  return cudaGetLastError();
}

cudaError_t launch_nonlin(chan_s* h, const double2* H1, const double2* H2, const double2* H3, double2* Nchi,
                          double2* Nom) {
  size_t sm = ysm(h, 14, kRingNonlin);
  const void* fn = use_df(h) ? (const void*)k_nonlin_df : (const void*)k_nonlin;
  cudaError_t e = smem_attr(fn, sm);
  if (e != cudaSuccess) return e;
  if (use_df(h))
    k_nonlin_df<<<ygrid(h), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), H1, H2, H3, Nchi, Nom, h->scr);
  else
    k_nonlin<<<ygrid(h), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), H1, H2, H3, Nchi, Nom, h->scr);
  return cudaGetLastError();
}

cudaError_t launch_nonlin_scratch(chan_s* h, const double2* H1, const double2* H2, const double2* H3, double2* Nchi,
                                 double2* Nom, double2* scr) {
  size_t sm = ysm(h, 14, kRingNonlin);
  cudaError_t e = smem_attr((const void*)k_nonlin, sm);
  if (e != cudaSuccess) return e;
  k_nonlin<<<ygrid(h), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), H1, H2, H3, Nchi, Nom, scr);
  return cudaGetLastError();
}

cudaError_t launch_helm(chan_s* h, const double2* Nchi, const double2* Nom, int s) {
  size_t sm = ysm(h, 14, kRingHelm);
  const void* fn = use_df(h) ? (const void*)k_helm<YDF> : (const void*)k_helm<YF64>;
  cudaError_t e = smem_attr(fn, sm);
  if (e != cudaSuccess) return e;
  if (use_df(h))
    k_helm<YDF><<<dim3(ygrid(h).x, 2), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), (const dfr*)helm_slot_y(h, s), h->om,
                                                        h->chi, Nchi, Nom, h->Nchi_p, h->Nom_p, h->Rom, h->Rchi,
                                                        h->scal, h->scr, s);
  else
    k_helm<YF64><<<dim3(ygrid(h).x, 2), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), (const double*)helm_slot_y(h, s), h->om,
                                                         h->chi, Nchi, Nom, h->Nchi_p, h->Nom_p, h->Rom, h->Rchi,
                                                         h->scal, h->scr, s);
  return cudaGetLastError();
}

cudaError_t launch_poisson(chan_s* h, int s) {
  size_t sm = ysm(h, 23, kRingPois);
  const void* fn = use_df(h) ? (const void*)k_poisson<YDF> : (const void*)k_poisson<YF64>;
  cudaError_t e = smem_attr(fn, sm);
  if (e != cudaSuccess) return e;
  if (use_df(h))
    k_poisson<YDF><<<ygrid(h), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), (const dfr*)helm_slot_y(h, s),
                                                           (const dfr*)pois_y(h), (const dfr*)infl_slot_y(h, s),
                                                           h->v, h->chi, h->dv, h->scr, h->scal, s);
  else
    k_poisson<YF64><<<ygrid(h), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), (const double*)helm_slot_y(h, s),
                                                            (const double*)pois_y(h), (const double*)infl_slot_y(h, s),
                                                            h->v, h->chi, h->dv, h->scr, h->scal, s);
  return cudaGetLastError();
}

cudaError_t launch_mean(chan_s* h, const double2* H1, const double2* H3, int s, cudaStream_t st) {
  size_t sm = sizeof(double) * (9 * h->Ny + 256);
  cudaError_t e = smem_attr((const void*)k_mean, sm);
  if (e != cudaSuccess) return e;
  Geo g = geo(h);
  const double* helm = helm_slot(h, s);
  if (h->lean == 2) {   // the compact copies: one class, one mode per plane
    g.M = 1;
    g.C = 1;
    helm = h->mean_tab + (size_t)s * 11 * h->Ny;
    H1 = h->h00;
    H3 = h->h00 + h->Ny;
  }
  k_mean<<<1, 256, sm, st ? st : h->stream>>>(g, ytabs(h), helm, h->meanh, H1, H3, h->U1, h->U3, h->H1m_p,
                                    h->H3m_p, h->scal, s);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Packed launchers: the runs of hs[0..n) (n <= CHAN_MAXBATCH) in one grid on
// `stream`; w[r] holds run r's work-field pointers (see batch_step in chan_api).
// ---------------------------------------------------------------------------
template <class P>
static int fill_begin(YBatch<P>& B, chan_s* const* hs, int n, int extra = 0) {
  B.n = n;
  int acc = 0;
  for (int r = 0; r < n; ++r) {
    B.begin[r] = acc;
    acc += (hs[r]->M + kYThreads - 1) / kYThreads + extra;
  }
  B.begin[n] = acc;
  return acc;
}
static int max_ny(chan_s* const* hs, int n) {
  int m = 0;
  for (int r = 0; r < n; ++r) m = hs[r]->Ny > m ? hs[r]->Ny : m;
  return m;
}

cudaError_t launch_pre_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  YBatch<PreP> B;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    B.p[r] = PreP{geo(h), ytabs(h), h->v, h->om, h->dv, h->U1, h->U3, w[r].u1, w[r].u3, w[r].om1, w[r].om3};
  }
  const int blocks = fill_begin(B, hs, n, 1);   // + the mean-mode block of each run
  const size_t sm = ysm_batch(hs, n, 14, kRingPre);
  const bool df = use_df(hs[0]), f32 = prec_t32(hs[0]->prec);
  const void* fn = df ? (f32 ? (const void*)kb_pre<YDF, true> : (const void*)kb_pre<YDF>)
                      : (f32 ? (const void*)kb_pre<YF64, true> : (const void*)kb_pre<YF64>);
  cudaError_t e = smem_attr(fn, sm);
  if (e != cudaSuccess) return e;
  if (df && f32) kb_pre<YDF, true><<<blocks, kYThreads, sm, st>>>(B);
  else if (df) kb_pre<YDF><<<blocks, kYThreads, sm, st>>>(B);
  else if (f32) kb_pre<YF64, true><<<blocks, kYThreads, sm, st>>>(B);
  else kb_pre<YF64><<<blocks, kYThreads, sm, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_nonlin_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  YBatch<NonlinP> B;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    B.p[r] = NonlinP{geo(h), ytabs(h), w[r].H1, w[r].H2, w[r].H3, w[r].Nchi, w[r].Nom, h->scr};
  }
  const int blocks = fill_begin(B, hs, n);
  const size_t sm = ysm_batch(hs, n, 14, kRingNonlin);
  const bool df = use_df(hs[0]);
  cudaError_t e = smem_attr(df ? (const void*)kb_nonlin<YDF> : (const void*)kb_nonlin<YF64>, sm);
  if (e != cudaSuccess) return e;
  if (df) kb_nonlin<YDF><<<blocks, kYThreads, sm, st>>>(B);
  else kb_nonlin<YF64><<<blocks, kYThreads, sm, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_helm_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  YBatch<HelmP> B;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    B.p[r] = HelmP{geo(h), ytabs(h), helm_slot_y(h, (int)(h->nsub % 3)), h->om, h->chi, w[r].Nchi, w[r].Nom, h->Nchi_p, h->Nom_p,
                   h->Rom, h->Rchi, h->scal, h->scr, (int)(h->nsub % 3)};
  }
  const int blocks = fill_begin(B, hs, n);
  const size_t sm = ysm_batch(hs, n, 14, kRingHelm);
  const bool df = use_df(hs[0]);
  cudaError_t e = smem_attr(df ? (const void*)kb_helm<YDF> : (const void*)kb_helm<YF64>, sm);
  if (e != cudaSuccess) return e;
  if (df) kb_helm<YDF><<<blocks, kYThreads, sm, st>>>(B);
  else kb_helm<YF64><<<blocks, kYThreads, sm, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_poisson_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  (void)w;
  YBatch<PoisP> B;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    const int s = (int)(h->nsub % 3);
    B.p[r] = PoisP{geo(h), ytabs(h), helm_slot_y(h, s), pois_y(h), infl_slot_y(h, s), h->v, h->chi, h->dv, h->scr,
                   h->scal, (int)(h->nsub % 3)};
  }
  const int blocks = fill_begin(B, hs, n);
  const size_t sm = ysm_batch(hs, n, 23, kRingPois);
  const bool df = use_df(hs[0]);
  cudaError_t e = smem_attr(df ? (const void*)kb_poisson<YDF> : (const void*)kb_poisson<YF64>, sm);
  if (e != cudaSuccess) return e;
  if (df) kb_poisson<YDF><<<blocks, kYThreads, sm, st>>>(B);
  else kb_poisson<YF64><<<blocks, kYThreads, sm, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_mean_batch(chan_s* const* hs, int n, const BatchWork* w, cudaStream_t st) {
  YBatch<MeanP> B;
  B.n = n;
  for (int r = 0; r < n; ++r) {
    chan_s* h = hs[r];
    B.p[r] = MeanP{geo(h), ytabs(h), helm_slot(h, (int)(h->nsub % 3)), h->meanh, w[r].H1, w[r].H3, h->U1, h->U3, h->H1m_p, h->H3m_p,
                   h->scal, (int)(h->nsub % 3)};
  }
  const size_t sm = sizeof(double) * (9 * max_ny(hs, n) + 256);
  cudaError_t e = smem_attr((const void*)kb_mean, sm);
  if (e != cudaSuccess) return e;
  kb_mean<<<n, 256, sm, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_pressure(chan_s* h, const double2* const* P, double2* out) {
  if (!h->prs) return cudaErrorInvalidValue;
  size_t sm = sizeof(double) * 28 * h->Ny;
  cudaError_t e = smem_attr((const void*)k_pressure, sm);
  if (e != cudaSuccess) return e;
  k_pressure<<<ygrid(h), kYThreads, sm, h->stream>>>(geo(h), ytabs(h), h->pois_prs ? h->pois_prs : h->pois, h->prs, h->prsinv, P[0], P[1], P[2],
                                                     P[3], P[4], P[5], h->G, h->chi, out, h->scr);
  return cudaGetLastError();
}

cudaError_t launch_setup_pressure(chan_s* h) {
  k_setup_pressure<<<(h->C + 127) / 128, 128, 0, h->stream>>>(geo(h), ytabs(h), h->pois_prs ? h->pois_prs : h->pois,
                                                               h->prs, h->prsinv);
  return cudaGetLastError();
}

double chan_rk3_weight(int s) { return h_rk3[s][2] + h_rk3[s][3]; }
