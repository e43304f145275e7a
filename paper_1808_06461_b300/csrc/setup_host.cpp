// Host set-up of the channel library: wall-normal mesh, compact finite
// differences (Appendix B of arXiv:1808.06461), banded LU factors and FFT
// twiddles.  Coefficient systems are solved in IEEE quad precision
// (__float128) so that the double-precision tables are correctly rounded.
#include "chan_host.h"

#include <quadmath.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

typedef __float128 qd;

// Mesh with spacing proportional to a local Kolmogorov scale (Sec. 2.1 gives
// the criterion, not a formula): dy+/dj = C (eta_w^4 + kappa y+)^(1/4), whose
// integral is j(y+) = 4/(3 kappa C) [(eta_w^4 + kappa y+)^(3/4) - eta_w^3].
// Lower half from the closed form, upper half mirrored exactly.
int chanh_ygrid(int ny, double re, double eta_w, double* y) {
  if (ny < 9 || (ny % 2) != 1 || !(re > 0.0) || !(eta_w > 0.0)) return -1;
  const double kappa = 0.4;
  const int h = (ny - 1) / 2;
  const double c = (4.0 / (3.0 * kappa)) * (std::pow(std::pow(eta_w, 4.0) + kappa * re, 0.75) - std::pow(eta_w, 3.0)) / h;
  for (int j = 0; j < h; ++j) {
    double yp = (std::pow(3.0 * kappa * c * j / 4.0 + std::pow(eta_w, 3.0), 4.0 / 3.0) - std::pow(eta_w, 4.0)) / kappa;
    y[j] = -1.0 + yp / re;
  }
  y[h] = 0.0;
  for (int j = h + 1; j < ny; ++j) y[j] = -y[ny - 1 - j];
  return 0;
}

// Stencil of row i: seven points inside; rows 0..2 (and their mirrors) use
// columns [0, i+3], the progressive reduction at the corners.
static void support(int i, int n, int* lo, int* hi) {
  int ii = i < n - 1 - i ? i : n - 1 - i;
  if (ii >= 3) { *lo = i - 3; *hi = i + 3; return; }
  if (i == ii) { *lo = 0; *hi = ii + 3; return; }
  *lo = n - 1 - (ii + 3); *hi = n - 1;
}

// Solve m x m (m <= 16) in quad with partial pivoting.  Returns 0 or -3.
static int qsolve(int m, qd* M, qd* r) {
  for (int c = 0; c < m; ++c) {
    int p = c;
    for (int i = c + 1; i < m; ++i)
      if (fabsq(M[i * m + c]) > fabsq(M[p * m + c])) p = i;
    if (M[p * m + c] == 0) return -3;
    if (p != c) {
      for (int j = 0; j < m; ++j) { qd t = M[c * m + j]; M[c * m + j] = M[p * m + j]; M[p * m + j] = t; }
      qd t = r[c]; r[c] = r[p]; r[p] = t;
    }
    for (int i = c + 1; i < m; ++i) {
      qd f = M[i * m + c] / M[c * m + c];
      if (f == 0) continue;
      for (int j = c; j < m; ++j) M[i * m + j] -= f * M[c * m + j];
      r[i] -= f * r[c];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    qd s = r[i];
    for (int j = i + 1; j < m; ++j) s -= M[i * m + j] * r[j];
    r[i] = s / M[i * m + i];
  }
  return 0;
}

// Coefficients of row i of A f^(deriv) = B f with A_ii = 1: the remaining
// unknowns make the row exact for (y - y_i)^k, k = 0 .. unknowns-1 (maximum
// order, Eq. (diff)); equation k is scaled by s^(deriv-k).
static int compact_row(const double* y, int n, int i, int deriv, qd* Arow, qd* Brow) {
  int lo, hi;
  support(i, n, &lo, &hi);
  int na = 0, nb = hi - lo + 1;
  int acol[8], bcol[8];
  for (int j = lo; j <= hi; ++j) { bcol[j - lo] = j; if (j != i) acol[na++] = j; }
  const int m = na + nb;
  qd M[16 * 16], r[16];
  qd yi = (qd)y[i];
  qd s = fabsq((qd)(i + 2 < n ? y[i + 2] : y[i - 2]) - yi);
  for (int k = 0; k < m; ++k) {
    qd sc = powq(s, (qd)(deriv - k));
    qd fac = deriv == 2 ? (qd)(k * (k - 1)) : (qd)k;
    for (int c = 0; c < na; ++c) {
      qd hj = (qd)y[acol[c]] - yi;
      M[k * m + c] = (k >= deriv) ? -fac * powq(hj, (qd)(k - deriv)) * sc : (qd)0;
    }
    for (int c = 0; c < nb; ++c) {
      qd hj = (qd)y[bcol[c]] - yi;
      M[k * m + na + c] = (k == 0) ? sc : powq(hj, (qd)k) * sc;
    }
    r[k] = (k == deriv) ? fac * sc : (qd)0;
  }
  if (qsolve(m, M, r)) return -3;
  for (int d = 0; d < 7; ++d) { Arow[d] = 0; Brow[d] = 0; }
  Arow[3] = 1;
  for (int c = 0; c < na; ++c) Arow[acol[c] - i + 3] = r[c];
  for (int c = 0; c < nb; ++c) Brow[bcol[c] - i + 3] = r[na + c];
  return 0;
}

// LU without pivoting of a (3,3)-banded matrix given as [n][7] quad bands:
// L(i, i-3..i-1) -> Lq[i*3 + 0..2], U(i, i..i+3) -> Uq[i*4 + 0..3].
static int qband_lu(int n, const qd* M, std::vector<qd>& Lq, std::vector<qd>& Uq) {
  Lq.assign((size_t)n * 3, (qd)0);
  Uq.assign((size_t)n * 4, (qd)0);
  auto m = [&](int i, int j) -> qd { int d = j - i + 3; return (d >= 0 && d < 7) ? M[(size_t)i * 7 + d] : (qd)0; };
  auto u = [&](int k, int j) -> qd { int d = j - k; return (d >= 0 && d <= 3) ? Uq[(size_t)k * 4 + d] : (qd)0; };
  auto l = [&](int i, int j) -> qd { int d = i - j; return (d >= 1 && d <= 3) ? Lq[(size_t)i * 3 + (3 - d)] : (qd)0; };
  for (int i = 0; i < n; ++i) {
    int k0 = i - 3 < 0 ? 0 : i - 3;
    for (int j = k0; j < i; ++j) {
      qd s = m(i, j);
      for (int k = k0; k < j; ++k) s -= l(i, k) * u(k, j);
      if (Uq[(size_t)j * 4] == 0) return -3;
      Lq[(size_t)i * 3 + (3 - (i - j))] = s / Uq[(size_t)j * 4];
    }
    for (int j = i; j <= i + 3 && j < n; ++j) {
      qd s = m(i, j);
      for (int k = k0; k < i; ++k) s -= l(i, k) * u(k, j);
      Uq[(size_t)i * 4 + (j - i)] = s;
    }
    if (Uq[(size_t)i * 4] == 0) return -3;
  }
  return 0;
}

// Packed double LU factors: l(i, i-3..i-1), u(i, i+1..i+3), 1/u(i, i).
static int band_lu(int n, const qd* M, double* lu) {
  std::vector<qd> L, U;
  if (qband_lu(n, M, L, U)) return -3;
  for (int i = 0; i < n; ++i) {
    for (int d = 0; d < 3; ++d) lu[(size_t)i * 7 + d] = (double)L[(size_t)i * 3 + d];
    for (int d = 0; d < 3; ++d) lu[(size_t)i * 7 + 3 + d] = (double)U[(size_t)i * 4 + 1 + d];
    lu[(size_t)i * 7 + 6] = (double)(1 / U[(size_t)i * 4]);
  }
  return 0;
}

// Row r of A^-1 B for banded A, B: w solves A^T w = e_r, then row = B^T w.
static int dense_row(int n, const qd* A, const qd* B, int r, double* out) {
  std::vector<qd> At((size_t)n * 7, (qd)0);
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 7; ++d) {
      int j = i - 3 + d;
      if (j < 0 || j >= n) continue;
      At[(size_t)j * 7 + (i - j + 3)] = A[(size_t)i * 7 + d];  // (A^T)(j, i) = A(i, j)
    }
  std::vector<qd> Lq, Uq;
  if (qband_lu(n, At.data(), Lq, Uq)) return -3;
  std::vector<qd> z(n), w(n);
  for (int i = 0; i < n; ++i) {
    qd s = (i == r) ? (qd)1 : (qd)0;
    for (int k = (i - 3 < 0 ? 0 : i - 3); k < i; ++k) s -= Lq[(size_t)i * 3 + (3 - (i - k))] * z[k];
    z[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    qd s = z[i];
    for (int k = i + 1; k <= i + 3 && k < n; ++k) s -= Uq[(size_t)i * 4 + (k - i)] * w[k];
    w[i] = s / Uq[(size_t)i * 4];
  }
  for (int j = 0; j < n; ++j) {
    qd s = 0;
    for (int i = (j - 3 < 0 ? 0 : j - 3); i <= j + 3 && i < n; ++i) s += B[(size_t)i * 7 + (j - i + 3)] * w[i];
    out[j] = (double)s;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Near-wall mesh optimisation (Appendix B): move the first npts-1 interior
// points of each wall so that the discrete homogeneous Helmholtz solution
// (B - k* A) g = 0, g(-1) = 1, g(+1) = 0 approaches the analytic one, with a
// penalty C |mu - mu_ref| on the displacement; steepest descent with a
// finite-difference gradient and backtracking.  Long double arithmetic.
// ---------------------------------------------------------------------------
typedef long double ld;

static int ld_solve(int m, ld* M, ld* r) {
  for (int c = 0; c < m; ++c) {
    int p = c;
    for (int i = c + 1; i < m; ++i)
      if (fabsl(M[i * m + c]) > fabsl(M[p * m + c])) p = i;
    if (M[p * m + c] == 0) return -3;
    if (p != c) {
      for (int j = 0; j < m; ++j) { ld t = M[c * m + j]; M[c * m + j] = M[p * m + j]; M[p * m + j] = t; }
      ld t = r[c]; r[c] = r[p]; r[p] = t;
    }
    for (int i = c + 1; i < m; ++i) {
      ld f = M[i * m + c] / M[c * m + c];
      for (int j = c; j < m; ++j) M[i * m + j] -= f * M[c * m + j];
      r[i] -= f * r[c];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    ld s = r[i];
    for (int j = i + 1; j < m; ++j) s -= M[i * m + j] * r[j];
    r[i] = s / M[i * m + i];
  }
  return 0;
}

// Second-derivative row i on mesh y (the same equations as compact_row).
static int d2_row_ld(const ld* y, int n, int i, ld* Arow, ld* Brow) {
  int lo, hi;
  support(i, n, &lo, &hi);
  int na = 0, nb = hi - lo + 1, acol[8], bcol[8];
  for (int j = lo; j <= hi; ++j) { bcol[j - lo] = j; if (j != i) acol[na++] = j; }
  const int m = na + nb;
  ld M[16 * 16], r[16];
  const ld s = fabsl((i + 2 < n ? y[i + 2] : y[i - 2]) - y[i]);
  for (int k = 0; k < m; ++k) {
    const ld sc = powl(s, (ld)(2 - k));
    const ld fac = (ld)(k * (k - 1));
    for (int c = 0; c < na; ++c) M[k * m + c] = k >= 2 ? -fac * powl(y[acol[c]] - y[i], (ld)(k - 2)) * sc : (ld)0;
    for (int c = 0; c < nb; ++c) M[k * m + na + c] = k == 0 ? sc : powl(y[bcol[c]] - y[i], (ld)k) * sc;
    r[k] = k == 2 ? fac * sc : (ld)0;
  }
  if (ld_solve(m, M, r)) return -3;
  for (int d = 0; d < 7; ++d) { Arow[d] = 0; Brow[d] = 0; }
  Arow[3] = 1;
  for (int c = 0; c < na; ++c) Arow[acol[c] - i + 3] = r[c];
  for (int c = 0; c < nb; ++c) Brow[bcol[c] - i + 3] = r[na + c];
  return 0;
}

// |g - g_ana|_2 over the mesh for (B - k* A) g = 0, g(-1) = 1, g(+1) = 0.
static ld helm_error(const ld* y, int n, const ld* A, const ld* B, ld kstar) {
  std::vector<ld> M((size_t)n * 7, 0), L((size_t)n * 3, 0), U((size_t)n * 4, 0), z(n), g(n);
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 7; ++d)
      M[(size_t)i * 7 + d] = (i == 0 || i == n - 1) ? (d == 3 ? 1 : 0) : B[(size_t)i * 7 + d] - kstar * A[(size_t)i * 7 + d];
  auto m = [&](int i, int j) -> ld { int d = j - i + 3; return (d >= 0 && d < 7) ? M[(size_t)i * 7 + d] : (ld)0; };
  auto u = [&](int k, int j) -> ld { int d = j - k; return (d >= 0 && d <= 3) ? U[(size_t)k * 4 + d] : (ld)0; };
  auto l = [&](int i, int j) -> ld { int d = i - j; return (d >= 1 && d <= 3) ? L[(size_t)i * 3 + (3 - d)] : (ld)0; };
  for (int i = 0; i < n; ++i) {
    const int k0 = i - 3 < 0 ? 0 : i - 3;
    for (int j = k0; j < i; ++j) {
      ld s = m(i, j);
      for (int k = k0; k < j; ++k) s -= l(i, k) * u(k, j);
      L[(size_t)i * 3 + (3 - (i - j))] = s / U[(size_t)j * 4];
    }
    for (int j = i; j <= i + 3 && j < n; ++j) {
      ld s = m(i, j);
      for (int k = k0; k < i; ++k) s -= l(i, k) * u(k, j);
      U[(size_t)i * 4 + (j - i)] = s;
    }
  }
  for (int i = 0; i < n; ++i) {
    ld s = i == 0 ? 1 : 0;
    for (int k = (i - 3 < 0 ? 0 : i - 3); k < i; ++k) s -= l(i, k) * z[k];
    z[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    ld s = z[i];
    for (int k = i + 1; k <= i + 3 && k < n; ++k) s -= u(i, k) * g[k];
    g[i] = s / U[(size_t)i * 4];
  }
  const ld r = sqrtl(kstar);
  ld e = 0;
  for (int i = 0; i < n; ++i) {
    const ld ana = expl(-r * (y[i] + 1)) * (1 - expl(-2 * r * (1 - y[i]))) / (1 - expl(-4 * r));
    e += (g[i] - ana) * (g[i] - ana);
  }
  return sqrtl(e);
}

int chanh_optimize_mesh(int ny, const double* y_in, double kstar, int npts, double C, int iters, double* y_out,
                        double* err_before, double* err_after) {
  if (ny < 9 || ny % 2 == 0 || !(kstar > 0)) return -1;
  const int h = (ny - 1) / 2;
  if (npts > h - 3) npts = h - 3;
  if (npts < 2) npts = 2;
  std::vector<ld> y(y_in, y_in + ny), A((size_t)ny * 7), B((size_t)ny * 7);
  for (int i = 0; i < ny; ++i)
    if (d2_row_ld(y.data(), ny, i, &A[(size_t)i * 7], &B[(size_t)i * 7])) return -3;
  const std::vector<ld> mu_ref(y.begin(), y.begin() + npts);
  auto apply = [&](const std::vector<ld>& mu) {   // move points 1..npts-1 and their mirrors, refresh rows
    for (int j = 1; j < npts; ++j) { y[j] = mu[j]; y[ny - 1 - j] = -mu[j]; }
    for (int i = 0; i < npts + 3; ++i) {
      d2_row_ld(y.data(), ny, i, &A[(size_t)i * 7], &B[(size_t)i * 7]);
      d2_row_ld(y.data(), ny, ny - 1 - i, &A[(size_t)(ny - 1 - i) * 7], &B[(size_t)(ny - 1 - i) * 7]);
    }
  };
  auto loss = [&](const std::vector<ld>& mu) {
    for (int j = 1; j < npts + 1 && j < ny; ++j)
      if (!(mu[j - 1] < (j < npts ? mu[j] : y[npts]))) return (ld)1e30L;   // keep the mesh ordered
    // Keep every moved cell within a factor of two of its starting size: the optimal grid
    // only slightly changes the near-wall spacing, and without such a bound the functional
    // is lowest where the first cell collapses onto the wall (at Re_tau 2000, Ny 513 the
    // descent shrank it to 0.3 % of its size; the size penalty C does not prevent it).
    for (int j = 1; j <= npts && j < ny; ++j) {
      const ld c = (j < npts ? mu[j] : y[npts]) - mu[j - 1];
      const ld c0 = (j < npts ? mu_ref[j] : y[npts]) - mu_ref[j - 1];
      if (!(c >= 0.5L * c0 && c <= 2 * c0)) return (ld)1e30L;
    }
    apply(mu);
    ld pen = 0;
    for (int j = 1; j < npts; ++j) pen += (mu[j] - mu_ref[j]) * (mu[j] - mu_ref[j]);
    return helm_error(y.data(), ny, A.data(), B.data(), (ld)kstar) + (ld)C * sqrtl(pen);
  };
  std::vector<ld> mu = mu_ref;
  ld f = loss(mu);
  if (err_before) *err_before = (double)helm_error(y.data(), ny, A.data(), B.data(), (ld)kstar);
  std::vector<ld> grad(npts), trial(npts);
  for (int it = 0; it < iters; ++it) {
    ld gnorm = 0;
    for (int j = 1; j < npts; ++j) {
      const ld dj = 1e-7L * (mu[j + 1 < npts ? j + 1 : j] - mu[j - 1]);
      trial = mu;
      trial[j] += dj;
      const ld fp = loss(trial);
      trial[j] = mu[j] - dj;
      const ld fm = loss(trial);
      grad[j] = (fp - fm) / (2 * dj);
      gnorm += grad[j] * grad[j];
    }
    gnorm = sqrtl(gnorm);
    if (!(gnorm > 0)) break;
    ld step = 0.2L * (mu_ref[1] - mu_ref[0]) / gnorm;   // first trial: move the points by up to 20 % of the wall cell
    bool improved = false;
    for (int ls = 0; ls < 40; ++ls, step *= 0.5L) {
      for (int j = 0; j < npts; ++j) trial[j] = j == 0 ? mu[0] : mu[j] - step * grad[j];
      const ld ft = loss(trial);
      if (ft < f) { mu = trial; f = ft; improved = true; break; }
    }
    if (!improved) break;
  }
  loss(mu);
  if (err_after) *err_after = (double)helm_error(y.data(), ny, A.data(), B.data(), (ld)kstar);
  for (int i = 0; i < ny; ++i) y_out[i] = (double)y[i];
  return 0;
}

int chanh_build(int ny, double grid_re, double eta_w, chanh_tables* t) { return chanh_build_mesh(ny, grid_re, eta_w, nullptr, t); }

int chanh_build_mesh(int ny, double grid_re, double eta_w, const double* mesh, chanh_tables* t) {
  std::memset(t, 0, sizeof(*t));
  if (ny < 9 || (ny % 2) != 1) return -1;
  t->ny = ny;
  double** bufs[] = {&t->y, &t->A2, &t->B2, &t->A1, &t->B1, &t->lu1, &t->lu2f, &t->d0, &t->dN, &t->wq};
  size_t sizes[] = {1, 7, 7, 7, 7, 7, 7, 1, 1, 1};
  for (int b = 0; b < 10; ++b) {
    *bufs[b] = (double*)std::calloc((size_t)ny * sizes[b], sizeof(double));
    if (!*bufs[b]) { chanh_free(t); return -2; }
  }
  if (mesh) std::memcpy(t->y, mesh, (size_t)ny * sizeof(double));
  else if (chanh_ygrid(ny, grid_re, eta_w, t->y)) { chanh_free(t); return -1; }
  std::vector<qd> qA2((size_t)ny * 7), qB2((size_t)ny * 7), qA1((size_t)ny * 7), qB1((size_t)ny * 7);
  for (int i = 0; i < ny; ++i) {
    if (compact_row(t->y, ny, i, 2, &qA2[(size_t)i * 7], &qB2[(size_t)i * 7]) ||
        compact_row(t->y, ny, i, 1, &qA1[(size_t)i * 7], &qB1[(size_t)i * 7])) { chanh_free(t); return -3; }
  }
  for (size_t k = 0; k < (size_t)ny * 7; ++k) {
    t->A2[k] = (double)qA2[k]; t->B2[k] = (double)qB2[k];
    t->A1[k] = (double)qA1[k]; t->B1[k] = (double)qB1[k];
  }
  if (band_lu(ny, qA1.data(), t->lu1) || band_lu(ny, qA2.data(), t->lu2f) ||
      dense_row(ny, qA1.data(), qB1.data(), 0, t->d0) || dense_row(ny, qA1.data(), qB1.data(), ny - 1, t->dN)) {
    chanh_free(t);
    return -3;
  }
  for (int j = 0; j + 1 < ny; ++j) {
    double dy = t->y[j + 1] - t->y[j];
    t->wq[j] += 0.5 * dy;
    t->wq[j + 1] += 0.5 * dy;
  }
  return 0;
}

void chanh_free(chanh_tables* t) {
  double** bufs[] = {&t->y, &t->A2, &t->B2, &t->A1, &t->B1, &t->lu1, &t->lu2f, &t->d0, &t->dN, &t->wq};
  for (auto b : bufs) { std::free(*b); *b = nullptr; }
}

void chanh_twiddles(int L, double* tw) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int t = 0; t < L; ++t) {
    long double a = -2.0L * pi * (long double)t / (long double)L;
    tw[2 * t] = (double)cosl(a);
    tw[2 * t + 1] = (double)sinl(a);
  }
}

// Radix order of the decimation-in-frequency transforms: a radix-3 stage first
// (it carries the zero middle third of a 3/2-padded spectrum), then the other
// threes, fours and at most one two.  The decimation-in-time transforms run the
// same list backwards.
int chanh_radix_plan(int L, int* radix) {
  int n = 0, r = L;
  if (r % 3 != 0) return -1;
  while (r % 3 == 0) { radix[n++] = 3; r /= 3; }
  while (r % 4 == 0) { radix[n++] = 4; r /= 4; }
  while (r % 2 == 0) { radix[n++] = 2; r /= 2; }
  if (r != 1 || n > 16) return -1;
  return n;
}
