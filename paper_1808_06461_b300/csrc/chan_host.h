// Host-side set-up tables of the channel library (internal header).
#pragma once
#ifdef __cplusplus
extern "C" {
#endif

// Banded operators are stored row-major as [ny][7]: entry d of row i is the
// coefficient of column i - 3 + d (zero outside the row's stencil).
// LU factors of a (3,3)-banded matrix without pivoting are packed as
// [ny][7]: l(i, i-3..i-1), u(i, i+1..i+3), 1/u(i, i).
typedef struct chanh_tables {
  int ny;
  double* y;     // mesh
  double* A2;    // second derivative:  A2 f'' = B2 f
  double* B2;
  double* A1;    // first derivative:   A1 f' = B1 f
  double* B1;
  double* lu1;   // LU of A1 (all rows)
  double* lu2f;  // LU of A2 (all rows)
  double* d0;    // row 0 of A1^-1 B1 (dv/dy at y = -1 as a dot product), [ny]
  double* dN;    // row ny-1 of A1^-1 B1, [ny]
  double* wq;    // trapezoid weights of the flux integral, [ny]
} chanh_tables;

// Build every table for an ny-point mesh clustered for grid_re (returns 0,
// or -1 for bad arguments, -2 for allocation failure, -3 when a pivot of a
// coefficient system or an LU vanishes).
int chanh_build(int ny, double grid_re, double eta_w, chanh_tables* t);
void chanh_free(chanh_tables* t);
// Same, on a given mesh (double[ny], increasing, mirror symmetric) instead of the formula.
int chanh_build_mesh(int ny, double grid_re, double eta_w, const double* mesh, chanh_tables* t);

// Near-wall mesh optimisation of Appendix B (see setup_host.cpp).  y_in: the
// starting mesh; kstar: the Helmholtz modified wavenumber to fit; npts: mesh
// points per wall in the optimisation (the wall point stays; each moved cell stays
// within a factor of two of its starting size); C: displacement penalty; iters:
// steepest-descent iterations.  Writes the mesh to y_out and
// the Helmholtz errors before and after.  Returns 0, or < 0 on bad input.
int chanh_optimize_mesh(int ny, const double* y_in, double kstar, int npts, double C, int iters, double* y_out,
                        double* err_before, double* err_after);

// The same mesh formula as the tables use (double[ny]).
int chanh_ygrid(int ny, double grid_re, double eta_w, double* y);

// Twiddles w_t = exp(-2 pi i t / L), t = 0..L-1, interleaved (re, im).
void chanh_twiddles(int L, double* tw);

// Radix plan of a 3^a 2^b length (a >= 1) in decimation-in-frequency order:
// 3s first, then 4s, then at most one 2.  Returns the number of stages (<= 16)
// or -1 if L is not of that form.
int chanh_radix_plan(int L, int* radix);

#ifdef __cplusplus
}
#endif
