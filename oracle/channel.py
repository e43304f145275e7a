"""Plain FP64 oracle of one RK3 substep of the v - omega_2 channel DNS.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by tests,
the smoke check and the CPU-baseline leg of the benchmark, never by the
library.

Paper: Vela-Martin, Encinar, Garcia-Gutierrez & Jimenez, "A low-storage
method consistent with second-order statistics for time-resolved databases
of turbulent channel flow up to Re_tau = 5300" (arXiv:1808.06461).

Conventions (readings of the paper, each listed in the design notes):
  * walls at y = -1 and y = +1 (the paper's x_2 = 0, 2h with h = 1);
    nu = 1 / Re_tau, so lengths are in h and velocities in u_tau;
  * N_1 and N_3 are collocation points (Sec. 2.1); stored modes are
    kx = 0 .. N1/2-1 and kz in FFT order with the kz Nyquist held at zero;
  * synthesis u(x, z) = sum_k u_k exp(+i(k1 x + k3 z)); analysis on the
    3/2-padded grid divides by its point count;
  * Fourier fields are complex arrays of shape (Ny, Nz, Nx/2), [j, jz, kx].
"""
import functools
import math

import mpmath
import numpy as np

# Low-storage semi-implicit RK3 of Spalart, Moser & Rogers (1991), the
# scheme Appendix A cites for Eqs. (chi1)-(psi).  Per substep:
# (gamma, zeta, alpha, beta); alpha + beta = gamma + zeta.
RK3 = ((8.0 / 15.0, 0.0, 29.0 / 96.0, 37.0 / 160.0),
       (5.0 / 12.0, -17.0 / 60.0, -3.0 / 40.0, 5.0 / 24.0),
       (3.0 / 4.0, -5.0 / 12.0, 1.0 / 6.0, 1.0 / 6.0))


# --------------------------------------------------------------------------
# Wall-normal grid and compact finite differences (Sec. 2.1, Appendix B)
# --------------------------------------------------------------------------

def ygrid(ny, re_tau, eta_w=1.0, kappa=0.4):
    """Wall-normal mesh with spacing proportional to a local Kolmogorov scale.

    Sec. 2.1 asks for a non-uniform mesh of N_2 points keeping roughly
    constant resolution in local Kolmogorov units, without a formula.
    Reading: dy+/dj = C eta+(y+) with eta+ = (eta_w^4 + kappa y+)^(1/4)
    (eta_w at the wall, (kappa y+)^(1/4) in the log layer).  Integrating,
    j(y+) = (4 / (3 kappa C)) [(eta_w^4 + kappa y+)^(3/4) - eta_w^3]; C makes
    the half channel span (ny - 1) / 2 intervals.  The upper half mirrors the
    lower half exactly.
    """
    if ny % 2 != 1 or ny < 9:
        raise ValueError("ny must be odd and >= 9")
    h = (ny - 1) // 2
    c = (4.0 / (3.0 * kappa)) * ((eta_w ** 4 + kappa * re_tau) ** 0.75 - eta_w ** 3) / h
    y = np.empty(ny)
    for j in range(h):
        yp = ((3.0 * kappa * c * j / 4.0 + eta_w ** 3) ** (4.0 / 3.0) - eta_w ** 4) / kappa
        y[j] = -1.0 + yp / re_tau
    y[h] = 0.0
    for j in range(h + 1, ny):
        y[j] = -y[ny - 1 - j]
    return y


def _support(i, n):
    """Stencil columns of row i: seven points inside, reduced at the walls.

    Appendix B: seven-point stencils, "reduced progressively" at the corner
    points.  Reading: rows 0, 1, 2 use columns [0, i+3] (and mirrored at the
    top wall), for both A and B.
    """
    ii = min(i, n - 1 - i)
    if ii >= 3:
        return i - 3, i + 3
    if i == ii:
        return 0, ii + 3
    return n - 1 - (ii + 3), n - 1


@functools.lru_cache(maxsize=16)
def _compact_coeffs_cached(ybytes, deriv):
    y = np.frombuffer(ybytes, dtype=np.float64)
    n = y.size
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    with mpmath.workdps(50):
        for i in range(n):
            lo, hi = _support(i, n)
            cols = list(range(lo, hi + 1))
            acols = [j for j in cols if j != i]
            m = len(acols) + len(cols)
            hs = [mpmath.mpf(float(y[j])) - mpmath.mpf(float(y[i])) for j in cols]
            ha = [mpmath.mpf(float(y[j])) - mpmath.mpf(float(y[i])) for j in acols]
            s = abs(mpmath.mpf(float(y[i + 2] if i + 2 < n else y[i - 2])) - mpmath.mpf(float(y[i])))
            M = mpmath.matrix(m, m)
            r = mpmath.matrix(m, 1)
            for k in range(m):
                # Eq. (diff): sum_j B_ij h^k - [k!/(k-deriv)!] sum_j A_ij h^(k-deriv) = 0,
                # with A_ii = 1 moved to the right-hand side; each equation is
                # premultiplied by s^(deriv-k) (the paper's conditioning step).
                sc = s ** (deriv - k)
                fac = k * (k - 1) if deriv == 2 else k
                for c_, hj in enumerate(ha):
                    M[k, c_] = -fac * hj ** (k - deriv) * sc if k >= deriv else 0
                for c_, hj in enumerate(hs):
                    M[k, len(ha) + c_] = hj ** k * sc
                r[k] = (fac * sc) if k == deriv else 0
            x = mpmath.lu_solve(M, r)
            A[i, i] = 1.0
            for c_, j in enumerate(acols):
                A[i, j] = float(x[c_])
            for c_, j in enumerate(cols):
                B[i, j] = float(x[len(acols) + c_])
    A.setflags(write=False)
    B.setflags(write=False)
    return A, B


def compact_coeffs(y, deriv):
    """Banded (A, B) with A d^deriv f = B f, maximum order per row (Appendix B, Eq. (diff)).

    Reading of the garbled Eq. (diff): A_ii = 1; the remaining A and B
    coefficients of the row's stencil are the unique solution that makes the
    relation exact for f = (y - y_i)^k, k = 0 .. (number of unknowns - 1):
    12 for the seven-point interior rows.  The first-derivative pair
    (deriv = 1) is built the same way.  Solved in 50-digit arithmetic.
    """
    y = np.ascontiguousarray(y, dtype=np.float64)
    return _compact_coeffs_cached(y.tobytes(), int(deriv))


# --------------------------------------------------------------------------
# Problem set-up
# --------------------------------------------------------------------------

class Setup:
    """Grid, operators and wavenumbers of one channel box (Sec. 2.1).

    ``grid_re`` (default Re_tau) is the Reynolds number the wall-normal mesh
    is clustered for; ``mesh`` replaces the formula by a given mesh (e.g. the
    Appendix B optimised one); nu = 1 / re_tau always.
    """

    def __init__(self, re_tau, Lx, Lz, Nx, Ny, Nz, dt, eta_w=1.0, grid_re=None, mesh=None):
        if Nx % 2 or Nz % 2:
            raise ValueError("Nx and Nz must be even")
        self.re_tau, self.Lx, self.Lz = float(re_tau), float(Lx), float(Lz)
        self.Nx, self.Ny, self.Nz, self.dt = int(Nx), int(Ny), int(Nz), float(dt)
        self.nu = 1.0 / self.re_tau
        self.nxh = self.Nx // 2
        self.Lx3, self.Lz3 = 3 * self.Nx // 2, 3 * self.Nz // 2
        if mesh is not None:
            self.y = np.array(mesh, dtype=np.float64)
        else:
            self.y = ygrid(self.Ny, self.re_tau if grid_re is None else float(grid_re), eta_w)
        self.A2, self.B2 = compact_coeffs(self.y, 2)
        self.A1, self.B1 = compact_coeffs(self.y, 1)
        self.D1 = np.linalg.solve(self.A1, self.B1)
        self.D2 = np.linalg.solve(self.A2, self.B2)
        k1 = 2.0 * math.pi / self.Lx * np.arange(self.nxh)
        kzi = np.array([j if j < self.Nz // 2 else j - self.Nz for j in range(self.Nz)])
        k3 = 2.0 * math.pi / self.Lz * kzi
        self.K1 = np.broadcast_to(k1[None, :], (self.Nz, self.nxh)).copy()
        self.K3 = np.broadcast_to(k3[:, None], (self.Nz, self.nxh)).copy()
        self.K2 = self.K1 ** 2 + self.K3 ** 2
        self.keep = np.ones((self.Nz, self.nxh), dtype=bool)
        self.keep[self.Nz // 2, :] = False            # kz Nyquist held at zero
        dy = np.diff(self.y)
        self.wq = np.zeros(self.Ny)                   # trapezoid weights for the flux
        self.wq[:-1] += 0.5 * dy
        self.wq[1:] += 0.5 * dy

    def flux(self, U):
        """Mass flux per unit span, trapezoid rule on the mesh."""
        return float(self.wq @ U)


def apply_y(M, F):
    """Apply an Ny x Ny matrix along the wall-normal axis of a field stack."""
    return np.tensordot(M, F, axes=(1, 0))


# --------------------------------------------------------------------------
# Fourier transforms with 3/2 zero padding (Sec. 2.1)
# --------------------------------------------------------------------------

def to_physical(st, F):
    """Fourier (Ny, Nz, Nx/2) -> real values on the padded (Ny, 3Nz/2, 3Nx/2) grid.

    Zero padding to 3N/2 points per direction (the 3/2 rule of Canuto et al.
    cited in Sec. 2.1); kx > 0 modes stand for themselves and their
    conjugates, and the real part of each kx = 0 coefficient is used.
    """
    hz = st.Nz // 2
    G = np.zeros((F.shape[0], st.Lz3, st.Lx3 // 2 + 1), dtype=np.complex128)
    G[:, :hz, :st.nxh] = F[:, :hz, :]
    G[:, st.Lz3 - (hz - 1):, :st.nxh] = F[:, hz + 1:, :]
    G = np.fft.ifft(G, axis=1) * st.Lz3
    return np.fft.irfft(G, n=st.Lx3, axis=2) * st.Lx3


def to_fourier(st, u):
    """Padded physical grid -> retained Fourier modes (truncation = dealiasing)."""
    hz = st.Nz // 2
    G = np.fft.rfft(u, axis=2) / st.Lx3
    G = np.fft.fft(G, axis=1) / st.Lz3
    F = np.zeros((u.shape[0], st.Nz, st.nxh), dtype=np.complex128)
    F[:, :hz, :] = G[:, :hz, :st.nxh]
    F[:, hz + 1:, :] = G[:, st.Lz3 - (hz - 1):, :st.nxh]
    return F


# --------------------------------------------------------------------------
# State
# --------------------------------------------------------------------------

def initial_state(st, v, omega2, U1, U3):
    """State at the start of an RK3 step from (v, omega_2, U_1, U_3).

    chi = Lap v = (D2 - k^2) v with D2 = A^-1 B over all rows (Appendix A
    evolves chi).  The target mass flux is the initial one (Sec. 2.1: a
    constant mass flux is imposed).
    """
    v = np.array(v, dtype=np.complex128) * st.keep
    om = np.array(omega2, dtype=np.complex128) * st.keep
    v[:, 0, 0] = 0.0
    om[:, 0, 0] = 0.0
    chi = apply_y(st.D2, v) - st.K2 * v
    z = np.zeros_like(v)
    U1 = np.array(U1, dtype=np.float64)
    U3 = np.array(U3, dtype=np.float64)
    return dict(v=v, omega2=om, chi=chi, U1=U1, U3=U3,
                Nchi_prev=z.copy(), Nom_prev=z.copy(),
                H1m_prev=np.zeros(st.Ny), H3m_prev=np.zeros(st.Ny),
                Q0=st.flux(U1), f=0.0, s=0, t=0.0)


def velocities(st, S):
    """u_1, u_3 from omega_2 and d v/dy; d u_1/dy, d u_3/dy (Appendix C order).

    Continuity i k1 u1 + dv/dy + i k3 u3 = 0 and omega_2 = i k3 u1 - i k1 u3
    give u1 = i (k1 dv - k3 omega_2) / k^2, u3 = i (k3 dv + k1 omega_2) / k^2.
    The (0, 0) mode carries the mean profiles U_1, U_3.
    """
    v, om = S["v"], S["omega2"]
    dv = apply_y(st.D1, v)
    k2 = np.where(st.K2 > 0, st.K2, 1.0)
    u1 = 1j * (st.K1 * dv - st.K3 * om) / k2
    u3 = 1j * (st.K3 * dv + st.K1 * om) / k2
    u1[:, 0, 0] = S["U1"]
    u3[:, 0, 0] = S["U3"]
    u1 *= st.keep
    u3 *= st.keep
    du1 = apply_y(st.D1, u1)
    du3 = apply_y(st.D1, u3)
    return u1, v, u3, du1, dv, du3


def vorticity(st, S, u1, v, u3, du1, du3):
    """omega = curl u in Fourier space: omega_1 = du3/dy - i k3 v, omega_3 = i k1 v - du1/dy."""
    om1 = du3 - 1j * st.K3 * v
    om3 = 1j * st.K1 * v - du1
    return om1, S["omega2"], om3


def nonlinear(st, S):
    """Fourier coefficients of H = u x omega (Appendix A), dealiased."""
    u1, v, u3, du1, dv, du3 = velocities(st, S)
    om1, om2, om3 = vorticity(st, S, u1, v, u3, du1, du3)
    p = [to_physical(st, F) for F in (u1, v, u3, om1, om2, om3)]
    u, w = p[:3], p[3:]
    H1 = u[1] * w[2] - u[2] * w[1]
    H2 = u[2] * w[0] - u[0] * w[2]
    H3 = u[0] * w[1] - u[1] * w[0]
    return to_fourier(st, H1), to_fourier(st, H2), to_fourier(st, H3)


def rhs_terms(st, H1, H2, H3):
    """Eq. (hghv): N_chi = -d/dy(i k1 H1 + i k3 H3) - k^2 H2, N_omega2 = i k3 H1 - i k1 H3."""
    Nchi = -apply_y(st.D1, 1j * st.K1 * H1 + 1j * st.K3 * H3) - st.K2 * H2
    Nom = 1j * st.K3 * H1 - 1j * st.K1 * H3
    return Nchi * st.keep, Nom * st.keep


# --------------------------------------------------------------------------
# Implicit wall-normal solves (Appendix A, Eqs. (chi1), (chi2), (psi))
# --------------------------------------------------------------------------

def _dirichlet_solve(lhs, rhs):
    """Solve stacked dense systems whose rows 0 and Ny-1 become identity rows.

    lhs: (M, Ny, Ny) real, rhs: (M, Ny, R) real.
    """
    L = lhs.copy()
    L[:, 0, :] = 0.0
    L[:, -1, :] = 0.0
    L[:, 0, 0] = 1.0
    L[:, -1, -1] = 1.0
    return np.linalg.solve(L, rhs)


def _modes(F):
    """(Ny, Nz, nxh) -> (M, Ny) with M = Nz * nxh."""
    return F.reshape(F.shape[0], -1).T


def _unmodes(X, shape):
    return X.T.reshape(shape)


def implicit_step(st, S, Nchi, Nom, s, chunk=512):
    """omega_2 and chi/v implicit steps with the influence-matrix correction.

    Each equation is multiplied by A, using A D2 = B, so interior rows read
      [(1 + b dt nu k^2) A - b dt nu B] X+ = A[(1 - a dt nu k^2) X + dt(g N + z Nprev)] + a dt nu B X,
    the semi-implicit RK3 step (chi1)/(psi) with Lap = D2 - k^2 and
    (g, z, a, b) = (gamma, zeta, alpha, beta) of substep s.  omega_2+ = 0 at
    both walls.  For chi the particular solution has chi_p(+-1) = 0; then
    (B - k^2 A) v_p = A chi_p with v_p(+-1) = 0 (Eq. (chi2)); homogeneous
    solutions chi_a (= 1 at y = -1), chi_b (= 1 at y = +1) and their v_a,
    v_b are combined so that dv/dy = 0 at both walls (Kim, Moin & Moser 1987,
    as Appendix A describes).
    """
    g, z, a, b = RK3[s]
    dt, nu, ny = st.dt, st.nu, st.Ny
    shape = S["v"].shape
    k2 = st.K2.reshape(-1)
    A, B = st.A2, st.B2

    def rhs(X, N, Np):
        inner = X * (1.0 - a * dt * nu * st.K2) + dt * (g * N + z * Np)
        r = apply_y(A, inner) + a * dt * nu * apply_y(B, X)
        r[0] = 0.0
        r[-1] = 0.0
        return r

    r_om = _modes(rhs(S["omega2"], Nom, S["Nom_prev"]))
    r_chi = _modes(rhs(S["chi"], Nchi, S["Nchi_prev"]))
    om_new = np.empty_like(r_om)
    chi_new = np.empty_like(r_chi)
    v_new = np.empty_like(r_chi)
    M = k2.size
    e0 = np.zeros(ny)
    e0[0] = 1.0
    eN = np.zeros(ny)
    eN[-1] = 1.0
    d0, dN = st.D1[0], st.D1[-1]
    for m0 in range(0, M, chunk):
        m1 = min(M, m0 + chunk)
        kk = k2[m0:m1, None, None]
        helm = (1.0 + b * dt * nu * kk) * A[None] - b * dt * nu * B[None]
        pois = B[None] - kk * A[None]
        # omega_2 and the particular chi: real and imaginary parts as separate right-hand sides
        rr = np.stack([r_om[m0:m1].real, r_om[m0:m1].imag, r_chi[m0:m1].real, r_chi[m0:m1].imag,
                       np.broadcast_to(e0, (m1 - m0, ny)), np.broadcast_to(eN, (m1 - m0, ny))], axis=2)
        sol = _dirichlet_solve(helm, rr)
        om_new[m0:m1] = sol[:, :, 0] + 1j * sol[:, :, 1]
        chi_p = sol[:, :, 2] + 1j * sol[:, :, 3]
        chi_a = sol[:, :, 4]
        chi_b = sol[:, :, 5]
        # Poisson solves (B - k^2 A) v = A chi, v(+-1) = 0
        src = np.stack([chi_p.real, chi_p.imag, chi_a, chi_b], axis=2)
        prhs = np.einsum("ij,mjr->mir", A, src)
        prhs[:, 0, :] = 0.0
        prhs[:, -1, :] = 0.0
        vs = _dirichlet_solve(pois, prhs)
        v_p = vs[:, :, 0] + 1j * vs[:, :, 1]
        v_a = vs[:, :, 2]
        v_b = vs[:, :, 3]
        # influence matrix: (D1 v)(+-1) = 0
        g11, g12 = v_a @ d0, v_b @ d0
        g21, g22 = v_a @ dN, v_b @ dN
        p0, pN = v_p @ d0, v_p @ dN
        det = g11 * g22 - g12 * g21
        ca = -(g22 * p0 - g12 * pN) / det
        cb = -(-g21 * p0 + g11 * pN) / det
        v_new[m0:m1] = v_p + ca[:, None] * v_a + cb[:, None] * v_b
        chi_new[m0:m1] = chi_p + ca[:, None] * chi_a + cb[:, None] * chi_b
    return (_unmodes(om_new, shape) * st.keep, _unmodes(chi_new, shape) * st.keep,
            _unmodes(v_new, shape) * st.keep)


def mean_flow_step(st, S, H1m, H3m, s):
    """Mean profiles U_1, U_3 (Sec. 2.1, Appendix A) with constant mass flux.

    Interior rows: (A - b dt nu B) U+ = A[U + dt(g <H> + z <H>prev)] + a dt nu B U,
    U+(+-1) = 0.  For U_1 the pressure-gradient correction c U_h is added,
    U_h solving (A - b dt nu B) U_h = A 1, U_h(+-1) = 0, with c fixed by
    flux(U_1+) = Q0 (trapezoid flux).  Returns (U1+, U3+, f) with
    f = c / ((a + b) dt) the mean pressure gradient of the substep.
    """
    g, z, a, b = RK3[s]
    dt, nu = st.dt, st.nu
    A, B = st.A2, st.B2
    L = A - b * dt * nu * B
    L[0, :] = 0.0
    L[-1, :] = 0.0
    L[0, 0] = 1.0
    L[-1, -1] = 1.0

    def adv(U, Hm, Hp):
        r = A @ (U + dt * (g * Hm + z * Hp)) + a * dt * nu * (B @ U)
        r[0] = 0.0
        r[-1] = 0.0
        return np.linalg.solve(L, r)

    U1s = adv(S["U1"], H1m, S["H1m_prev"])
    U3n = adv(S["U3"], H3m, S["H3m_prev"])
    r = A @ np.ones(st.Ny)
    r[0] = 0.0
    r[-1] = 0.0
    Uh = np.linalg.solve(L, r)
    c = (S["Q0"] - st.flux(U1s)) / st.flux(Uh)
    return U1s + c * Uh, U3n, c / ((a + b) * dt)


def substep(st, S):
    """One RK3 substep (Appendix A; operation order of Appendix C's table)."""
    s = S["s"] % 3
    H1, H2, H3 = nonlinear(st, S)
    Nchi, Nom = rhs_terms(st, H1, H2, H3)
    om, chi, v = implicit_step(st, S, Nchi, Nom, s)
    H1m = H1[:, 0, 0].real.copy()
    H3m = H3[:, 0, 0].real.copy()
    U1, U3, f = mean_flow_step(st, S, H1m, H3m, s)
    g, z, a, b = RK3[s]
    return dict(v=v, omega2=om, chi=chi, U1=U1, U3=U3, Nchi_prev=Nchi, Nom_prev=Nom,
                H1m_prev=H1m, H3m_prev=H3m, Q0=S["Q0"], f=f, s=S["s"] + 1,
                t=S["t"] + (a + b) * st.dt)


def run(st, S, nsub):
    for _ in range(nsub):
        S = substep(st, S)
    return S


# --------------------------------------------------------------------------
# Filter and filtered stresses (Sec. 3.1)
# --------------------------------------------------------------------------

SHARP, BOX = 0, 1


def filter_transfer(st, kind, p1, p3):
    """Filter transfer function G(k1, k3) on the stored modes.

    SHARP (Eq. (fou_fil)): G = 1 if |k1| < k1c and |k3| < k3c, else 0, with
    k_c = pi / l_c and l_c = p / Re_tau (p1, p3 are l_c^+; the paper's
    database uses 120 and 60).  BOX: the top-hat of widths Delta = p / Re_tau
    applied to the trigonometric interpolant, G = sinc(k1 D1 / 2) sinc(k3 D3 / 2).
    """
    if kind == SHARP:
        k1c = math.pi * st.re_tau / p1
        k3c = math.pi * st.re_tau / p3
        G = ((np.abs(st.K1) < k1c) & (np.abs(st.K3) < k3c)).astype(np.float64)
    elif kind == BOX:
        d1, d3 = p1 / st.re_tau, p3 / st.re_tau
        G = np.sinc(st.K1 * d1 / (2 * math.pi)) * np.sinc(st.K3 * d3 / (2 * math.pi))
    else:
        raise ValueError("unknown filter kind")
    return G * st.keep


PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def filter_stresses(st, S, kind, p1, p3):
    """Filtered velocities and tau_ij = filt(u_i u_j) - ubar_i ubar_j (Sec. 3.1).

    filt(u_i u_j) = G . P(u_i u_j), P the dealiased projection on the stored
    modes; ubar_i ubar_j is the dealiased product of the filtered velocities.
    (The printed tau_ij = filt(u_i u_j) - ubar_j ubar_j is read as ubar_i ubar_j.)
    Returns ubar (3, Ny, Nz, Nx/2) and tau (6, ...) in PAIRS order
    (11, 22, 33, 12, 13, 23).
    """
    G = filter_transfer(st, kind, p1, p3)
    u1, v, u3, _, _, _ = velocities(st, S)
    u = [u1, v, u3]
    ub = [G * f for f in u]
    pu = [to_physical(st, f) for f in u]
    pb = [to_physical(st, f) for f in ub]
    tau = []
    for i, j in PAIRS:
        tau.append(G * to_fourier(st, pu[i] * pu[j]) - to_fourier(st, pb[i] * pb[j]))
    return np.stack(ub), np.stack(tau)


def helmholtz_error(y, kstar):
    """|g - g_ana|_2 of (B - k* A) g = 0, g(-1) = 1, g(+1) = 0 (Appendix B, Eq. (modpoisson)).

    g_ana = sinh(sqrt(k*)(1 - y)) / sinh(2 sqrt(k*)), the error functional the
    paper's mesh optimisation minimises (its first term).
    """
    A, B = compact_coeffs(y, 2)
    n = len(y)
    M = B - kstar * A
    M[0, :] = 0.0
    M[-1, :] = 0.0
    M[0, 0] = M[-1, -1] = 1.0
    rhs = np.zeros(n)
    rhs[0] = 1.0
    g = np.linalg.solve(M, rhs)
    r = math.sqrt(kstar)
    ana = np.exp(-r * (y + 1)) * (1 - np.exp(-2 * r * (1 - y))) / (1 - np.exp(-4 * r))
    return float(np.linalg.norm(g - ana))


def pressure_solve(st, rhs_A, dp_lo, dp_hi):
    """Per-mode Neumann Poisson problem of the filtered pressure.

    Interior rows (B - k^2 A) p = rhs_A (the equation already multiplied by A,
    as every implicit step of the method is); wall rows (D1 p)(-1) = dp_lo and
    (D1 p)(+1) = dp_hi with D1 = A1^-1 B1.  rhs_A: (Ny, Nz, nxh); dp_*: (Nz, nxh).
    The (0, 0) mode (singular for Neumann conditions) is left at zero here.
    """
    p = np.zeros_like(rhs_A)
    k2 = st.K2.reshape(-1)
    R = _modes(rhs_A)
    d_lo, d_hi = dp_lo.reshape(-1), dp_hi.reshape(-1)
    out = np.zeros_like(R)
    for m in range(k2.size):
        if k2[m] == 0 or not st.keep.reshape(-1)[m]:
            continue
        L = st.B2 - k2[m] * st.A2
        L[0, :] = st.D1[0]
        L[-1, :] = st.D1[-1]
        r = R[m].copy()
        r[0] = d_lo[m]
        r[-1] = d_hi[m]
        out[m] = np.linalg.solve(L, r)
    return _unmodes(out, rhs_A.shape)


def filtered_pressure(st, S, kind, p1, p3):
    """Filtered pressure from the filtered stresses, Sec. 3.1 Eq. (2): d_kk pbar = -d_ij filt(u_i u_j).

    With F_ij = filt(u_i u_j) = G P(u_i u_j), the right-hand side in Fourier
    space is k1^2 F11 + k3^2 F33 + 2 k1 k3 F13 - 2 i k1 D1 F12 - 2 i k3 D1 F23 - D2 F22,
    multiplied by A on interior rows (so D2 F22 enters as B F22).  The paper
    gives no boundary condition; the reading is the wall value of the filtered
    wall-normal momentum equation, d pbar/dy = nu chibar = nu G chi at y = +-1.
    The mean mode follows the mean wall-normal momentum balance, P = -F22(0,0).
    """
    G = filter_transfer(st, kind, p1, p3)
    u1, v, u3, _, _, _ = velocities(st, S)
    pu = [to_physical(st, f) for f in (u1, v, u3)]
    F = {(i, j): G * to_fourier(st, pu[i] * pu[j]) for i, j in PAIRS}
    K1, K3 = st.K1, st.K3
    r = (K1 ** 2 * F[0, 0] + K3 ** 2 * F[2, 2] + 2 * K1 * K3 * F[0, 2]
         - 2j * K1 * apply_y(st.D1, F[0, 1]) - 2j * K3 * apply_y(st.D1, F[1, 2]))
    rhs_A = apply_y(st.A2, r) - apply_y(st.B2, F[1, 1])
    chib = G * S["chi"]
    p = pressure_solve(st, rhs_A, st.nu * chib[0], st.nu * chib[-1])
    p[:, 0, 0] = -F[1, 1][:, 0, 0]
    return p * st.keep


def filtered_enstrophy(st, S, kind, p1, p3):
    """filt(omega_i omega_i) = G . P(omega_i omega_i), the tenth database variable (Sec. 3.1)."""
    G = filter_transfer(st, kind, p1, p3)
    u1, v, u3, du1, dv, du3 = velocities(st, S)
    om1, om2, om3 = vorticity(st, S, u1, v, u3, du1, du3)
    p = [to_physical(st, F) for F in (om1, om2, om3)]
    return G * to_fourier(st, p[0] ** 2 + p[1] ** 2 + p[2] ** 2)


def retained_modes(st, p1, p3):
    """Sharp cut-off retained set (Eq. (fou_fil)): kx < M1 and |kz| <= K3; returns (M1, K3)."""
    k1c = math.pi * st.re_tau / p1
    k3c = math.pi * st.re_tau / p3
    m1 = sum(1 for kx in range(st.nxh) if 2 * math.pi / st.Lx * kx < k1c)
    k3 = [kz for kz in range(st.Nz // 2) if 2 * math.pi / st.Lz * kz < k3c]
    return m1, (max(k3) if k3 else -1)


def database_record(st, S, p1, p3):
    """The ten database variables (Sec. 3.1) on the retained modes, (10, Ny, 2 K3 + 1, M1).

    ubar_i = G u_i, filt(u_i u_j) = G P(u_i u_j), filt(omega_i omega_i) with the
    sharp filter; kz ordered 0..K3 then -K3..-1.
    """
    G = filter_transfer(st, SHARP, p1, p3)
    u1, v, u3, _, _, _ = velocities(st, S)
    u = [u1, v, u3]
    pu = [to_physical(st, f) for f in u]
    fields = [G * f for f in u] + [G * to_fourier(st, pu[i] * pu[j]) for i, j in PAIRS]
    fields.append(filtered_enstrophy(st, S, SHARP, p1, p3))
    m1, K3 = retained_modes(st, p1, p3)
    jz = list(range(K3 + 1)) + [st.Nz - k for k in range(K3, 0, -1)]
    return np.stack([F[:, jz, :m1] for F in fields])


def spectra(st, S):
    """E_i(k1, y, k3) = w |u_i|^2 (w = 2 for kx > 0), mean mode excluded (Sec. 3.3)."""
    u1, v, u3, _, _, _ = velocities(st, S)
    w = np.where(np.arange(st.nxh) == 0, 1.0, 2.0)[None, None, :]
    E = np.stack([w * np.abs(f) ** 2 for f in (u1, v, u3)])
    E[:, :, 0, 0] = 0.0
    return E


# --------------------------------------------------------------------------
# Statistics (Sec. 3.3) and invariants
# --------------------------------------------------------------------------

def plane_mean_product(st, F, G):
    """<f g>(y) over an x-z plane by Parseval on the stored modes."""
    w = np.where(np.arange(st.nxh) == 0, 1.0, 2.0)[None, None, :]
    return np.sum(w * (F * np.conj(G)).real, axis=(1, 2))


def stats(st, S, ubar=None, tau=None):
    """20 profiles: U1, U3, <u_i u_j> (6), <ubar_i ubar_j> (6), <tau_ij> (6).

    Also u_tau = sqrt(nu |dU1/dy|) averaged over the two walls and the bulk
    velocity U_b = flux / 2.  Rows 8..19 are zero without filter output.
    """
    u1, v, u3, _, _, _ = velocities(st, S)
    u = [u1, v, u3]
    out = np.zeros((20, st.Ny))
    out[0] = S["U1"]
    out[1] = S["U3"]
    for p, (i, j) in enumerate(PAIRS):
        out[2 + p] = plane_mean_product(st, u[i], u[j])
        if ubar is not None:
            out[8 + p] = plane_mean_product(st, ubar[i], ubar[j])
            out[14 + p] = tau[p][:, 0, 0].real
    dU = st.D1 @ S["U1"]
    utau = math.sqrt(st.nu * 0.5 * (abs(dU[0]) + abs(dU[-1])))
    return out, utau, st.flux(S["U1"]) / 2.0


def divergence(st, S):
    """max |i k1 u1 + dv/dy + i k3 u3| over all modes and heights (continuity, Eq. (e2))."""
    u1, v, u3, _, dv, _ = velocities(st, S)
    d = 1j * st.K1 * u1 + dv + 1j * st.K3 * u3
    return float(np.abs(d).max())
