"""Pins of the CPU oracle against closed forms, invariants and brute force.

None of these compares the oracle with itself: each checks a property that
the paper or the mathematics fixes (see each test's docstring).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import pins
import synthetic as SY

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def c1():
    """Re_tau = 180 minimal box, 32 x 49 x 32, dt = 1e-3 (the small channel workload)."""
    return O.Setup(180, math.pi, math.pi / 2, 32, 49, 32, 1e-3)


def _row_order(i, n):
    ii = min(i, n - 1 - i)
    return 12 if ii >= 3 else {0: 6, 1: 8, 2: 10}[ii]


@pytest.mark.parametrize("deriv", [1, 2])
def test_compact_exact_on_polynomials(c1, deriv):
    """Appendix B, Eq. (diff): each row is exact for (y - y_i)^k up to its maximum order.

    The order per row is fixed by the stencil width: 12 inside (7 + 7 points,
    A_ii = 1), 10, 8, 6 on the reduced wall rows.  A wrong factorial, a
    dropped term or a wrong stencil makes some monomial fail.
    """
    y = c1.y
    A, B = (c1.A1, c1.B1) if deriv == 1 else (c1.A2, c1.B2)
    n = y.size
    for i in range(n):
        h = np.abs(y[min(i + 1, n - 1)] - y[max(i - 1, 0)])
        for k in range(_row_order(i, n) + 1):
            p = (y - y[i]) ** k
            dp = (k * (y - y[i]) ** (k - 1) if k >= 1 else 0 * y) if deriv == 1 else \
                 (k * (k - 1) * (y - y[i]) ** (k - 2) if k >= 2 else 0 * y)
            res = A[i] @ dp - B[i] @ p
            scale = np.abs(B[i]) @ np.abs(p) + np.abs(A[i]) @ np.abs(dp)
            assert abs(res) <= 1e-12 * scale, (i, k, res, scale)
        # the next two degrees are not both exact (maximum order, not more;
        # a symmetric stencil is exact for one extra odd degree)
        worst = 0.0
        for k in (_row_order(i, n) + 1, _row_order(i, n) + 2):
            p = (y - y[i]) ** k
            dp = k * (y - y[i]) ** (k - 1) if deriv == 1 else k * (k - 1) * (y - y[i]) ** (k - 2)
            res = A[i] @ dp - B[i] @ p
            scale = np.abs(B[i]) @ np.abs(p) + np.abs(A[i]) @ np.abs(dp)
            worst = max(worst, abs(res) / scale)
        assert worst > 1e-6, (i, worst)


def test_compact_convergence_order():
    """D1 and D2 errors on sin(pi y + 0.3) fall faster than N^-6 and N^-7 (wall rows are sixth order)."""
    errs1, errs2, ns = [], [], [33, 65]
    for n in ns:
        y = O.ygrid(n, 180)
        A1, B1 = O.compact_coeffs(y, 1)
        A2, B2 = O.compact_coeffs(y, 2)
        f = np.sin(np.pi * y + 0.3)
        d1 = np.linalg.solve(A1, B1 @ f)
        errs1.append(np.abs(d1 - np.pi * np.cos(np.pi * y + 0.3)).max())
        I = slice(1, n - 1)
        fpp = -np.pi ** 2 * f
        # interior second derivative from interior rows with exact wall values
        rhs = B2[I] @ f - A2[I, 0] * fpp[0] - A2[I, -1] * fpp[-1]
        d2 = np.linalg.solve(A2[I, I], rhs)
        errs2.append(np.abs(d2 - fpp[I]).max())
    r1 = math.log(errs1[0] / errs1[1]) / math.log(2.0)
    r2 = math.log(errs2[0] / errs2[1]) / math.log(2.0)
    assert r1 > 6 and r2 > 7, (errs1, errs2)


@pytest.mark.parametrize("ny,re", [(49, 180), (97, 395), (129, 550), (257, 550)])
def test_dirichlet_d2_spectrum_real_negative(ny, re):
    """Stability of the implicit viscous step: interior A^-1 B has real negative eigenvalues.

    The leading one approaches -pi^2/4, the exact first Dirichlet eigenvalue
    of d^2/dy^2 on [-1, 1].
    """
    y = O.ygrid(ny, re)
    A, B = O.compact_coeffs(y, 2)
    I = slice(1, ny - 1)
    ev = np.linalg.eigvals(np.linalg.solve(A[I, I], B[I, I]))
    assert np.abs(ev.imag).max() <= 1e-8 * np.abs(ev.real).max()
    assert ev.real.max() < 0
    assert abs(ev.real.max() + np.pi ** 2 / 4) < 1e-6


@pytest.mark.parametrize("ny,re,dt,kmax2", [(49, 180, 1e-3, 4 ** 2 * 15 ** 2 + 4 ** 2 * 15 ** 2),
                                            (257, 550, 2e-4, 191 ** 2 + (2 * 191) ** 2)])
def test_helmholtz_homogeneous_vs_sinh(ny, re, dt, kmax2):
    """Appendix B, Eq. (modpoisson): (B - k* A) g = 0, g(-1) = 1, g(+1) = 0 vs the sinh solution.

    k* = k^2 + 1/(beta nu dt) (the printed beta/(nu dt) read dimensionally).
    Where the boundary layer 1/sqrt(k*) spans grid points the discrete
    solution matches sinh(sqrt(k*)(1 - y)) / sinh(2 sqrt(k*)) to 1e-8; at the
    stiffest k* of the box (layer thinner than the first cell, the regime the
    paper's Appendix B optimises the mesh for) the error stays below 0.1.
    """
    y = O.ygrid(ny, re)
    A, B = O.compact_coeffs(y, 2)
    I = slice(1, ny - 1)
    nu = 1.0 / re

    def err(ks):
        M = B[I, I] - ks * A[I, I]
        g = np.linalg.solve(M, -(B[I, 0] - ks * A[I, 0]))
        r = math.sqrt(ks)
        ana = np.exp(-r * (y[I] + 1)) * (1 - np.exp(-2 * r * (1 - y[I]))) / (1 - np.exp(-4 * r))
        return np.abs(g - ana).max()

    assert err(1.0) < 1e-8
    assert err(100.0) < 1e-6
    worst = max(err(kmax2 + 1.0 / (b * nu * dt)) for (_, _, _, b) in O.RK3)
    assert worst < 0.1


def test_rk3_coefficients():
    """Spalart-Moser-Rogers low-storage RK3: alpha+beta = gamma+zeta, weights sum to 1."""
    tot = 0.0
    for g, z, a, b in O.RK3:
        assert abs((a + b) - (g + z)) < 1e-15
        tot += a + b
    assert abs(tot - 1.0) < 1e-15
    # third-order accuracy of the explicit part on y' = y: exact Taylor to O(dt^3)
    h = 1e-2
    yv, yprev = 1.0, 0.0
    for g, z, a, b in O.RK3:
        ynew = yv + h * (g * yv + z * yprev)
        yprev, yv = yv, ynew
    assert abs(yv - math.exp(h)) < 1e-8


def _tiny():
    return O.Setup(180, 2.0, 1.5, 8, 9, 6, 1e-3)


def test_transform_vs_brute_force_dft():
    """to_physical equals the direct sum over stored modes (and conjugates) on the padded grid."""
    st = _tiny()
    rng = np.random.default_rng(3)
    F = rng.standard_normal((st.Ny, st.Nz, st.nxh)) + 1j * rng.standard_normal((st.Ny, st.Nz, st.nxh))
    F[:, st.Nz // 2, :] = 0
    F[:, 0, 0] = F[:, 0, 0].real
    for jz in range(1, st.Nz // 2):          # Hermitian kx = 0 column
        F[:, st.Nz - jz, 0] = np.conj(F[:, jz, 0])
    u = O.to_physical(st, F)
    x = np.arange(st.Lx3) * st.Lx / st.Lx3
    z = np.arange(st.Lz3) * st.Lz / st.Lz3
    ref = np.zeros((st.Ny, st.Lz3, st.Lx3))
    for jz in range(st.Nz):
        for kx in range(st.nxh):
            e = np.exp(1j * (st.K3[jz, kx] * z[:, None] + st.K1[jz, kx] * x[None, :]))
            term = F[:, jz, kx][:, None, None] * e[None]
            ref += term.real if kx == 0 else 2 * term.real
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()
    # and analysis inverts synthesis on the stored modes
    assert np.abs(O.to_fourier(st, u) - F).max() < 1e-13 * np.abs(F).max()


def test_dealiasing_single_mode_products():
    """3/2 rule: a product of two stored modes has exactly its true retained modes, no aliases."""
    st = _tiny()
    x = np.arange(st.Lx3) * st.Lx / st.Lx3
    z = np.arange(st.Lz3) * st.Lz / st.Lz3
    a, b = 3, 2          # kx indices; a + b = 5 >= Nx/2 = 4 is not stored, a - b = 1 is
    fa = np.cos(st.K1[0, a] * x)[None, None, :] * np.ones((st.Ny, st.Lz3, 1))
    fb = np.cos(st.K1[0, b] * x)[None, None, :] * np.ones((st.Ny, st.Lz3, 1))
    P = O.to_fourier(st, fa * fb)
    expect = np.zeros_like(P)
    expect[:, 0, a - b] = 0.25        # cos a cos b = (cos(a-b) + cos(a+b))/2, kx>0 half-amplitude
    assert np.abs(P - expect).max() < 1e-15
    # in z: kz = 2 and kz = 2 -> kz = 4 is beyond the retained |kz| < Nz/2 = 3
    gz = np.cos(st.K3[2, 0] * z)[None, :, None] * np.ones((st.Ny, 1, st.Lx3))
    P = O.to_fourier(st, gz * gz)
    expect = np.zeros_like(P)
    expect[:, 0, 0] = 0.5
    assert np.abs(P - expect).max() < 1e-15


def test_poiseuille_steady(c1):
    """Laminar Poiseuille stays steady to 1e-13 and f equals the exact gradient 3 nu U_b."""
    ic = SY.perturbed_poiseuille(c1.y, 180, c1.Lx, c1.Lz, 32, 32, seed=1, amp=0.0)
    S = O.initial_state(c1, ic["v"], ic["omega2"], ic["U1"], ic["U3"])
    S = O.run(c1, S, 30)
    assert np.abs(S["U1"] - ic["U1"]).max() <= 1e-13 * np.abs(ic["U1"]).max()
    assert abs(S["f"] - 3 * c1.nu * ic["Ub"]) < 1e-12 * 3 * c1.nu * ic["Ub"]
    assert np.abs(S["v"]).max() == 0 and np.abs(S["omega2"]).max() == 0


@pytest.fixture(scope="module")
def c1_run(c1):
    ic = SY.perturbed_poiseuille(c1.y, 180, c1.Lx, c1.Lz, 32, 32, seed=7, amp=0.1)
    S0 = O.initial_state(c1, ic["v"], ic["omega2"], ic["U1"], ic["U3"])
    return S0, O.run(c1, S0, 10)


def test_flux_divergence_walls_hermitian(c1, c1_run):
    """Constant mass flux, continuity (Eq. (e2)) to 1e-12, v = dv/dy = omega_2 = 0 at the walls."""
    S0, S = c1_run
    assert abs(c1.flux(S["U1"]) - S0["Q0"]) < 1e-13 * abs(S0["Q0"])
    u1, v, u3, _, dv, _ = O.velocities(c1, S)
    scale = np.abs(u1[:, :, 1:]).max()
    assert O.divergence(c1, S) < 1e-12 * scale
    assert np.abs(v[[0, -1]]).max() < 1e-12 * scale
    assert np.abs(dv[[0, -1]]).max() < 1e-12 * scale
    assert np.abs(S["omega2"][[0, -1]]).max() == 0
    for F in (S["v"], S["omega2"]):      # kx = 0 column stays Hermitian in kz
        for jz in range(1, c1.Nz // 2):
            assert np.abs(F[:, jz, 0] - np.conj(F[:, c1.Nz - jz, 0])).max() < 1e-13 * np.abs(F).max()


def test_u_dot_h_vanishes(c1, c1_run):
    """H = u x omega is orthogonal to u at every point of the padded grid."""
    _, S = c1_run
    u1, v, u3, du1, dv, du3 = O.velocities(c1, S)
    om1 = du3 - 1j * c1.K3 * v
    om3 = 1j * c1.K1 * v - du1
    p = [O.to_physical(c1, F) for F in (u1, v, u3, om1, S["omega2"], om3)]
    H1 = p[1] * p[5] - p[2] * p[4]
    H2 = p[2] * p[3] - p[0] * p[5]
    H3 = p[0] * p[4] - p[1] * p[3]
    dot = p[0] * H1 + p[1] * H2 + p[2] * H3
    mag = np.sqrt(p[0] ** 2 + p[1] ** 2 + p[2] ** 2) * np.sqrt(H1 ** 2 + H2 ** 2 + H3 ** 2)
    assert np.abs(dot).max() < 1e-13 * mag.max()


def test_viscous_decay_single_mode():
    """Linear decay of an omega_2 eigenmode: per substep (1 + a z)/(1 - b z), z = nu dt (lam - k^2).

    With no mean flow and amplitude 1e-30 the non-linear term is ~1e-60,
    so Eq. (psi) reduces to the RK3 amplification factor of the discrete
    Dirichlet eigenvalue lam; over a full step it approaches exp(z) to O(z^3).
    """
    st = O.Setup(180, math.pi, math.pi / 2, 8, 33, 4, 2e-3)
    I = slice(1, st.Ny - 1)
    lam, V = np.linalg.eig(np.linalg.solve(st.A2[I, I], st.B2[I, I]))
    k = int(np.argmax(lam.real))
    phi = np.zeros(st.Ny)
    phi[I] = V[:, k].real
    S0 = SY.single_mode(st.y, 8, 4, 1, 1, omega_profile=1e-30 * phi)
    S = O.initial_state(st, S0["v"], S0["omega2"], S0["U1"], S0["U3"])
    k2 = st.K2[1, 1]
    prod = 1.0
    for s in range(3):
        S = O.substep(st, S)
        g, z, a, b = O.RK3[s]
        zz = st.nu * st.dt * (lam[k].real - k2)
        prod *= (1 + a * zz) / (1 - b * zz)
        ratio = S["omega2"][I, 1, 1] / (1e-30 * phi[I])
        assert np.abs(ratio - prod).max() < 1e-13
    zz = st.nu * st.dt * (lam[k].real - k2)
    # the implicit/explicit viscous split is second order: local error O(z^3)
    assert abs(prod - math.exp(zz)) < 0.05 * abs(zz) ** 3


def _golden_os():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "orr_sommerfeld.txt"))
            if l.strip() and not l.startswith("#")]
    return {float(r[0]): complex(float(r[2]), float(r[3])) for r in rows}


def test_os_eigenvalue_literature():
    """The input generator's Orr-Sommerfeld solve reproduces Orszag's published eigenvalues."""
    for re, c_ref in _golden_os().items():
        c, _ = SY.orr_sommerfeld_mode(re, 1.0, np.linspace(-1, 1, 5))
        assert abs(c - c_ref) < 1e-7


def test_orr_sommerfeld_growth():
    """Orr-Sommerfeld mode at Re = 7500, alpha = 1 grows at c_i = 0.00223497 through the DNS substep.

    Linear regime (amplitude 1e-6); 97 points, dt = 0.02, t in [0, 10];
    relative tolerance 1 %, set by the wall-normal resolution and the
    initial transient of the interpolated eigenfunction.
    """
    c_ref = _golden_os()[7500.0]
    st = O.Setup(7500, 2 * math.pi, 1.0, 4, 97, 2, 0.02, grid_re=180)
    _, vprof = SY.orr_sommerfeld_mode(7500, 1.0, st.y)
    S0 = SY.single_mode(st.y, 4, 2, 1, 0, v_profile=1e-6 * vprof, U1=1 - st.y ** 2)
    S = O.initial_state(st, S0["v"], S0["omega2"], S0["U1"], S0["U3"])

    def amp(S):
        return math.sqrt(np.sum(st.wq * np.abs(S["v"][:, 0, 1]) ** 2))

    a0, t0 = amp(S), S["t"]
    S = O.run(st, S, 3 * 500)
    growth = math.log(amp(S) / a0) / (S["t"] - t0)
    assert abs(growth - c_ref.imag) < 0.01 * c_ref.imag, growth


def test_filter_transfer_single_mode(c1):
    """Filtered single modes: ubar = G u with G = sinc product (BOX) or an indicator (SHARP)."""
    G = O.filter_transfer(c1, O.BOX, 50, 50)
    d = 50 / 180
    k1, k3 = c1.K1[2, 3], c1.K3[2, 3]
    assert abs(G[2, 3] - (math.sin(k1 * d / 2) / (k1 * d / 2)) * (math.sin(k3 * d / 2) / (k3 * d / 2))) < 1e-15
    assert G[0, 0] == 1.0
    Gs = O.filter_transfer(c1, O.SHARP, 120, 60)
    k1c, k3c = math.pi * 180 / 120, math.pi * 180 / 60
    assert np.array_equal(Gs > 0, (np.abs(c1.K1) < k1c) & (np.abs(c1.K3) < k3c) & c1.keep)
    S0 = SY.single_mode(c1.y, 32, 32, 3, 2, v_profile=(1 - c1.y ** 2) ** 2)
    S = O.initial_state(c1, S0["v"], S0["omega2"], S0["U1"], S0["U3"])
    ub, tau = O.filter_stresses(c1, S, O.BOX, 50, 50)
    assert np.abs(ub[1][:, 2, 3] - G[2, 3] * S["v"][:, 2, 3]).max() < 1e-16
    assert np.abs(np.delete(ub[1].reshape(c1.Ny, -1), 2 * c1.nxh + 3, axis=1)).max() == 0


@pytest.mark.parametrize("kind,p", [(O.BOX, (50, 50)), (O.SHARP, (120, 60))])
def test_second_order_identity(c1, c1_run, kind, p):
    """<u_i u_j> = <ubar_i ubar_j> + <tau_ij> to rounding when G(0) = 1 (Sec. 3.1)."""
    _, S = c1_run
    ub, tau = O.filter_stresses(c1, S, kind, *p)
    out, utau, ubulk = O.stats(c1, S, ub, tau)
    scale = np.abs(out[2:8]).max()
    assert np.abs(out[2:8] - out[8:14] - out[14:20]).max() < 1e-13 * scale
    # the Parseval mean of u_i u_j equals the (0,0) mode of the dealiased product
    u1, v, u3, _, _, _ = O.velocities(c1, S)
    pu = O.to_physical(c1, u1)
    assert np.abs(O.to_fourier(c1, pu * pu)[:, 0, 0].real - out[2]).max() < 1e-13 * scale
    assert utau > 0 and ubulk > 0


def test_filtered_enstrophy_mean_is_parseval(c1, c1_run):
    """The (0,0) mode of filt(omega_i omega_i) (G(0) = 1) equals the Parseval plane mean of |omega|^2."""
    _, S = c1_run
    ens = O.filtered_enstrophy(c1, S, O.BOX, 50, 50)
    u1, v, u3, du1, dv, du3 = O.velocities(c1, S)
    om1 = du3 - 1j * c1.K3 * v
    om3 = 1j * c1.K1 * v - du1
    par = sum(O.channel.plane_mean_product(c1, F, F) for F in (om1, S["omega2"], om3))
    assert np.abs(ens[:, 0, 0].real - par).max() < 1e-12 * np.abs(par).max()
    G = O.filter_transfer(c1, O.SHARP, 120, 60)
    ens_s = O.filtered_enstrophy(c1, S, O.SHARP, 120, 60)
    assert np.abs(ens_s[:, ~(G > 0)]).max() == 0.0     # the sharp filter removes the cut modes exactly


def test_database_record_holds_exactly_the_retained_modes(c1, c1_run):
    """The compact record's modes are exactly those the sharp filter keeps, and its
    filtered fields are the filtered fields (Sec. 3.1, Eq. (fou_fil))."""
    _, S = c1_run
    G = O.filter_transfer(c1, O.SHARP, 120, 60)
    m1, K3 = O.retained_modes(c1, 120, 60)
    assert int((G > 0).sum()) == m1 * (2 * K3 + 1)
    rec = O.database_record(c1, S, 120, 60)
    ub, tau = O.filter_stresses(c1, S, O.SHARP, 120, 60)
    jz = list(range(K3 + 1)) + [c1.Nz - k for k in range(K3, 0, -1)]
    assert np.array_equal(rec[1], ub[1][:, jz, :m1])
    # filt(u_i u_j) - ubar_i ubar_j is tau on the retained modes
    u1, v, u3, _, _, _ = O.velocities(c1, S)
    pb = [O.to_physical(c1, f) for f in ub]
    for p, (i, j) in enumerate(O.PAIRS):
        bb = O.to_fourier(c1, pb[i] * pb[j])[:, jz, :m1]
        assert np.abs(rec[3 + p] - bb - tau[p][:, jz, :m1]).max() < 1e-12 * np.abs(rec[3 + p]).max()


def test_spectra_sum_to_the_variances(c1, c1_run):
    """Parseval: the spectrum summed over modes is <u_i u_i> - U_i^2 at every height."""
    _, S = c1_run
    E = O.spectra(c1, S)
    out, _, _ = O.stats(c1, S)
    var = out[2:5] - np.array([S["U1"] ** 2, 0 * S["U1"], S["U3"] ** 2])
    assert np.abs(E.sum(axis=(2, 3)) - var).max() < 1e-12 * np.abs(out[2:5]).max()


def test_pressure_solve_reproduces_a_polynomial_exactly(c1):
    """Manufactured solution: p = (1 - y^2)^2 (1 + 0.3 y) + 0.2 y in every mode; with the
    right-hand side A (p'' - k^2 p) and wall slopes p'(+-1) from calculus, the Neumann
    solve must return p to rounding (the compact operators are exact on this degree)."""
    y = c1.y
    w = 1 - y * y
    p = w * w * (1 + 0.3 * y) + 0.2 * y
    dp = -4 * y * w * (1 + 0.3 * y) + 0.3 * w * w + 0.2
    d2p = (-4 * w + 8 * y * y) * (1 + 0.3 * y) - 2.4 * y * w
    P = np.broadcast_to(p[:, None, None], (c1.Ny, c1.Nz, c1.nxh)).astype(np.complex128)
    rhs = O.apply_y(c1.A2, d2p[:, None, None] - c1.K2[None] * P)
    lo = np.full((c1.Nz, c1.nxh), dp[0], dtype=np.complex128)
    hi = np.full((c1.Nz, c1.nxh), dp[-1], dtype=np.complex128)
    out = O.pressure_solve(c1, rhs, lo, hi)
    mask = (c1.K2 > 0) & c1.keep
    assert np.abs(out[:, mask] - P[:, mask]).max() < 1e-11 * np.abs(p).max()


def test_filtered_pressure_source_is_the_strain_minus_rotation_identity(c1, c1_run):
    """Incompressible identity d_ij(u_i u_j) = S:S - |omega|^2 / 2 (the paper prints 1/4):
    the Poisson source built from the stress tensor (the pressure's route) equals the one
    built from velocity gradients, to the truncation error of the compact scheme."""
    _, S = c1_run
    u1, v, u3, du1, dv, du3 = O.velocities(c1, S)
    u = [u1, v, u3]
    pu = [O.to_physical(c1, f) for f in u]
    F = {(i, j): O.to_fourier(c1, pu[i] * pu[j]) for i, j in O.PAIRS}
    K1, K3 = c1.K1, c1.K3
    src = (-K1 ** 2 * F[0, 0] - K3 ** 2 * F[2, 2] - 2 * K1 * K3 * F[0, 2]
           + 2j * K1 * O.apply_y(c1.D1, F[0, 1]) + 2j * K3 * O.apply_y(c1.D1, F[1, 2])
           + O.apply_y(c1.D2, F[1, 1]))                                   # d_ij (u_i u_j)
    grads = [[1j * K1 * f, df, 1j * K3 * f] for f, df in zip(u, (du1, dv, du3))]   # d_j u_i
    g = [[O.to_physical(c1, grads[i][j]) for j in range(3)] for i in range(3)]
    ss = sum(0.25 * (g[i][j] + g[j][i]) ** 2 for i in range(3) for j in range(3))
    om = [g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]]
    ident = O.to_fourier(c1, ss - 0.5 * (om[0] ** 2 + om[1] ** 2 + om[2] ** 2))
    scale = np.abs(ident).max()
    # equal up to the compact scheme's truncation on the product fields (largest at the
    # reduced wall rows); a wrong factor or sign is O(1)
    assert np.abs(src - ident)[3:-3].max() < 1e-3 * scale
    assert np.abs(src - ident).max() < 2e-2 * scale
    wrong = O.to_fourier(c1, ss - 0.25 * (om[0] ** 2 + om[1] ** 2 + om[2] ** 2))
    assert np.abs(src - wrong).max() > 0.5 * scale      # the printed 1/4 does not hold


def test_filtered_pressure_mean_and_wall_condition(c1, c1_run):
    _, S = c1_run
    P = O.filtered_pressure(c1, S, O.BOX, 50, 50)
    ub, tau = O.filter_stresses(c1, S, O.BOX, 50, 50)
    G = O.filter_transfer(c1, O.BOX, 50, 50)
    u1, v, u3, _, _, _ = O.velocities(c1, S)
    pv = O.to_physical(c1, v)
    F22 = G * O.to_fourier(c1, pv * pv)
    assert np.abs(P[:, 0, 0] + F22[:, 0, 0]).max() == 0.0
    dP = O.apply_y(c1.D1, P)
    chib = G * S["chi"]
    mask = (c1.K2 > 0) & c1.keep
    assert np.abs(dP[0][mask] - c1.nu * chib[0][mask]).max() < 1e-10 * np.abs(dP).max()


def test_os_squire_generator_obeys_squires_transformation():
    """The coupled-mode generator's 3-D eigenvalue equals the 2-D one at (k, Re alpha / k)."""
    for a, b in ((2.0, 1.0), (1.0, 1.0)):
        k = math.hypot(a, b)
        c3, _, _ = SY.os_squire_mode(7500, a, b, np.linspace(-1, 1, 5))
        c2, _ = SY.orr_sommerfeld_mode(7500 * a / k, k, np.linspace(-1, 1, 5))
        assert abs(c3 - c2) < 1e-7, (a, b, c3, c2)


def test_oblique_orr_sommerfeld_squire_mode():
    """Oblique mode (k_1, k_3) = (2, 1) at Re 7500: |v| and |omega_2| change at alpha c_i.

    Appendix A, Eqs. (hghv), (chi1), (psi) in the linear regime.  Unlike the
    two-dimensional Orr-Sommerfeld pin, this one has omega_2, u_3 and omega_1
    non-zero: omega_2 follows the Squire equation only if N_omega2 =
    i k_3 H_1 - i k_1 H_3 carries the right signs and wavenumbers, and v keeps
    the Orr-Sommerfeld rate only if the omega_2 parts of H_3 cancel in N_chi.
    Rates within 0.2 % of alpha c_i = -0.0566 (measured 1e-4) and the
    omega_2 / v profile within 1e-3 of the eigenmode over t = 2.
    """
    rate, rv, rw, prof = pins.oblique_mode_rates()
    assert abs(rv - rate) < 2e-3 * abs(rate), (rate, rv)
    assert abs(rw - rate) < 2e-3 * abs(rate), (rate, rw)
    assert prof < 1e-3, prof


def test_energy_identity_of_the_nonlinear_term(c1, c1_run):
    """sum_k w Re(conj(u_k) . H_k) = 0 at every height for a fully 3-D state.

    <u, P(u x omega)> = <u, u x omega> = 0 (u lies in the retained set, where
    the 3/2 rule is exact): a dropped, mis-signed or mis-indexed term in any
    component of H breaks it.
    """
    _, S = c1_run
    assert pins.energy_residual(c1, S) < 1e-14


def test_vorticity_is_divergence_free(c1, c1_run):
    """i k_1 omega_1 + D1 omega_2 + i k_3 omega_3 = 0 to rounding (the divergence of a curl)."""
    _, S = c1_run
    assert pins.vorticity_divergence(c1, S) < 1e-13


def test_utau_and_bulk_velocity_of_laminar_poiseuille(c1):
    """Sec. 3.3 outputs on U = 1.5 U_b (1 - y^2): u_tau^2 = 3 nu U_b exactly (the wall
    rows of D1 are exact on quadratics) and U_b = flux / 2 with the trapezoid rule, whose
    error on a quadratic is known in closed form: U_b (1 - sum_i h_i^3 / 8)."""
    ub = 15.98
    S = dict(v=np.zeros((c1.Ny, c1.Nz, c1.nxh), complex), omega2=np.zeros((c1.Ny, c1.Nz, c1.nxh), complex),
             U1=1.5 * ub * (1 - c1.y ** 2), U3=np.zeros(c1.Ny))
    _, utau, bulk = O.stats(c1, S)
    assert abs(utau ** 2 - 3 * c1.nu * ub) < 1e-12 * 3 * c1.nu * ub   # D1 wall rows: ~1e-13 rounding
    h = np.diff(c1.y)
    assert abs(bulk - ub * (1 - np.sum(h ** 3) / 8)) < 1e-14 * ub


def test_utau_averages_the_two_walls(c1):
    """An asymmetric profile U = (1 - y^2)(1 + y/2) has |dU/dy| = 1 at y = -1 and 3 at y = +1:
    u_tau^2 = nu (1 + 3) / 2."""
    S = dict(v=np.zeros((c1.Ny, c1.Nz, c1.nxh), complex), omega2=np.zeros((c1.Ny, c1.Nz, c1.nxh), complex),
             U1=(1 - c1.y ** 2) * (1 + 0.5 * c1.y), U3=np.zeros(c1.Ny))
    _, utau, _ = O.stats(c1, S)
    assert abs(utau ** 2 - 2 * c1.nu) < 1e-12 * c1.nu
