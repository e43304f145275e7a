"""Least-stable Orr-Sommerfeld mode of plane Poiseuille flow, as an input.

A Chebyshev-collocation solve of the Orr-Sommerfeld eigenproblem for
U = 1 - y^2 (centre-line units), with clamped conditions v = v' = 0 at
y = +-1 built in through v = (1 - y^2) q (the standard clamped fourth
derivative).  This is a separate spectral method for a textbook linear
stability problem, not the channel substep: it only produces the initial
wall-normal velocity profile for the linear-growth check, evaluated on a
caller-given grid by barycentric interpolation.
"""
import numpy as np
import scipy.linalg


def _cheb(n):
    """Chebyshev points x_j = cos(pi j / n) and the differentiation matrix."""
    x = np.cos(np.pi * np.arange(n + 1) / n)
    c = np.hstack([2.0, np.ones(n - 1), 2.0]) * (-1.0) ** np.arange(n + 1)
    X = np.tile(x, (n + 1, 1)).T
    dX = X - X.T
    D = np.outer(c, 1.0 / c) / (dX + np.eye(n + 1))
    D = D - np.diag(D.sum(axis=1))
    return D, x


def orr_sommerfeld_mode(re, alpha, y_eval, n=120):
    """Return (c, v_hat(y_eval)) for the mode with the largest Im(c).

    The eigenproblem is A v = c B v with
    A = (1/Re)(D^4 - 2 a^2 D^2 + a^4) - i a U (D^2 - a^2) + i a U'',
    B = -i a (D^2 - a^2), from i a [(U - c)(D^2 - a^2) v - U'' v] = (1/Re)(D^2 - a^2)^2 v.
    The profile is normalised to max |v| = 1 with v real and positive there.
    """
    D, x = _cheb(n)
    D2 = D @ D
    S = np.diag(np.hstack([0.0, 1.0 / (1.0 - x[1:-1] ** 2), 0.0]))
    D4 = (np.diag(1.0 - x ** 2) @ np.linalg.matrix_power(D, 4)
          - 8.0 * np.diag(x) @ np.linalg.matrix_power(D, 3) - 12.0 * D2) @ S
    I = np.eye(n + 1)
    U = 1.0 - x ** 2
    Upp = -2.0 * np.ones_like(x)
    a = alpha
    A = (D4 - 2 * a * a * D2 + a ** 4 * I) / re - 1j * a * np.diag(U) @ (D2 - a * a * I) + 1j * a * np.diag(Upp)
    B = -1j * a * (D2 - a * a * I)
    A = A[1:-1, 1:-1]
    B = B[1:-1, 1:-1]
    w, V = scipy.linalg.eig(A, B)
    ok = np.isfinite(w)
    w, V = w[ok], V[:, ok]
    i = int(np.argmax(w.imag))
    c = w[i]
    v = np.hstack([0.0, V[:, i], 0.0])
    # barycentric interpolation at the Chebyshev points (weights (-1)^j, halved at the ends)
    wts = (-1.0) ** np.arange(n + 1)
    wts[0] *= 0.5
    wts[-1] *= 0.5
    y_eval = np.asarray(y_eval, dtype=np.float64)
    out = np.empty(y_eval.size, dtype=np.complex128)
    for m, yy in enumerate(y_eval):
        d = yy - x
        hit = np.nonzero(np.abs(d) < 1e-15)[0]
        if hit.size:
            out[m] = v[hit[0]]
        else:
            t = wts / d
            out[m] = np.sum(t * v) / np.sum(t)
    j = int(np.argmax(np.abs(out)))
    out = out / out[j]
    out[np.abs(y_eval) >= 1.0] = 0.0
    return c, out


def _barycentric(x, f, y_eval):
    """Values at y_eval of the polynomial through (x_j, f_j) at the Chebyshev points."""
    n = x.size - 1
    wts = (-1.0) ** np.arange(n + 1)
    wts[0] *= 0.5
    wts[-1] *= 0.5
    out = np.empty(y_eval.size, dtype=np.complex128)
    for m, yy in enumerate(y_eval):
        d = yy - x
        hit = np.nonzero(np.abs(d) < 1e-15)[0]
        if hit.size:
            out[m] = f[hit[0]]
        else:
            t = wts / d
            out[m] = np.sum(t * f) / np.sum(t)
    return out


def os_squire_mode(re, alpha, beta, y_eval, n=120):
    """Least-stable oblique Orr-Sommerfeld mode with its Squire (wall-normal vorticity) part.

    For a disturbance exp(i(alpha x + beta z) + lam t) of U = 1 - y^2 with
    k^2 = alpha^2 + beta^2, the wall-normal velocity solves the three-dimensional
    Orr-Sommerfeld problem A v = c B v with
    A = (1/Re)(D^2 - k^2)^2 - i alpha U (D^2 - k^2) + i alpha U'', B = -i alpha (D^2 - k^2),
    lam = -i alpha c; the wall-normal vorticity eta = d u/dz - d w/dx is then the forced
    solution of the linearised Squire equation
    [lam + i alpha U - (1/Re)(D^2 - k^2)] eta = -i beta U' v,  eta(+-1) = 0,
    so (v, eta) is an eigenmode of the coupled linear system: both grow as exp(alpha c_i t).
    Returns (c, v(y_eval), eta(y_eval)), scaled together so that v is 1 where |v| peaks.
    """
    D, x = _cheb(n)
    D2 = D @ D
    S = np.diag(np.hstack([0.0, 1.0 / (1.0 - x[1:-1] ** 2), 0.0]))
    D4 = (np.diag(1.0 - x ** 2) @ np.linalg.matrix_power(D, 4)
          - 8.0 * np.diag(x) @ np.linalg.matrix_power(D, 3) - 12.0 * D2) @ S
    I = np.eye(n + 1)
    U = 1.0 - x ** 2
    Up = -2.0 * x
    Upp = -2.0 * np.ones_like(x)
    a, b = float(alpha), float(beta)
    k2 = a * a + b * b
    L = D2 - k2 * I
    A = (D4 - 2 * k2 * D2 + k2 * k2 * I) / re - 1j * a * np.diag(U) @ L + 1j * a * np.diag(Upp)
    B = -1j * a * L
    w, V = scipy.linalg.eig(A[1:-1, 1:-1], B[1:-1, 1:-1])
    ok = np.isfinite(w)
    w, V = w[ok], V[:, ok]
    i = int(np.argmax(w.imag))
    c = w[i]
    v = np.hstack([0.0, V[:, i], 0.0])
    lam = -1j * a * c
    Sq = lam * I + 1j * a * np.diag(U) - L / re
    eta = np.zeros(n + 1, dtype=np.complex128)
    eta[1:-1] = np.linalg.solve(Sq[1:-1, 1:-1], (-1j * b * Up * v)[1:-1])
    y_eval = np.asarray(y_eval, dtype=np.float64)
    ve = _barycentric(x, v, y_eval)
    ee = _barycentric(x, eta, y_eval)
    j = int(np.argmax(np.abs(ve)))
    s = 1.0 / ve[j]
    ve, ee = ve * s, ee * s
    edge = np.abs(y_eval) >= 1.0
    ve[edge] = 0.0
    ee[edge] = 0.0
    return c, ve, ee
