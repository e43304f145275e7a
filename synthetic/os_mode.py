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
