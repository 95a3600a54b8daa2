"""Error bounds shared by the GPU tests.

Oscillator strengths f_n = (2/3) omega_n |F^H x_n|^2 depend on the
eigenvector.  A computed unit vector x with residual ||M x - omega x|| <=
conv lies within an angle sin(theta) <= conv / gap of the exact
eigenvector (Davis-Kahan; gap = distance from its root to the nearest other
eigenvalue), and f is quadratic in x, so |f - f_exact| is a few times
(conv / gap) times the scale of f.  Clustered roots (core excitations into
a dense virtual space) make the gap, not the precision, set the bound.
"""

import numpy as np


def osc_tolerance(omega, omega_next, conv, osc, factor=10.0):
    """Per-root bound on |f - f_exact|: factor * conv / gap_n * max |f|, with
    omega the k exact roots and omega_next the exact root k + 1."""
    w = np.append(np.asarray(omega, dtype=float), float(omega_next))
    fmax = float(np.abs(np.asarray(osc)).max())
    out = []
    for q in range(len(omega)):
        gap = min(abs(w[q] - w[p]) for p in range(len(w)) if p != q)
        out.append(factor * conv / gap * fmax)
    return np.array(out)
