"""Broadened absorption spectrum from excitation energies and oscillator
strengths.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section "Computational Details" and the results sections: the computed
spectra are sums of Lorentzian lines of a given full width at half maximum
(0.3 eV for SiCl4, Ar, the metal oxyanions and TiCl4; 0.25 eV for VOCl3),
optionally moved by one uniform energy shift to align an edge with
experiment.  Written out:

    I(E) = sum_n f_n L(E - (omega_n [eV] + shift)),
    L(x) = (g / (2 pi)) / (x^2 + (g / 2)^2),   g = FWHM,

with omega_n in Hartree converted at 27.211386245988 eV/Eh.  L has unit
area, its maximum 2 / (pi g) at x = 0 and half of that at x = +-g/2.

Pins (tests/test_oracle_pins.py): the integral over [a, b] equals the closed
form sum_n f_n [atan((b - E_n) / h) - atan((a - E_n) / h)] / pi (h = g/2),
one line's peak height and half-maximum points, linearity in f.
"""

from __future__ import annotations

import numpy as np

EV_PER_EH = 27.211386245988


def lorentzian_spectrum(omega_eh, osc, grid_ev, fwhm_ev=0.3, shift_ev=0.0):
    """I(E) on the energy grid (eV) from roots omega (Eh) and strengths f."""
    omega_eh = np.asarray(omega_eh, dtype=np.float64)
    osc = np.asarray(osc, dtype=np.float64)
    grid_ev = np.asarray(grid_ev, dtype=np.float64)
    h = 0.5 * fwhm_ev
    out = np.zeros_like(grid_ev)
    for w, f in zip(omega_eh, osc):
        x = grid_ev - (w * EV_PER_EH + shift_ev)
        out += f * (h / np.pi) / (x * x + h * h)
    return out
