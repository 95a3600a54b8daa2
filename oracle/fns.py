"""Frozen natural spinors from the MP2 virtual-virtual density.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section "State-Average Frozen Natural Spinors", steps 1-4:

1. D V = V n (Eq. 17): eigenvectors of the vv density are the virtual
   natural spinors, eigenvalues their occupation numbers;
2. keep the natural spinors with occupation n >= tau and transform the vv
   Fock block, F^NS = V~^H F_vv V~ (Eq. 18); the Fock matrix is diag(eps);
3. F^NS Z~ = Z~ eps~ (Eq. 19): semicanonical natural virtuals;
4. U = V~ Z~ (Eq. 20).

The Cholesky vectors are then rotated into the truncated basis (section
"Implementation and Computational Details"): occupied spinors keep their
canonical form, virtual indices transform with U.

The density used is the MP2 one (Eq. 15).  The state-averaged density of
Eq. 16 adds CIS(D) densities whose expressions are in the paper's
supporting information, which is not available; the MP2 density alone is
the reading taken here.
"""

from __future__ import annotations

import numpy as np

from .mp2 import density_vv


def natural_spinors(eps, B, ncore, nval, nvirt, tau, D=None):
    """Return (occupations descending, U [v, v'], eps~ [v'])."""
    o = ncore + nval
    if D is None:
        D = density_vv(eps, B, ncore, nval, nvirt)
    n, V = np.linalg.eigh(D)
    order = np.argsort(-n, kind="stable")
    n, V = n[order], V[:, order]
    # degenerate pairs straddling tau are kept together (relative guard)
    keep = n >= tau * (1.0 - 1e-10)
    Vt = V[:, keep]
    Fvv = np.diag(eps[o:o + nvirt]).astype(np.complex128)
    Fns = Vt.conj().T @ Fvv @ Vt
    et, Z = np.linalg.eigh(Fns)
    U = Vt @ Z
    return n, U, et


def rotate(eps, B, ncore, nval, nvirt, U, eps_t):
    """B'_oo = B_oo, B'_ov = B_ov U, B'_vo = U^H B_vo, B'_vv = U^H B_vv U."""
    o = ncore + nval
    vk = U.shape[1]
    n2 = o + vk
    Bn = np.empty((B.shape[0], n2, n2), dtype=np.complex128)
    Bn[:, :o, :o] = B[:, :o, :o]
    Bn[:, :o, o:] = B[:, :o, o:] @ U
    Bn[:, o:, :o] = U.conj().T @ B[:, o:, :o]
    Bn[:, o:, o:] = U.conj().T @ B[:, o:, o:] @ U
    en = np.concatenate([eps[:o], eps_t])
    return en, Bn
