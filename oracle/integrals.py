"""Explicit two-electron integrals from Cholesky vectors.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section "Implementation and Computational Details": the integrals are
generated from the (MO-basis) Cholesky vectors.  Chemist notation
(pq|rs) = sum_P B^P_pq B^P_rs (no complex conjugation; every B^P is
Hermitian, B^P_pq = conj(B^P_qp)), physicist notation <pq|rs> = (pr|qs), and
the antisymmetrised integral <pq||rs> = <pq|rs> - <pq|sr> that enters the
normal-ordered Hamiltonians of Eqs. 4c / x2c.
"""

from __future__ import annotations

import numpy as np


def chem(B: np.ndarray, p, q, r, s) -> np.ndarray:
    """(pq|rs) for index arrays p, q, r, s; result shape [|p|,|q|,|r|,|s|]."""
    Bpq = B[:, p][:, :, q]
    Brs = B[:, r][:, :, s]
    return np.einsum("Ppq,Prs->pqrs", Bpq, Brs, optimize=True)


def antisym(B: np.ndarray, p, q, r, s) -> np.ndarray:
    """<pq||rs> = (pr|qs) - (ps|qr) for index arrays p, q, r, s."""
    direct = chem(B, p, r, q, s).transpose(0, 2, 1, 3)  # (pr|qs) -> [p,q,r,s]
    exch = chem(B, p, s, q, r).transpose(0, 2, 3, 1)  # (ps|qr) -> [p,q,r,s]
    return direct - exch
