"""Reference gradient of a sum of CVS-ADC(2) roots, by automatic
differentiation of the explicit matrix in PyTorch (CPU, complex128).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

E(eps, B) = sum of the lowest nroots eigenvalues of the dense CVS-ADC(2)
matrix built from the same explicit formulas as ``oracle.adc2`` (integrals
from the Cholesky vectors, MP2 amplitudes, M11 through second order, M21,
M22), written with torch operations so that autograd differentiates the
eigenvalues (torch.linalg.eigvalsh).  Tiny spaces only (dense matrix).

Gradient convention: g_z = dE/dRe z + i dE/dIm z (PyTorch's), and the B
gradient is projected on Hermitian matrices, since every B^P is
constrained Hermitian; for a Hermitian dB, dE = Re sum conj(g) dB.

Pinned by central finite differences of ``oracle.adc2`` eigenvalues along
random Hermitian directions (tests/test_oracle_pins.py).
"""

from __future__ import annotations

import itertools

import numpy as np
import torch


def _asym(B, p, q, r, s):
    """<pq||rs> = (pr|qs) - (ps|qr) as [|p|, |q|, |r|, |s|]."""
    def chem(a, b, c, d):
        return torch.einsum("Pab,Pcd->abcd", B[:, a][:, :, b], B[:, c][:, :, d])
    direct = chem(p, r, q, s).permute(0, 2, 1, 3)
    exch = chem(p, s, q, r).permute(0, 2, 3, 1)
    return direct - exch


def adc_matrix(eps, B, ncore, nval, nvirt):
    """Dense CVS-ADC(2) matrix (torch), same formulas as oracle.adc2."""
    o = ncore + nval
    C = torch.arange(ncore)
    W = torch.arange(ncore, o)
    O = torch.arange(o)
    V = torch.arange(o, o + nvirt)
    eo, ev = eps[O], eps[V]
    D = (eo[:, None, None, None] + eo[None, :, None, None]
         - ev[None, None, :, None] - ev[None, None, None, :])
    t2 = _asym(B, V, V, O, O).permute(2, 3, 0, 1) / D
    tc = t2[C]
    oovv = _asym(B, O, O, V, V)
    vvoo = _asym(B, V, V, O, O)
    covv = _asym(B, C, O, V, V)
    vvco = _asym(B, V, V, C, O)
    vcvc = _asym(B, V, C, V, C)
    Ivv = (torch.einsum("klac,klbc->ab", t2, oovv)
           + torch.einsum("ackl,klbc->ab", vvoo, torch.conj(t2)))
    Joo = (torch.einsum("Jkcd,Ikcd->IJ", covv, tc)
           + torch.einsum("Jkcd,cdIk->IJ", torch.conj(tc), vvco))
    K = (torch.einsum("Ikac,Jkbc->IaJb", tc, covv)
         + torch.einsum("acIk,Jkbc->IaJb", vvco, torch.conj(tc)))
    eyeC = torch.eye(ncore, dtype=B.dtype)
    eyeV = torch.eye(nvirt, dtype=B.dtype)
    diag = (ev[None, :] - eps[C][:, None]).to(B.dtype)
    m11 = torch.einsum("IJ,ab,Ia->IaJb", eyeC, eyeV, diag)
    m11 = m11 - torch.einsum("aJbI->IaJb", vcvc)
    m11 = m11 - 0.25 * torch.einsum("IJ,ab->IaJb", eyeC, Ivv)
    m11 = m11 - 0.25 * torch.einsum("IJ,ab->IaJb", Joo, eyeV)
    m11 = m11 + 0.5 * K
    N1 = ncore * nvirt
    m11 = m11.reshape(N1, N1)
    # M21 over all (a, b): -d_IK <ab||cj> + d_ac <Kb||Ij> - d_bc <Ka||Ij>
    vvvw = _asym(B, V, V, V, W)  # <ab||cj> [a, b, c, j]
    cvcw = _asym(B, C, V, C, W)  # <Kb||Ij> [K, b, I, j]
    full = (-torch.einsum("IK,abcj->IjabKc", eyeC, vvvw)
            + torch.einsum("ac,KbIj->IjabKc", eyeV, cvcw)
            - torch.einsum("bc,KaIj->IjabKc", eyeV, cvcw))
    pairs = list(itertools.combinations(range(nvirt), 2))
    pa = torch.tensor([p[0] for p in pairs])
    pb = torch.tensor([p[1] for p in pairs])
    m21 = full[:, :, pa, pb].reshape(ncore * nval * len(pairs), N1)
    ec, ew = eps[C], eps[W]
    m22 = (ev[pa][None, None, :] + ev[pb][None, None, :]
           - ec[:, None, None] - ew[None, :, None]).reshape(-1)
    top = torch.cat([m11, m21.conj().T], dim=1)
    bot = torch.cat([m21, torch.diag(m22).to(B.dtype)], dim=1)
    return torch.cat([top, bot], dim=0)


def energy_gradient(eps, B, ncore, nval, nvirt, nroots, root_mask=None):
    """(roots, dE/deps, dE/dB projected Hermitian) for E = sum of selected
    lowest roots."""
    e = torch.tensor(np.asarray(eps), dtype=torch.float64, requires_grad=True)
    b = torch.tensor(np.asarray(B), dtype=torch.complex128, requires_grad=True)
    M = adc_matrix(e, b, ncore, nval, nvirt)
    M = 0.5 * (M + M.conj().T)
    w = torch.linalg.eigvalsh(M)[:nroots]
    mask = torch.ones(nroots, dtype=torch.float64) if root_mask is None else \
        torch.tensor(np.asarray(root_mask), dtype=torch.float64)
    E = (w * mask).sum()
    E.backward()
    gB = b.grad.numpy()
    gB = 0.5 * (gB + np.conj(gB.transpose(0, 2, 1)))
    return w.detach().numpy(), e.grad.numpy().copy(), gB
