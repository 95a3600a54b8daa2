"""Determinant-space (full CI) engine and brute-force intermediate-state
representation (ISR) for tiny spinor spaces.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this.

This module is the independent pin for the CVS-ADC(2) element formulas in
``oracle.adc2``.  It never uses those formulas: it builds the many-electron
Hamiltonian in the N-electron determinant space from second-quantised
operators, finds the exact ground state of H(lambda) = H0 + lambda*V, and
constructs the intermediate states exactly as section "Relativistic Algebraic
Diagrammatic Construction Method" defines them:

* correlated excited states C_J Psi_0 with C_J in {a_a^+ a_i ; a_a^+ a_b^+ a_i
  a_j} (a<b, i<j) (the excitation-operator equation and Eq. ces);
* precursor states: Gram-Schmidt orthogonalisation of each class against
  every lower class (the precursor equation);
* symmetric orthonormalisation S^{-1/2} inside a class (the S^{-1/2} and
  overlap equations);
* M_IJ = <Psi~_I|H - E_0|Psi~_J> (the secular-matrix equation), and the
  modified transition moments F_I = <Psi~_I|D|Psi_0> (section "Properties in
  ISR formulation");
* the exact ground state's own expansion (its determinant amplitudes and
  one-particle density), for the Rayleigh-Schrodinger pieces.

The perturbation expansion M = M(0) + M(1) + M(2) + ... (Eq. 12) is then
read off as the Taylor coefficients of M(lambda) at lambda = 0, obtained by a
least-squares polynomial fit on Chebyshev nodes.

Hamiltonian: H = sum_pq h_pq a_p^+ a_q + 1/4 sum_pqrs <pq||rs> a_p^+ a_q^+
a_s a_r with h = diag(eps) - sum_i <p i||q i>, so that the Fock matrix of the
reference determinant is exactly diag(eps) (canonical Hartree-Fock, Eqs. 4c
and x2c).  H0 = sum_p eps_p a_p^+ a_p is the Moller-Plesset partitioning.
Antisymmetrised integrals come from the Cholesky vectors as
<pq||rs> = (pr|qs) - (ps|qr), (pq|rs) = sum_P B^P_pq B^P_rs (section
"Implementation and Computational Details").
"""

from __future__ import annotations

import itertools

import numpy as np


# --------------------------------------------------------------------------
# fermionic operators on bit-string determinants
# --------------------------------------------------------------------------

def _popcount_below(det: int, p: int) -> int:
    return bin(det & ((1 << p) - 1)).count("1")


def apply_string(ops, det: int):
    """Apply an operator string to |det>.

    ``ops`` lists (create, orbital) pairs in the order they appear in the
    written product, left to right; they act right to left.  A determinant is
    a_{p1}^+ a_{p2}^+ ... |vac> with p1 < p2 < ..., encoded as a bit mask.
    Returns (sign, new_det) or None if the result vanishes.
    """
    sign = 1
    for create, p in reversed(ops):
        occ = (det >> p) & 1
        if create:
            if occ:
                return None
            if _popcount_below(det, p) & 1:
                sign = -sign
            det |= 1 << p
        else:
            if not occ:
                return None
            if _popcount_below(det, p) & 1:
                sign = -sign
            det &= ~(1 << p)
    return sign, det


class DetSpace:
    """All determinants of ``nelec`` electrons in ``n`` spinors."""

    def __init__(self, n: int, nelec: int):
        self.n = n
        self.nelec = nelec
        dets = []
        for occ in itertools.combinations(range(n), nelec):
            d = 0
            for p in occ:
                d |= 1 << p
            dets.append(d)
        self.dets = dets
        self.index = {d: k for k, d in enumerate(dets)}
        self.dim = len(dets)
        self.ref = (1 << nelec) - 1  # lowest nelec spinors occupied

    def occupied(self, det: int):
        return [p for p in range(self.n) if (det >> p) & 1]

    def operator(self, ops):
        """Sparse representation (src, dst, sign) of a number-conserving
        operator string restricted to this space."""
        src, dst, sgn = [], [], []
        for k, d in enumerate(self.dets):
            r = apply_string(ops, d)
            if r is None:
                continue
            s, d2 = r
            src.append(k)
            dst.append(self.index[d2])
            sgn.append(s)
        return (np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64),
                np.array(sgn, dtype=np.float64))

    @staticmethod
    def act(op, vec: np.ndarray) -> np.ndarray:
        src, dst, sgn = op
        out = np.zeros_like(vec)
        np.add.at(out, dst, sgn * vec[src])
        return out

    def hamiltonian(self, h: np.ndarray, g: np.ndarray) -> np.ndarray:
        """Dense H = sum h_pq p^+ q + sum_{p<q, r<s} g_pqrs p^+ q^+ s r.

        The restricted pair sum equals 1/4 of the unrestricted sum for an
        antisymmetrised g (both index pairs flip sign together)."""
        n = self.n
        H = np.zeros((self.dim, self.dim), dtype=np.complex128)
        for col, d in enumerate(self.dets):
            occ = self.occupied(d)
            for q in occ:
                for p in range(n):
                    if abs(h[p, q]) == 0.0:
                        continue
                    r = apply_string([(1, p), (0, q)], d)
                    if r is None:
                        continue
                    s, d2 = r
                    H[self.index[d2], col] += s * h[p, q]
            for r_, s_ in itertools.combinations(occ, 2):
                r1 = apply_string([(0, s_), (0, r_)], d)
                if r1 is None:
                    continue
                s1, dm = r1
                for p, q in itertools.combinations(range(n), 2):
                    val = g[p, q, r_, s_]
                    if val == 0.0:
                        continue
                    r2 = apply_string([(1, p), (1, q)], dm)
                    if r2 is None:
                        continue
                    s2, d2 = r2
                    H[self.index[d2], col] += s1 * s2 * val
        return H

    def one_body(self, d1: np.ndarray) -> np.ndarray:
        """Dense matrix of sum_pq d_pq p^+ q."""
        H = np.zeros((self.dim, self.dim), dtype=np.complex128)
        for col, d in enumerate(self.dets):
            for q in self.occupied(d):
                for p in range(self.n):
                    r = apply_string([(1, p), (0, q)], d)
                    if r is None:
                        continue
                    s, d2 = r
                    H[self.index[d2], col] += s * d1[p, q]
        return H

    def diag_h0(self, eps: np.ndarray) -> np.ndarray:
        return np.array([sum(eps[p] for p in self.occupied(d)) for d in self.dets])


# --------------------------------------------------------------------------
# model Hamiltonian from (eps, B)
# --------------------------------------------------------------------------

def full_antisym_integrals(B: np.ndarray) -> np.ndarray:
    """<pq||rs> over all spinors, straight from the definition."""
    chem = np.einsum("Ppq,Prs->pqrs", B, B)  # (pq|rs)
    phys = chem.transpose(0, 2, 1, 3)  # <pq|rs> = (pr|qs)
    return phys - phys.transpose(0, 1, 3, 2)


def model_hamiltonian(space: DetSpace, eps: np.ndarray, B: np.ndarray):
    """Return (H, H0 diagonal, E_HF) for canonical-HF one-electron part."""
    nocc = space.nelec
    g = full_antisym_integrals(B)
    h = np.diag(eps).astype(np.complex128)
    for i in range(nocc):
        h = h - g[:, i, :, i]
    H = space.hamiltonian(h, g)
    h0 = space.diag_h0(eps)
    e_hf = H[space.index[space.ref], space.index[space.ref]].real
    return H, h0, e_hf


# --------------------------------------------------------------------------
# brute-force ISR
# --------------------------------------------------------------------------

def _inv_sqrt(S: np.ndarray) -> np.ndarray:
    w, V = np.linalg.eigh(S)
    if w.min() <= 0:
        raise np.linalg.LinAlgError("overlap matrix not positive definite")
    return (V / np.sqrt(w)) @ V.conj().T


class ISR:
    """Exact ISR of H(lambda) in the full singles and doubles classes.

    The CVS quantities are the core-singles (I, a) and core-valence doubles
    (I, j, a<b) rows and columns of the full ISR (CVS as a projection: the
    CVS section drops couplings to valence- and doubly-core-excited states,
    it does not change the intermediate states of the kept classes).
    """

    def __init__(self, eps, B, ncore, nval, nvirt, dip=None):
        self.ncore, self.nval, self.nvirt = ncore, nval, nvirt
        o = ncore + nval
        n = o + nvirt
        self.space = DetSpace(n, o)
        self.H, self.h0, self.e_hf = model_hamiltonian(self.space, eps, B)
        self.V = self.H - np.diag(self.h0)
        occ = range(o)
        vir = range(o, n)
        self.singles = [(i, a) for i in occ for a in vir]
        self.doubles = [(i, j, a, b) for i, j in itertools.combinations(occ, 2)
                        for a, b in itertools.combinations(vir, 2)]
        sp = self.space
        self.op_s = [sp.operator([(1, a), (0, i)]) for i, a in self.singles]
        self.op_d = [sp.operator([(1, a), (1, b), (0, i), (0, j)])
                     for i, j, a, b in self.doubles]
        # CVS selections (indices into the full lists), in packed CVS order:
        # singles s = I*nvirt + a; doubles ((I*nval + j)*npair + pair(a,b))
        self.cvs_s = [k for k, (i, a) in enumerate(self.singles) if i < ncore]
        dpos = {d: k for k, d in enumerate(self.doubles)}
        self.cvs_d = []
        for I in range(ncore):
            for j in range(ncore, o):
                for a, b in itertools.combinations(range(nvirt), 2):
                    self.cvs_d.append(dpos[(I, j, o + a, o + b)])
        self.D = None
        if dip is not None:
            self.D = [sp.one_body(dip[x]) for x in range(dip.shape[0])]

    def at(self, lam: float):
        """Return (M_cvs, F_cvs or None, E0) at coupling strength lam."""
        Hl = np.diag(self.h0) + lam * self.V
        E, U = np.linalg.eigh(Hl)
        E0 = E[0]
        psi0 = U[:, 0]
        ref = self.space.index[self.space.ref]
        psi0 = psi0 * (np.conj(psi0[ref]) / abs(psi0[ref]))
        act = self.space.act
        Cs = np.stack([act(op, psi0) for op in self.op_s], axis=1)
        Cs = Cs - np.outer(psi0, psi0.conj() @ Cs)
        Ts = Cs @ _inv_sqrt(Cs.conj().T @ Cs)
        Cd = np.stack([act(op, psi0) for op in self.op_d], axis=1)
        Cd = Cd - np.outer(psi0, psi0.conj() @ Cd)
        Cd = Cd - Ts @ (Ts.conj().T @ Cd)
        Td = Cd @ _inv_sqrt(Cd.conj().T @ Cd)
        basis = np.concatenate([Ts[:, self.cvs_s], Td[:, self.cvs_d]], axis=1)
        Hs = Hl - E0 * np.eye(Hl.shape[0])
        M = basis.conj().T @ Hs @ basis
        F = None
        if self.D is not None:
            F = np.stack([basis.conj().T @ (Dx @ psi0) for Dx in self.D], axis=0)
        return M, F, E0

    def taylor(self, order: int = 2, h: float = 0.02, deg: int = 8,
               npts: int = 17):
        """Taylor coefficients [0..order] of M(lambda), F(lambda), E0(lambda)
        at lambda = 0 from a least-squares fit on Chebyshev nodes."""
        k = np.arange(npts)
        lams = h * np.cos((2 * k + 1) * np.pi / (2 * npts))
        Ms, Fs, Es = [], [], []
        for lam in lams:
            M, F, E0 = self.at(lam)
            Ms.append(M)
            Fs.append(F)
            Es.append(E0)
        Vm = np.vander(lams / h, deg + 1, increasing=True)
        pinv = np.linalg.pinv(Vm)  # (deg+1, npts)
        scale = h ** -np.arange(deg + 1)

        def fit(stack):
            arr = np.stack(stack, axis=0)
            flat = arr.reshape(npts, -1)
            c = (pinv @ flat) * scale[:, None]
            return c[: order + 1].reshape((order + 1,) + arr.shape[1:])

        cM = fit(Ms)
        cF = fit(Fs) if Fs[0] is not None else None
        cE = fit([np.array([e]) for e in Es])[:, 0]
        return cM, cF, cE

    def ground_rdm1_taylor(self, order: int = 2, h: float = 0.02, deg: int = 8,
                           npts: int = 17):
        """Taylor coefficients [0..order] at lambda = 0 of the exact ground
        state's one-particle density matrix, gamma[p, q](lambda) =
        <Psi_0(lambda)| a_p^+ a_q |Psi_0(lambda)>, over all spinors, from the
        same Chebyshev least-squares fit as ``taylor``.  At lambda^2 its
        virtual-virtual block is the second-order (MP2) density that Eq. 15
        writes in closed form."""
        sp = self.space
        n = sp.n
        ops = {(p, q): sp.operator([(1, p), (0, q)]) for p in range(n) for q in range(n)}
        k = np.arange(npts)
        lams = h * np.cos((2 * k + 1) * np.pi / (2 * npts))
        gs = []
        for lam in lams:
            Hl = np.diag(self.h0) + lam * self.V
            _, U = np.linalg.eigh(Hl)
            psi0 = U[:, 0]
            g = np.zeros((n, n), dtype=np.complex128)
            for (p, q), op in ops.items():
                g[p, q] = np.vdot(psi0, sp.act(op, psi0))
            gs.append(g)
        Vm = np.vander(lams / h, deg + 1, increasing=True)
        c = (np.linalg.pinv(Vm) @ np.stack(gs).reshape(npts, -1)) * (h ** -np.arange(deg + 1))[:, None]
        return c[: order + 1].reshape(order + 1, n, n)

    def ground_state_taylor(self, order: int = 2, h: float = 0.02, deg: int = 8,
                            npts: int = 17):
        """Taylor coefficients [0..order] at lambda = 0 of the exact ground
        state Psi_0(lambda) of H(lambda), normalised with <Phi_0|Psi_0> real
        and positive, as vectors over the determinants (the same Chebyshev
        least-squares fit as ``taylor``).  Its lambda^1 and lambda^2
        coefficients on a determinant are the first- and second-order
        amplitudes of Rayleigh-Schrodinger theory (the normalisation enters
        only the reference coefficient at lambda^2)."""
        ref = self.space.index[self.space.ref]
        k = np.arange(npts)
        lams = h * np.cos((2 * k + 1) * np.pi / (2 * npts))
        vecs = []
        for lam in lams:
            _, U = np.linalg.eigh(np.diag(self.h0) + lam * self.V)
            p = U[:, 0]
            vecs.append(p * (np.conj(p[ref]) / abs(p[ref])))
        Vm = np.vander(lams / h, deg + 1, increasing=True)
        c = (np.linalg.pinv(Vm) @ np.stack(vecs)) * (h ** -np.arange(deg + 1))[:, None]
        return c[: order + 1]

    def amplitude(self, coeff: np.ndarray, creators, annihilators) -> complex:
        """<Phi|coeff> for Phi = a^+_{c1} a^+_{c2} .. a_{k2} a_{k1} Phi_0, the
        determinant made by the given creators (left to right) and
        annihilators (applied first, in reversed order)."""
        ops = [(1, c) for c in creators] + [(0, k) for k in reversed(annihilators)]
        ref = np.zeros(self.space.dim, dtype=np.complex128)
        ref[self.space.index[self.space.ref]] = 1.0
        return np.vdot(self.space.act(self.space.operator(ops), ref), coeff)

    def rspt_e2(self) -> float:
        """Second-order Rayleigh-Schrodinger energy from the determinant
        space: sum_D |<D|V|Phi0>|^2 / (E0(0) - E_D(0))."""
        ref = self.space.index[self.space.ref]
        col = self.V[:, ref]
        den = self.h0[ref] - self.h0
        mask = np.arange(self.space.dim) != ref
        return float(np.sum(np.abs(col[mask]) ** 2 / den[mask]))
