"""CVS-ADC(2) secular matrix, sigma-vector, transition moments and
eigen-solvers, written out from the definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Spaces (section "Core-Valence Separation (CVS)"): excitation operators
a_a^+ a_I (core singles) and a_a^+ a_b^+ a_I a_j (core-valence doubles,
I core, j valence, a < b), acting on the ground state.  The basis vectors of
the packed CVS space are, at zeroth order, the normalised determinants
a_a^+ a_I |Phi_0> and a_a^+ a_b^+ a_I a_j |Phi_0> -- exactly the operator
order the CVS section prints.

* singles index  s = I * nvirt + a
* doubles index  d = (I * nval + j) * npair + pair(a, b),
  pair(a, b) = a * (2 nvirt - a - 1) / 2 + (b - a - 1) for a < b.

The ADC(2) matrix (Eqs. 11-12: M through second order in the singles
block, first order in the singles-doubles coupling, zeroth order in the
doubles block), restricted to the CVS rows and columns:

  M11_{Ia,Jb} = d_IJ d_ab (e_a - e_I) - <aJ||bI>
                - 1/4 d_IJ Ivv_ab - 1/4 d_ab Joo_IJ + 1/2 K_{Ia,Jb}
  Ivv_ab   = sum_{ckl} [ t^{ac}_{kl} <kl||bc> + <ac||kl> conj(t^{bc}_{kl}) ]
  Joo_IJ   = sum_{cdk} [ <Jk||cd> t^{cd}_{Ik} + conj(t^{cd}_{Jk}) <cd||Ik> ]
  K_{Ia,Jb}= sum_{ck}  [ t^{ac}_{Ik} <Jk||bc> + <ac||Ik> conj(t^{bc}_{Jk}) ]
  M21_{(Ijab),(Kc)} = - d_IK <ab||cj> + d_ac <Kb||Ij> - d_bc <Ka||Ij>
  M12 = M21^H,   M22 = diag(e_a + e_b - e_I - e_j)

with k, l over all correlated occupied spinors (core included) and t the
MP2 amplitudes of ``oracle.mp2``.  The paper prints only the ISR definition
of M (section "Relativistic Algebraic Diagrammatic Construction Method");
every coefficient and sign above is pinned against the brute-force ISR of
``oracle.fci`` (tests/test_oracle_pins.py): M11 through lambda^2, M21 at
lambda^1, M22 at lambda^0.

Modified transition moments F_J = <Psi~_J|D|Psi_0> (section "Properties in
ISR formulation"), through first order (pinned by the same brute force):

  F_{Ia}   = d_aI + sum_{kc} d_kc t^{ac}_{Ik}
  F_{Ijab} = - sum_c (d_ac t^{cb}_{Ij} - d_bc t^{ca}_{Ij})
             + sum_k (d_kI t^{ab}_{kj} - d_kj t^{ab}_{kI})

and, with ``order=2``, the second-order singles term (the full ISR's
singles class, CVS as a projection; s and u the second-order ground-state
amplitudes of ``oracle.mp2``):

  F^(2)_{Ia} = sum_c d_ac s_Ic - sum_k d_kI s_ka + sum_{kc} d_kc u^{ac}_{Ik}
               - 1/4 sum_k d_ak H_kI + 1/2 sum_{ld} w_ld t^{ad}_{Il}
               - 1/4 sum_c d_cI P_ca
  H_kI = sum_{lde} conj(t^{de}_{kl}) t^{de}_{Il},
  P_ca = sum_{lmd} conj(t^{cd}_{lm}) t^{ad}_{lm},
  w_ld = sum_{ck} d_ck conj(t^{cd}_{kl}).

The last three terms are half of sum_{ck} d_ck (<Psi1|a_I^+ a_a a_c^+ a_k|Psi1>
- <Psi1|Psi1> d_Ik d_ac): the ground state's own second-order pieces carry
that expectation value whole, and the S^{-1/2} of the singles class takes
back half of it.  Pinned by the brute-force ISR at lambda^2.

T_n = X_n^H F, f_n = 2/3 omega_n |T_n|^2.
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg
import scipy.optimize
import scipy.sparse.linalg

from .integrals import antisym
from .mp2 import second_order_doubles, second_order_singles, t2_amplitudes


# --------------------------------------------------------------------------
# CVS spaces and packing
# --------------------------------------------------------------------------

def sizes(ncore, nval, nvirt):
    npair = nvirt * (nvirt - 1) // 2
    return ncore * nvirt, npair, ncore * nval * npair


def pair_list(nvirt):
    """All (a, b) with a < b in packed order."""
    return np.array(list(itertools.combinations(range(nvirt), 2)),
                    dtype=np.int64).reshape(-1, 2)


def doubles_list(ncore, nval, nvirt):
    """[N2, 4] int64 table of (I, j, a, b) in packed order, enumerated by
    plain nested loops (I outer, then j, then a < b)."""
    rows = []
    for I in range(ncore):
        for j in range(nval):
            for a in range(nvirt):
                for b in range(a + 1, nvirt):
                    rows.append((I, j, a, b))
    return np.array(rows, dtype=np.int64).reshape(-1, 4)


def pack(full, nvirt):
    """[ncore, nval, v, v] -> [N2] taking a < b."""
    pl = pair_list(nvirt)
    return full[:, :, pl[:, 0], pl[:, 1]].reshape(-1)


def unpack(x2, ncore, nval, nvirt):
    """[N2] -> antisymmetric [ncore, nval, v, v]."""
    pl = pair_list(nvirt)
    out = np.zeros((ncore, nval, nvirt, nvirt), dtype=np.complex128)
    x = x2.reshape(ncore, nval, -1)
    out[:, :, pl[:, 0], pl[:, 1]] = x
    out[:, :, pl[:, 1], pl[:, 0]] = -x
    return out


def m22(eps, ncore, nval, nvirt):
    """Diagonal doubles block e_a + e_b - e_I - e_j in packed order."""
    o = ncore + nval
    pl = pair_list(nvirt)
    ec, ew, ev = eps[:ncore], eps[ncore:o], eps[o:]
    return (ev[pl[:, 0]][None, None, :] + ev[pl[:, 1]][None, None, :]
            - ec[:, None, None] - ew[None, :, None]).reshape(-1)


# --------------------------------------------------------------------------
# explicit blocks
# --------------------------------------------------------------------------

def _idx(ncore, nval, nvirt):
    o = ncore + nval
    return (np.arange(ncore), np.arange(ncore, o), np.arange(o),
            np.arange(o, o + nvirt))


def m11(eps, B, ncore, nval, nvirt, t2=None, second_order=True):
    """Explicit core-singles block M11 as an [N1, N1] matrix."""
    C, W, O, V = _idx(ncore, nval, nvirt)
    ec, ev = eps[C], eps[V]
    N1 = ncore * nvirt
    m = np.zeros((ncore, nvirt, ncore, nvirt), dtype=np.complex128)
    idx_c = np.arange(ncore)[:, None]
    idx_v = np.arange(nvirt)[None, :]
    m[idx_c, idx_v, idx_c, idx_v] = ev[None, :] - ec[:, None]
    vcvc = antisym(B, V, C, V, C)  # <aJ||bI> as [a, J, b, I]
    m -= np.einsum("aJbI->IaJb", vcvc)
    if second_order:
        if t2 is None:
            t2 = t2_amplitudes(eps, B, ncore, nval, nvirt)
        tc = t2[C]  # t^{ab}_{Ik} as [I, k, a, b]
        oovv = antisym(B, O, O, V, V)  # <kl||bc>
        vvoo = antisym(B, V, V, O, O)  # <ac||kl>
        Ivv = (np.einsum("klac,klbc->ab", t2, oovv, optimize=True)
               + np.einsum("ackl,klbc->ab", vvoo, np.conj(t2), optimize=True))
        covv = antisym(B, C, O, V, V)  # <Jk||cd>
        vvco = antisym(B, V, V, C, O)  # <cd||Ik>
        Joo = (np.einsum("Jkcd,Ikcd->IJ", covv, tc, optimize=True)
               + np.einsum("Jkcd,cdIk->IJ", np.conj(tc), vvco, optimize=True))
        K = (np.einsum("Ikac,Jkbc->IaJb", tc, covv, optimize=True)
             + np.einsum("acIk,Jkbc->IaJb", vvco, np.conj(tc), optimize=True))
        m -= 0.25 * np.einsum("IJ,ab->IaJb", np.eye(ncore), Ivv)
        m -= 0.25 * np.einsum("IJ,ab->IaJb", Joo, np.eye(nvirt))
        m += 0.5 * K
    return m.reshape(N1, N1)


def m21(eps, B, ncore, nval, nvirt):
    """Explicit singles->doubles coupling M21 as a dense [N2, N1] matrix."""
    C, W, O, V = _idx(ncore, nval, nvirt)
    pl = pair_list(nvirt)
    npair = pl.shape[0]
    vvvw = antisym(B, V, V, V, W)  # <ab||cj> [a, b, c, j]
    cvcw = antisym(B, C, V, C, W)  # <Kb||Ij> [K, b, I, j]
    out = np.zeros((ncore, nval, npair, ncore, nvirt), dtype=np.complex128)
    g = vvvw[pl[:, 0], pl[:, 1]]  # [p, c, j]
    for I in range(ncore):
        out[I, :, :, I, :] -= g.transpose(2, 0, 1)
    pa, pb = pl[:, 0], pl[:, 1]
    pidx = np.arange(npair)
    # + d_ac <Kb||Ij>: column (K, c = a)
    out[:, :, pidx, :, pa] += cvcw[:, pb, :, :].transpose(1, 2, 3, 0)
    # - d_bc <Ka||Ij>: column (K, c = b)
    out[:, :, pidx, :, pb] -= cvcw[:, pa, :, :].transpose(1, 2, 3, 0)
    return out.reshape(ncore * nval * npair, ncore * nvirt)


def adc_matrix(eps, B, ncore, nval, nvirt, second_order=True):
    """Dense CVS-ADC(2) matrix [[M11, M12], [M21, diag M22]] (tiny spaces)."""
    a = m11(eps, B, ncore, nval, nvirt, second_order=second_order)
    c = m21(eps, B, ncore, nval, nvirt)
    if not second_order:
        c = np.zeros_like(c)
    d = m22(eps, ncore, nval, nvirt)
    return np.block([[a, c.conj().T], [c, np.diag(d).astype(np.complex128)]])


# --------------------------------------------------------------------------
# matrix-free sigma from explicit integral blocks
# --------------------------------------------------------------------------

class Sigma:
    """sigma = M x without the dense matrix.

    M11 is explicit; the couplings use the explicit integrals <ab||cj>
    (built per valence spinor j) and <Kb||Ij>, exactly as in M21 above.
    """

    def __init__(self, eps, B, ncore, nval, nvirt, M11=None, cache_blocks=True):
        self.eps, self.B = eps, B
        self.ncore, self.nval, self.nvirt = ncore, nval, nvirt
        self.M11 = M11 if M11 is not None else m11(eps, B, ncore, nval, nvirt)
        self.d22 = m22(eps, ncore, nval, nvirt)
        C, W, O, V = _idx(ncore, nval, nvirt)
        self.cvcw = antisym(B, C, V, C, W)  # [K, b, I, j]
        self.cache_blocks = cache_blocks
        self._vvv = {}

    def block(self, j, rows=None):
        """<ab||cj> for valence spinor j, as [a, b, c] (a over `rows`, a
        slice of the virtual indices, default all)."""
        if rows is None and j in self._vvv:
            return self._vvv[j]
        C, W, O, V = _idx(self.ncore, self.nval, self.nvirt)
        Va = V if rows is None else V[rows]
        g = antisym(self.B, Va, V, V, W[j:j + 1])[..., 0]
        if self.cache_blocks and rows is None:
            self._vvv[j] = g
        return g

    def coupling_block(self, X, Y, j, rows=None):
        """Valence spinor j's share of the couplings, from X = x1 as [K, c]
        and Y = the unpacked doubles [I, j, a, b]: (M21 x1)[:, j] as [I, a, b]
        and its term of M12 x2 as [K, c].  With `rows` (a slice of the first
        virtual index a) only those rows of (M21 x1)[:, j] and their part of
        the M12 x2 sum are formed: a bounded piece of the same work."""
        g = self.block(j, rows)
        h = self.cvcw
        ra = slice(None) if rows is None else rows
        # M21 x1
        s2j = (-np.einsum("abc,Ic->Iab", g, X)
               + np.einsum("KbI,Ka->Iab", h[:, :, :, j], X[:, ra])
               - np.einsum("KaI,Kb->Iab", h[:, ra, :, j], X))
        # M12 x2 = sum over a<b of conj(M21) x2 = 1/2 over all a, b; the
        # <ab||cj> term sums over the rows a, the <Kb||Ij> term fills the
        # columns c in the rows
        s1j = -0.5 * np.einsum("abc,Kab->Kc", np.conj(g), Y[:, j, ra])
        s1j[:, ra] += np.einsum("KbI,Icb->Kc", np.conj(h[:, :, :, j]), Y[:, j, ra])
        return s2j, s1j

    def __call__(self, x1, x2, jlist=None):
        nc, nw, nv = self.ncore, self.nval, self.nvirt
        X = x1.reshape(nc, nv)
        Y = unpack(x2, nc, nw, nv)  # [I, j, a, b]
        s1 = (self.M11 @ x1).reshape(nc, nv)
        s2 = np.zeros((nc, nw, nv, nv), dtype=np.complex128)
        jl = range(nw) if jlist is None else jlist
        for j in jl:
            s2[:, j], s1j = self.coupling_block(X, Y, j)
            s1 += s1j
        s2 = pack(s2, nv) + self.d22 * x2
        return s1.reshape(-1), s2


# --------------------------------------------------------------------------
# transition moments and oscillator strengths
# --------------------------------------------------------------------------

def singles_moments_second_order(eps, B, dip, ncore, nval, nvirt, t2=None):
    """F^(2)_{Ia} for each Cartesian component, as [x, I, a] (module
    docstring)."""
    C, W, O, V = _idx(ncore, nval, nvirt)
    if t2 is None:
        t2 = t2_amplitudes(eps, B, ncore, nval, nvirt)
    s = second_order_singles(eps, B, ncore, nval, nvirt, t2=t2)  # [k, c]
    u = second_order_doubles(eps, B, ncore, nval, nvirt, t2=t2, rows=C)  # [I, k, a, c]
    tI = t2[C]  # [I, l, a, d]
    H = np.einsum("klde,Ilde->kI", np.conj(t2), tI, optimize=True)
    P = np.einsum("lmcd,lmad->ca", np.conj(t2), t2, optimize=True)
    out = []
    for x in range(dip.shape[0]):
        d = dip[x]
        dvv, doo, dov, dvo = (d[np.ix_(V, V)], d[np.ix_(O, O)], d[np.ix_(O, V)],
                              d[np.ix_(V, O)])
        w = np.einsum("ck,klcd->ld", dvo, np.conj(t2), optimize=True)
        f2 = (np.einsum("ac,Ic->Ia", dvv, s[C])
              - np.einsum("kI,ka->Ia", doo[:, C], s)
              + np.einsum("kc,Ikac->Ia", dov, u, optimize=True)
              - 0.25 * np.einsum("ak,kI->Ia", dvo, H)
              + 0.5 * np.einsum("ld,Ilad->Ia", w, tI)
              - 0.25 * np.einsum("cI,ca->Ia", dvo[:, C], P))
        out.append(f2)
    return np.stack(out)


def transition_moments(eps, B, dip, ncore, nval, nvirt, t2=None, order=1):
    """F[x] = [F_S (N1), F_D (N2)] for each Cartesian component x, through
    first order; order=2 adds the second-order singles term."""
    C, W, O, V = _idx(ncore, nval, nvirt)
    if t2 is None:
        t2 = t2_amplitudes(eps, B, ncore, nval, nvirt)
    f2 = (singles_moments_second_order(eps, B, dip, ncore, nval, nvirt, t2=t2)
          if order >= 2 else None)
    out = []
    for x in range(dip.shape[0]):
        d = dip[x]
        fs = d[np.ix_(V, C)].T + np.einsum("kc,Ikac->Ia", d[np.ix_(O, V)], t2[C])
        if f2 is not None:
            fs = fs + f2[x]
        dvv = d[np.ix_(V, V)]
        doo = d[np.ix_(O, O)]
        tcw = t2[C][:, W]  # t^{ab}_{Ij}
        fd = (-np.einsum("ac,Ijcb->Ijab", dvv, tcw)
              + np.einsum("bc,Ijca->Ijab", dvv, tcw)
              + np.einsum("kI,kjab->Ijab", doo[:, C], t2[:, W])
              - np.einsum("kj,kIab->Ijab", doo[:, W], t2[:, C]))
        out.append(np.concatenate([fs.reshape(-1), pack(fd, nvirt)]))
    return np.stack(out)


def oscillator_strengths(omega, X, F):
    """f_n = 2/3 omega_n sum_x |X_n^H F^x|^2; X as [nroots, N]."""
    T = np.conj(X) @ F.T  # [nroots, 3]
    return (2.0 / 3.0) * omega * np.sum(np.abs(T) ** 2, axis=1)


def fix_phase(X):
    """Make the largest-|.| component of each row real and positive."""
    X = X.copy()
    for n in range(X.shape[0]):
        k = np.argmax(np.abs(X[n]))
        X[n] *= np.conj(X[n, k]) / abs(X[n, k])
    return X


# --------------------------------------------------------------------------
# eigen-solvers
# --------------------------------------------------------------------------

def eig_dense(M, nroots):
    w, U = np.linalg.eigh(M)
    return w[:nroots], fix_phase(U[:, :nroots].T)


def eig_partitioned(M11, M21, d22, nroots, tol=1e-13):
    """Lowest roots below the lowest M22 pole from the exact partitioning
    M_eff(w) = M11 + M12 (w - M22)^-1 M21 (valid because M22 is diagonal):
    w is an eigenvalue of M iff it is an eigenvalue of M_eff(w).  Each root
    solves lambda_k(M_eff(w)) = w by safeguarded Newton/bisection; the
    function is strictly decreasing in w below the pole."""
    M12 = M21.conj().T
    pole = d22.min()
    bound = np.linalg.norm(M12, 2)
    lo0 = min(np.linalg.eigvalsh(M11)[0], pole) - bound - 1.0

    def g(w, k):
        Meff = M11 + (M12 / (w - d22)) @ M21
        lam, U = np.linalg.eigh(Meff)
        u = U[:, k]
        z = M21 @ u
        dlam = -np.sum(np.abs(z) ** 2 / (w - d22) ** 2)
        return lam[k] - w, dlam - 1.0, lam, U

    roots, vecs = [], []
    for k in range(nroots):
        lo, hi = lo0, pole - 1e-9 * max(1.0, abs(pole))
        fhi = g(hi, k)[0]
        if fhi > 0:
            raise RuntimeError("root %d lies above the lowest M22 pole" % k)
        w = 0.5 * (lo + hi) if not roots else roots[-1]
        for _ in range(200):
            f, fp, lam, U = g(w, k)
            if f > 0:
                lo = w
            else:
                hi = w
            wn = w - f / fp
            if not (lo < wn < hi):
                wn = 0.5 * (lo + hi)
            if abs(wn - w) <= tol * max(1.0, abs(w)):
                w = wn
                break
            w = wn
        f, fp, lam, U = g(w, k)
        u = U[:, k]
        v2 = (M21 @ u) / (w - d22)
        x = np.concatenate([u, v2])
        x /= np.linalg.norm(x)
        roots.append(w)
        vecs.append(x)
    return np.array(roots), fix_phase(np.array(vecs))


def eig_lanczos(M11, M21, d22, nroots, tol=1e-12):
    """Implicitly restarted Lanczos (ARPACK) on the explicit blocks."""
    N1, N2 = M11.shape[0], d22.size
    M12 = M21.conj().T

    def mv(x):
        x = np.asarray(x).reshape(-1)
        return np.concatenate([M11 @ x[:N1] + M12 @ x[N1:],
                               M21 @ x[:N1] + d22 * x[N1:]])

    op = scipy.sparse.linalg.LinearOperator((N1 + N2, N1 + N2), matvec=mv,
                                            dtype=np.complex128)
    w, U = scipy.sparse.linalg.eigsh(op, k=nroots, which="SA", tol=tol,
                                     ncv=max(4 * nroots, 40), maxiter=100000)
    order = np.argsort(w)
    return w[order], fix_phase(U[:, order].T)
