"""Pins of the CPU oracle against things other than itself.

Each test fixes the oracle to an independent source: the determinant-space
Hamiltonian built from second-quantised operators, the brute-force ISR of
section "Relativistic Algebraic Diagrammatic Construction Method",
Rayleigh-Schrodinger perturbation theory, closed forms, and exact
symmetries.  A dropped term, a wrong sign, a transposed operand or a wrong
index anywhere in ``oracle.mp2`` / ``oracle.adc2`` / ``oracle.fns`` fails at
least one of them.
"""

import itertools

import numpy as np
import pytest

from oracle import adc2, cisd, fns, mp2, rootsel, spectrum
from oracle.fci import DetSpace, ISR, apply_string, full_antisym_integrals
from oracle.integrals import antisym
from synth import make_instance, make_kramers_instance, make_spinfree_instance


TINY = [dict(ncore=2, nval=2, nvirt=4, naux=6, seed=3, scale=0.15),
        dict(ncore=2, nval=2, nvirt=5, naux=7, seed=11, scale=0.2)]


@pytest.fixture(scope="module", params=range(len(TINY)))
def tiny(request):
    cfg = dict(TINY[request.param])
    inst = make_instance(cfg["ncore"], cfg["nval"], cfg["nvirt"], cfg["naux"],
                         seed=cfg["seed"], scale=cfg["scale"])
    isr = ISR(inst.eps, inst.B, inst.ncore, inst.nval, inst.nvirt, dip=inst.dip)
    cM, cF, cE = isr.taylor()
    return inst, isr, cM, cF, cE


# ---------------------------------------------------------------- T0 inputs

def test_generator_deterministic_and_hermitian():
    a = make_instance(3, 4, 6, 10, seed=5)
    b = make_instance(3, 4, 6, 10, seed=5)
    assert a.eps.tobytes() == b.eps.tobytes()
    assert a.B.tobytes() == b.B.tobytes()
    assert np.array_equal(a.B, np.conj(a.B.transpose(0, 2, 1)))
    assert np.array_equal(a.dip, np.conj(a.dip.transpose(0, 2, 1)))
    c = make_instance(3, 4, 6, 10, seed=6)
    assert a.B.tobytes() != c.B.tobytes()
    # Kramers-paired valence energies
    assert np.all(a.eps[3:7:2] == a.eps[4:7:2])


# ---------------------------------------------------- T1 determinant engine

def test_fermion_anticommutators():
    sp = DetSpace(5, 2)
    # {a_p, a_q^+} = delta_pq on every 2-electron determinant, checked by
    # applying a_p a_q^+ + a_q^+ a_p
    for d in sp.dets:
        for p in range(5):
            for q in range(5):
                acc = {}
                for ops in ([(0, p), (1, q)], [(1, q), (0, p)]):
                    r = apply_string(ops, d)
                    if r is not None:
                        acc[r[1]] = acc.get(r[1], 0) + r[0]
                acc = {k: v for k, v in acc.items() if v != 0}
                assert acc == ({d: 1} if p == q else {})


def test_slater_condon_reference_elements():
    inst = make_instance(2, 2, 3, 5, seed=2, scale=0.3)
    isr = ISR(inst.eps, inst.B, 2, 2, 3)
    sp, H = isr.space, isr.H
    g = full_antisym_integrals(inst.B)
    o = 4
    ref = sp.index[sp.ref]
    # E_HF = sum_i e_i - 1/2 sum_ij <ij||ij> for h = diag(e) - sum_k <pk||qk>
    ehf = inst.eps[:o].sum() - 0.5 * sum(g[i, j, i, j] for i in range(o) for j in range(o))
    assert abs(H[ref, ref] - ehf) < 1e-12
    assert np.abs(H - H.conj().T).max() < 1e-13
    for i in range(o):
        for a in range(o, 7):
            s, d = apply_string([(1, a), (0, i)], sp.ref)
            # Brillouin: <Phi_i^a|H|Phi_0> = f_ai = 0
            assert abs(H[sp.index[d], ref]) < 1e-13
    for i, j in itertools.combinations(range(o), 2):
        for a, b in itertools.combinations(range(o, 7), 2):
            s, d = apply_string([(1, a), (1, b), (0, j), (0, i)], sp.ref)
            assert abs(s * H[sp.index[d], ref] - g[a, b, i, j]) < 1e-13


# ------------------------------------------------------------------ T2 MP2

def test_mp2_energy_equals_rspt_and_fci_taylor(tiny):
    inst, isr, cM, cF, cE = tiny
    e2 = mp2.mp2_energy(inst.eps, inst.B, inst.ncore, inst.nval, inst.nvirt)
    assert abs(e2.imag) < 1e-14
    assert abs(e2.real - isr.rspt_e2()) < 1e-12 * abs(e2)
    # second Taylor coefficient of the exact ground-state energy
    assert abs(cE[2] - e2.real) < 1e-7 * abs(e2)
    # zeroth + first order reproduce E_HF
    assert abs(cE[0] + cE[1] - isr.e_hf) < 1e-9


def test_mp2_cholesky_equals_full_integrals():
    inst = make_instance(3, 4, 7, 12, seed=8)
    nc, nw, nv = 3, 4, 7
    o = nc + nw
    g = full_antisym_integrals(inst.B)
    e = inst.eps
    full = 0.0
    for i in range(o):
        for j in range(o):
            for a in range(o, o + nv):
                for b in range(o, o + nv):
                    full += 0.25 * abs(g[i, j, a, b]) ** 2 / (e[i] + e[j] - e[a] - e[b])
    e2 = mp2.mp2_energy(e, inst.B, nc, nw, nv)
    assert abs(e2 - full) < 1e-13 * abs(full)


def test_t2_antisymmetry_and_density():
    inst = make_instance(2, 4, 6, 9, seed=4)
    t = mp2.t2_amplitudes(inst.eps, inst.B, 2, 4, 6)
    tol = 1e-15 * np.abs(t).max()
    assert np.abs(t + t.transpose(1, 0, 2, 3)).max() <= tol
    assert np.abs(t + t.transpose(0, 1, 3, 2)).max() <= tol
    D = mp2.density_vv(inst.eps, inst.B, 2, 4, 6)
    assert np.abs(D - D.conj().T).max() < 1e-14 * np.abs(D).max()
    w = np.linalg.eigvalsh(D)
    assert w.min() > -1e-14 * w.max()
    assert abs(np.trace(D) - 0.5 * np.sum(np.abs(t) ** 2)) < 1e-13 * abs(np.trace(D))


def test_density_orientation_from_exact_ground_state(tiny):
    """Eq. 15's D_ab is the lambda^2 coefficient of the exact ground state's
    <a_b^+ a_a> (the density whose eigenvectors, as columns, are the natural
    spinors of Eqs. 17-20).  Trace, Hermiticity and positivity hold for D and
    D^T alike; this fixes which one the oracle builds: the lambda^2
    coefficient of <a_a^+ a_b> must equal D^T, and must differ from D."""
    inst, isr, cM, cF, cE = tiny
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    o = nc + nw
    D = mp2.density_vv(inst.eps, inst.B, nc, nw, nv)
    g = isr.ground_rdm1_taylor()
    gvv = g[2][o:, o:]  # lambda^2 coefficient of <a_a^+ a_b>, a, b virtual
    scale = np.abs(D).max()
    assert np.abs(g[1][o:, o:]).max() < 1e-9 * scale  # no first-order vv density
    assert np.abs(gvv - D.T).max() < 1e-7 * scale
    # negative control: the other orientation is measurably different
    assert np.abs(gvv - D).max() > 1e-3 * scale


# ------------------------------------------------------- T3 ISR brute force

def _blocks(inst):
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    return (adc2.m11(inst.eps, inst.B, nc, nw, nv),
            adc2.m11(inst.eps, inst.B, nc, nw, nv, second_order=False),
            adc2.m21(inst.eps, inst.B, nc, nw, nv),
            adc2.m22(inst.eps, nc, nw, nv))


def test_isr_pins_m11_through_second_order(tiny):
    inst, isr, cM, cF, cE = tiny
    M11, M11_01, M21, d22 = _blocks(inst)
    N1 = M11.shape[0]
    ref2 = cM[0][:N1, :N1] + cM[1][:N1, :N1] + cM[2][:N1, :N1]
    ref1 = cM[0][:N1, :N1] + cM[1][:N1, :N1]
    scale = np.abs(ref2).max()
    assert np.abs(M11_01 - ref1).max() < 1e-10 * scale
    second = M11 - M11_01
    assert np.abs(second).max() > 1e-3 * scale  # the second order term matters
    assert np.abs(M11 - ref2).max() < 1e-7 * scale


def test_isr_pins_coupling_and_doubles(tiny):
    inst, isr, cM, cF, cE = tiny
    M11, M11_01, M21, d22 = _blocks(inst)
    N1 = M11.shape[0]
    assert np.abs(cM[0][N1:, :N1]).max() < 1e-12
    assert np.abs(M21 - cM[1][N1:, :N1]).max() < 1e-9 * np.abs(M21).max()
    assert np.abs(cM[0][N1:, N1:] - np.diag(d22)).max() < 1e-10 * np.abs(d22).max()


def test_isr_pins_transition_moments(tiny):
    inst, isr, cM, cF, cE = tiny
    F = adc2.transition_moments(inst.eps, inst.B, inst.dip, inst.ncore,
                                inst.nval, inst.nvirt)
    ref = cF[0] + cF[1]
    assert np.abs(F - ref).max() < 1e-9 * np.abs(ref).max()
    # the first-order part is non-trivial
    assert np.abs(cF[1]).max() > 1e-3 * np.abs(cF[0]).max()


def test_isr_pins_second_order_amplitudes(tiny):
    """The lambda^1 and lambda^2 amplitudes of the exact ground state on
    singles and doubles determinants are t2 and the second-order s and u
    (Rayleigh-Schrodinger with the MP partitioning)."""
    inst, isr, cM, cF, cE = tiny
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    o = nc + nw
    c = isr.ground_state_taylor()
    t2 = mp2.t2_amplitudes(inst.eps, inst.B, nc, nw, nv)
    s = mp2.second_order_singles(inst.eps, inst.B, nc, nw, nv, t2=t2)
    u = mp2.second_order_doubles(inst.eps, inst.B, nc, nw, nv, t2=t2)
    s_ex = np.array([[isr.amplitude(c[2], [o + a], [k]) for a in range(nv)] for k in range(o)])
    assert np.abs(s - s_ex).max() < 1e-8 * np.abs(s_ex).max()
    assert np.abs(s_ex).max() > 1e-4
    err_u, err_t, mx = 0.0, 0.0, 0.0
    for k, l in itertools.combinations(range(o), 2):
        for a, b in itertools.combinations(range(nv), 2):
            ex2 = isr.amplitude(c[2], [o + a, o + b], [k, l])
            ex1 = isr.amplitude(c[1], [o + a, o + b], [k, l])
            err_u = max(err_u, abs(u[k, l, a, b] - ex2))
            err_t = max(err_t, abs(t2[k, l, a, b] - ex1))
            mx = max(mx, abs(ex2))
    assert err_t < 1e-10
    assert err_u < 1e-8 * mx and mx > 1e-4
    # the core rows alone, as the moments use them
    uc = mp2.second_order_doubles(inst.eps, inst.B, nc, nw, nv, t2=t2, rows=slice(0, nc))
    assert np.abs(uc - u[:nc]).max() < 1e-14


def test_isr_pins_second_order_singles_moments(tiny):
    """F^(2)_S = the lambda^2 coefficient of the brute-force ISR's singles
    moments (section "Properties in ISR formulation"), every term of it
    carrying weight."""
    inst, isr, cM, cF, cE = tiny
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    N1 = nc * nv
    f2 = adc2.singles_moments_second_order(inst.eps, inst.B, inst.dip, nc, nw, nv)
    ref = cF[2][:, :N1].reshape(f2.shape)
    scale = np.abs(ref).max()
    assert np.abs(f2 - ref).max() < 1e-8 * scale
    F = adc2.transition_moments(inst.eps, inst.B, inst.dip, nc, nw, nv, order=2)
    assert np.abs(F - (cF[0] + cF[1] + np.concatenate(
        [cF[2][:, :N1], np.zeros_like(cF[2][:, N1:])], axis=1))).max() < 1e-8 * scale
    # each of the six terms alone moves the result far beyond the tolerance
    C, O, V = np.arange(nc), np.arange(nc + nw), np.arange(nc + nw, nc + nw + nv)
    t2 = mp2.t2_amplitudes(inst.eps, inst.B, nc, nw, nv)
    s = mp2.second_order_singles(inst.eps, inst.B, nc, nw, nv, t2=t2)
    u = mp2.second_order_doubles(inst.eps, inst.B, nc, nw, nv, t2=t2, rows=C)
    d = inst.dip[0]
    dvv, doo, dov, dvo = d[np.ix_(V, V)], d[np.ix_(O, O)], d[np.ix_(O, V)], d[np.ix_(V, O)]
    H = np.einsum("klde,Ilde->kI", np.conj(t2), t2[C])
    P = np.einsum("lmcd,lmad->ca", np.conj(t2), t2)
    w = np.einsum("ck,klcd->ld", dvo, np.conj(t2))
    terms = [np.einsum("ac,Ic->Ia", dvv, s[C]), np.einsum("kI,ka->Ia", doo[:, C], s),
             np.einsum("kc,Ikac->Ia", dov, u), np.einsum("ak,kI->Ia", dvo, H),
             np.einsum("ld,Ilad->Ia", w, t2[C]), np.einsum("cI,ca->Ia", dvo[:, C], P)]
    for term in terms:
        assert np.abs(term).max() > 1e-4 * scale


# --------------------------------------------- CIS(D) and Eqs. 21-22 (N1)

CISD = dict(ncore=2, nval=3, nvirt=8, naux=14, seed=5, scale=0.1)


def _cisd_instance():
    c = CISD
    return make_instance(c["ncore"], c["nval"], c["nvirt"], c["naux"], seed=c["seed"],
                         scale=c["scale"])


def test_cisd_is_the_second_order_estimate_of_adc2():
    """omega_CIS(D) - omega_CIS is the lambda^2 coefficient of the lowest
    eigenvalues of [[M_CIS + lambda^2 M11^(2), lambda M12], [lambda M21,
    M22]] (exact eigenvalues of the scaled matrix, Chebyshev fit); the
    explicit u^{ab}_{Ij} gives the same doubles term as the folded form."""
    inst = _cisd_instance()
    nc, nw, nv = CISD["ncore"], CISD["nval"], CISD["nvirt"]
    k = 3
    w, wd, b = cisd.cisd_energies(inst.eps, inst.B, nc, nw, nv, k)
    A = cisd.cis_block(inst.eps, inst.B, nc, nw, nv)
    M2 = adc2.m11(inst.eps, inst.B, nc, nw, nv) - A
    M21 = adc2.m21(inst.eps, inst.B, nc, nw, nv)
    d22 = adc2.m22(inst.eps, nc, nw, nv)
    h, npts = 0.05, 17
    lams = h * np.cos((2 * np.arange(npts) + 1) * np.pi / (2 * npts))
    vals = []
    for lam in lams:
        M = np.block([[A + lam ** 2 * M2, lam * M21.conj().T],
                      [lam * M21, np.diag(d22).astype(complex)]])
        vals.append(np.linalg.eigvalsh(M)[:k])
    Vm = np.vander(lams / h, 9, increasing=True)
    c = (np.linalg.pinv(Vm) @ np.array(vals)) * (h ** -np.arange(9))[:, None]
    assert np.abs(c[0] - w).max() < 1e-10
    assert np.abs(c[2] - (wd - w)).max() < 1e-7 * np.abs(wd - w).max()
    assert np.abs(wd - w).min() > 1e-2
    M11b = np.einsum("ki,ij,kj->k", np.conj(b), M2, b).real
    for q in range(k):
        eu = cisd.doubles_term_explicit(inst.eps, inst.B, nc, nw, nv, w[q], b[q])
        assert abs(eu - (wd[q] - w[q] - M11b[q])) < 1e-12 * abs(eu)


def test_fns_correction_eqs_21_22():
    """Keeping every virtual leaves dE = 0; with two of eight natural
    virtuals dropped, the corrected roots (Eq. 22) are closer to the
    canonical CVS-ADC(2) roots than the uncorrected ones."""
    inst = _cisd_instance()
    nc, nw, nv = CISD["ncore"], CISD["nval"], CISD["nvirt"]
    k = 3
    dE, w_fns, w_corr = cisd.fns_correction(inst.eps, inst.B, nc, nw, nv, k, 1e-30)
    assert np.abs(dE).max() < 1e-12
    n, _, _ = fns.natural_spinors(inst.eps, inst.B, nc, nw, nv, 0.0)
    tau = 0.5 * (n[5] + n[6])
    dE, w_fns, w_corr = cisd.fns_correction(inst.eps, inst.B, nc, nw, nv, k, tau)
    w_can = np.linalg.eigvalsh(adc2.adc_matrix(inst.eps, inst.B, nc, nw, nv))[:k]
    assert np.all(np.abs(w_corr - w_can) < np.abs(w_fns - w_can))
    assert np.abs(w_fns - w_can).min() > 1e-2


def test_cis_guesses_map_into_the_fns_basis():
    """With every virtual kept U is unitary, so the canonical CIS
    eigenvectors mapped by U^H are CIS eigenvectors of the rotated problem
    with the same energies (the orientation U instead of U^H fails)."""
    inst = _cisd_instance()
    nc, nw, nv = CISD["ncore"], CISD["nval"], CISD["nvirt"]
    _, U, et = fns.natural_spinors(inst.eps, inst.B, nc, nw, nv, 0.0)
    e2, B2 = fns.rotate(inst.eps, inst.B, nc, nw, nv, U, et)
    w, _, _ = cisd.cisd_energies(inst.eps, inst.B, nc, nw, nv, 3)
    g = rootsel.cis_guesses_in_fns(inst.eps, inst.B, nc, nw, nv, 3, U)
    A2 = cisd.cis_block(e2, B2, nc, nw, nv)
    for k in range(3):
        assert np.linalg.norm(A2 @ g[k] - w[k] * g[k]) < 1e-12
        assert abs(np.linalg.norm(g[k]) - 1.0) < 1e-12


def test_root_following_selects_by_overlap():
    """Guesses equal to the singles parts of chosen eigenvectors select
    exactly those eigenpairs, in the guesses' order; following the CIS
    states in the keep-all FNS basis gives the roots that following them in
    the canonical basis gives."""
    inst = _cisd_instance()
    nc, nw, nv = CISD["ncore"], CISD["nval"], CISD["nvirt"]
    N1 = nc * nv
    M = adc2.adc_matrix(inst.eps, inst.B, nc, nw, nv)
    w, V = np.linalg.eigh(M)
    pick = [5, 1, 3]
    g = V[:N1, pick].T
    g = g / np.linalg.norm(g, axis=1)[:, None]
    wf, X = rootsel.follow_roots(M, N1, g)
    assert np.abs(wf - w[pick]).max() < 1e-12
    for k, j in enumerate(pick):
        assert abs(abs(np.vdot(X[k], V[:, j])) - 1.0) < 1e-10
    _, _, b = cisd.cisd_energies(inst.eps, inst.B, nc, nw, nv, 3)
    w_can, _ = rootsel.follow_roots(M, N1, b)
    w_fns, _, _ = rootsel.root_specific_fns(inst.eps, inst.B, nc, nw, nv, 3, 0.0)
    assert np.abs(w_fns - w_can).max() < 1e-10


# ------------------------------------------------ T4 Hermiticity and sigma

def test_hermitian_and_sigma_equals_dense():
    inst = make_instance(3, 4, 7, 12, seed=21)
    nc, nw, nv = 3, 4, 7
    M = adc2.adc_matrix(inst.eps, inst.B, nc, nw, nv)
    assert np.abs(M - M.conj().T).max() < 1e-13 * np.abs(M).max()
    sig = adc2.Sigma(inst.eps, inst.B, nc, nw, nv)
    rng = np.random.default_rng(0)
    N1, _, N2 = adc2.sizes(nc, nw, nv)
    x = rng.standard_normal(N1 + N2) + 1j * rng.standard_normal(N1 + N2)
    s1, s2 = sig(x[:N1], x[N1:])
    ref = M @ x
    assert np.abs(np.concatenate([s1, s2]) - ref).max() < 1e-12 * np.abs(ref).max()


# ------------------------------------------------------------ T5 CIS limit

def test_cis_limit_from_determinants():
    inst = make_instance(2, 3, 5, 8, seed=9, scale=0.4)
    nc, nw, nv = 2, 3, 5
    isr = ISR(inst.eps, inst.B, nc, nw, nv)
    sp, H = isr.space, isr.H
    ref = sp.index[sp.ref]
    o = nc + nw
    rows = []
    for I in range(nc):
        for a in range(nv):
            s, d = apply_string([(1, o + a), (0, I)], sp.ref)
            rows.append((sp.index[d], s))
    idx = np.array([r[0] for r in rows])
    sg = np.array([r[1] for r in rows], dtype=float)
    cis = (sg[:, None] * sg[None, :]) * H[np.ix_(idx, idx)] - H[ref, ref] * np.eye(len(rows))
    M = adc2.adc_matrix(inst.eps, inst.B, nc, nw, nv, second_order=False)
    w_adc = np.linalg.eigvalsh(M)[: nc * nv]
    # with the second order switched off the core-singles block decouples;
    # its eigenvalues are those of the CIS matrix over core singles
    M11 = adc2.m11(inst.eps, inst.B, nc, nw, nv, second_order=False)
    assert np.abs(M11 - cis).max() < 1e-12 * np.abs(cis).max()
    w_cis = np.linalg.eigvalsh(cis)
    assert np.allclose(np.sort(np.linalg.eigvalsh(M11)), w_cis, atol=1e-11)
    assert w_adc.min() <= w_cis.min() + 1e-9  # doubles only add states


# ---------------------------------------------------- T6 symmetry pins

def _tr_map(nc, nw, nv):
    """Time reversal on the packed CVS basis: basis vector P maps to
    eta_P * basis vector tau(P)."""
    o = nc + nw
    s = lambda p: 1 if p % 2 == 0 else -1  # noqa: E731
    perm, eta = [], []
    for I in range(nc):
        for a in range(nv):
            perm.append((I ^ 1) * nv + (a ^ 1))
            eta.append(s(I) * s(o + a))
    npair = nv * (nv - 1) // 2
    pos = {tuple(p): k for k, p in enumerate(adc2.pair_list(nv).tolist())}
    N1 = nc * nv
    for I in range(nc):
        for j in range(nw):
            for a, b in itertools.combinations(range(nv), 2):
                ta, tb = a ^ 1, b ^ 1
                sg = s(I) * s(nc + j) * s(o + a) * s(o + b)
                if ta > tb:
                    ta, tb = tb, ta
                    sg = -sg
                perm.append(N1 + ((I ^ 1) * nw + ((nc + j) ^ 1) - nc) * npair + pos[(ta, tb)])
                eta.append(sg)
    return np.array(perm), np.array(eta, dtype=float)


def test_time_reversal_covariance():
    inst = make_kramers_instance(2, 2, 6, 8, seed=13)
    nc, nw, nv = 2, 2, 6
    M = adc2.adc_matrix(inst.eps, inst.B, nc, nw, nv)
    perm, eta = _tr_map(nc, nw, nv)
    lhs = M[np.ix_(perm, perm)]
    rhs = eta[:, None] * eta[None, :] * np.conj(M)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(M).max()
    # the same map on a generic instance fails: the test has teeth
    gen = make_instance(2, 2, 6, 8, seed=13)
    Mg = adc2.adc_matrix(gen.eps, gen.B, nc, nw, nv)
    assert np.abs(Mg[np.ix_(perm, perm)] - eta[:, None] * eta[None, :] * np.conj(Mg)).max() > 1e-3


def test_spin_free_triplets_threefold():
    inst = make_spinfree_instance(2, 2, 6, 8, seed=17, scale=0.2)
    M = adc2.adc_matrix(inst.eps, inst.B, 2, 2, 6)
    w = np.linalg.eigvalsh(M)
    clusters, start = [], 0
    for k in range(1, len(w) + 1):
        if k == len(w) or w[k] - w[k - 1] > 1e-8:
            clusters.append(k - start)
            start = k
    # singlets, triplets and (two holes + two particles) quintets only
    assert set(clusters) <= {1, 3, 5}, clusters
    assert 3 in clusters and 1 in clusters
    # a generic (spin-orbit coupled) instance has no such multiplets
    gen = make_instance(2, 2, 6, 8, seed=17, scale=0.2)
    wg = np.linalg.eigvalsh(adc2.adc_matrix(gen.eps, gen.B, 2, 2, 6))
    assert np.min(np.diff(wg)) > 1e-7


# ------------------------------------------------------------------ T7 FNS

def test_fns_keep_all_is_exact_invariance():
    inst = make_instance(2, 3, 8, 10, seed=31)
    nc, nw, nv = 2, 3, 8
    n, U, et = fns.natural_spinors(inst.eps, inst.B, nc, nw, nv, tau=-1.0)
    assert U.shape == (nv, nv)
    assert np.abs(U.conj().T @ U - np.eye(nv)).max() < 1e-13
    D = mp2.density_vv(inst.eps, inst.B, nc, nw, nv)
    assert abs(n.sum() - np.trace(D).real) < 1e-14 * abs(n.sum())
    assert n.min() > -1e-15
    e2, B2 = fns.rotate(inst.eps, inst.B, nc, nw, nv, U, et)
    w0 = np.linalg.eigvalsh(adc2.adc_matrix(inst.eps, inst.B, nc, nw, nv))[:6]
    w1 = np.linalg.eigvalsh(adc2.adc_matrix(e2, B2, nc, nw, nv))[:6]
    assert np.abs(w0 - w1).max() < 1e-10
    # semicanonical: F stays diagonal, energies are the sorted originals
    assert np.allclose(np.sort(et), np.sort(inst.eps[nc + nw:]), atol=1e-13)


def test_fns_truncation_counts_and_rotation():
    inst = make_instance(2, 3, 10, 10, seed=32, scale=0.1)
    nc, nw, nv = 2, 3, 10
    D = mp2.density_vv(inst.eps, inst.B, nc, nw, nv)
    occ = np.sort(np.linalg.eigvalsh(D))[::-1]
    tau = 0.5 * (occ[4] + occ[5])
    n, U, et = fns.natural_spinors(inst.eps, inst.B, nc, nw, nv, tau)
    assert U.shape == (nv, 5)
    assert np.abs(U.conj().T @ U - np.eye(5)).max() < 1e-13
    e2, B2 = fns.rotate(inst.eps, inst.B, nc, nw, nv, U, et)
    o = nc + nw
    # rotated Fock block is diagonal with eps~
    F = U.conj().T @ np.diag(inst.eps[o:]) @ U
    assert np.abs(F - np.diag(et)).max() < 1e-13
    # rotated vectors are still Hermitian
    assert np.abs(B2 - np.conj(B2.transpose(0, 2, 1))).max() < 1e-14


# ------------------------------------------------------------ T8 solvers

def test_dense_partitioned_lanczos_agree():
    inst = make_instance(2, 4, 12, 16, seed=41)
    nc, nw, nv = 2, 4, 12
    M11 = adc2.m11(inst.eps, inst.B, nc, nw, nv)
    M21 = adc2.m21(inst.eps, inst.B, nc, nw, nv)
    d22 = adc2.m22(inst.eps, nc, nw, nv)
    M = np.block([[M11, M21.conj().T], [M21, np.diag(d22).astype(complex)]])
    wd, Xd = adc2.eig_dense(M, 4)
    wp, Xp = adc2.eig_partitioned(M11, M21, d22, 4)
    wl, Xl = adc2.eig_lanczos(M11, M21, d22, 4)
    assert np.abs(wd - wp).max() < 1e-10 * max(1, abs(wd).max())
    assert np.abs(wd - wl).max() < 1e-9 * max(1, abs(wd).max())
    for k in range(4):
        assert abs(abs(np.vdot(Xd[k], Xp[k])) - 1) < 1e-8
        assert np.linalg.norm(M @ Xp[k] - wp[k] * Xp[k]) < 1e-9 * abs(wp[k])


# ------------------------------------------------------------ T9 packing

def test_packing_bit_exact():
    for nc, nw, nv in [(2, 3, 5), (6, 14, 40), (1, 1, 2)]:
        tab = adc2.doubles_list(nc, nw, nv)
        N1, npair, N2 = adc2.sizes(nc, nw, nv)
        assert tab.shape == (N2, 4)
        I, j, a, b = tab.T
        pair = a * (2 * nv - a - 1) // 2 + (b - a - 1)
        d = (I * nw + j) * npair + pair
        assert np.array_equal(d, np.arange(N2, dtype=np.int64))
        rng = np.random.default_rng(1)
        x = rng.standard_normal(N2) + 1j * rng.standard_normal(N2)
        assert np.array_equal(adc2.pack(adc2.unpack(x, nc, nw, nv), nv), x)


# ------------------------------------------------ transition moment algebra

def test_oscillator_linearity_and_phase():
    inst = make_instance(2, 2, 6, 8, seed=5)
    nc, nw, nv = 2, 2, 6
    M = adc2.adc_matrix(inst.eps, inst.B, nc, nw, nv)
    w, X = adc2.eig_dense(M, 3)
    F = adc2.transition_moments(inst.eps, inst.B, inst.dip, nc, nw, nv)
    f = adc2.oscillator_strengths(w, X, F)
    F2 = adc2.transition_moments(inst.eps, inst.B, 2.5 * inst.dip, nc, nw, nv)
    assert np.allclose(adc2.oscillator_strengths(w, X, F2), 6.25 * f, rtol=1e-13)
    ph = np.exp(1j * np.array([0.3, -1.2, 2.0]))[:, None]
    assert np.allclose(adc2.oscillator_strengths(w, X * ph, F), f, rtol=1e-13)


# ------------------------------------------------- T10 reference gradient

@pytest.mark.parametrize("shape,nroots", [((2, 2, 5, 6), 3), ((2, 4, 6, 9), 4)])
def test_reference_gradient_matches_finite_differences(shape, nroots):
    from oracle.grad import energy_gradient

    nc, nw, nv, L = shape
    inst = make_instance(nc, nw, nv, L, seed=7, scale=0.2)
    w, ge, gB = energy_gradient(inst.eps, inst.B, nc, nw, nv, nroots)
    rng = np.random.default_rng(1)

    def E(eps, B):
        return np.linalg.eigvalsh(adc2.adc_matrix(eps, B, nc, nw, nv))[:nroots].sum()

    assert abs(E(inst.eps, inst.B) - w.sum()) < 1e-11
    h = 1e-5
    for _ in range(2):
        d = rng.standard_normal(inst.B.shape) + 1j * rng.standard_normal(inst.B.shape)
        d = 0.5 * (d + np.conj(d.transpose(0, 2, 1)))
        fd = (E(inst.eps, inst.B + h * d) - E(inst.eps, inst.B - h * d)) / (2 * h)
        ad = np.real(np.sum(np.conj(gB) * d))
        assert abs(fd - ad) < 1e-7 * max(1.0, abs(ad)), (fd, ad)
        de = rng.standard_normal(inst.eps.shape)
        fd = (E(inst.eps + h * de, inst.B) - E(inst.eps - h * de, inst.B)) / (2 * h)
        assert abs(fd - np.sum(ge * de)) < 1e-7 * max(1.0, abs(fd))
    # the projected gradient is Hermitian
    assert np.abs(gB - np.conj(gB.transpose(0, 2, 1))).max() < 1e-14


# ------------------------------------- folded doubles (Schur complement)

def test_self_energy_splits_into_five_structured_terms():
    """M12 (theta - M22)^-1 M21 from the oracle's explicit blocks equals the
    five pieces the GPU preconditioner builds: a weighted Gram of <ab||cj>
    per core index, a <ab||cj>-<Kb||Ij> cross term and its adjoint, and two
    <Kb||Ij> terms (sums over all a, b with w = 1/(theta - M22))."""
    from oracle.integrals import antisym

    nc, nw, nv, L = 3, 4, 7, 20
    inst = make_instance(nc, nw, nv, L, seed=1)
    eps, B = inst.eps, inst.B
    o = nc + nw
    C, W, V = np.arange(nc), np.arange(nc, o), np.arange(o, o + nv)
    M21 = adc2.m21(eps, B, nc, nw, nv)
    D = adc2.m22(eps, nc, nw, nv).reshape(-1)
    th = D.min() - 3.0
    explicit = (M21.conj().T / (th - D)) @ M21
    g = antisym(B, V, V, V, W)  # <ab||cj>
    h = antisym(B, C, V, C, W)  # <Kb||Ij>
    ec, ew, ev = eps[C], eps[W], eps[V]
    w = 1.0 / (th - (ev[None, None, :, None] + ev[None, None, None, :]
                     - ec[:, None, None, None] - ew[None, :, None, None]))
    S = np.zeros((nc, nv, nc, nv), complex)
    for K in range(nc):
        S[K, :, K, :] += 0.5 * np.einsum("jab,abcj,abdj->cd", w[K], g.conj(), g)
    X = -np.einsum("Kjdb,dbcj,EbKj->KcEd", w, g.conj(), h)
    S += X + np.conj(np.transpose(X, (2, 3, 0, 1)))
    S22 = np.einsum("Ijcb,KbIj,EbIj->KcE", w, h.conj(), h)
    for c in range(nv):
        S[:, c, :, c] += S22[:, c, :]
    S -= np.einsum("Ijcd,KdIj,EcIj->KcEd", w, h.conj(), h)
    S = S.reshape(nc * nv, nc * nv)
    assert np.abs(S - explicit).max() < 1e-13 * np.abs(explicit).max()


# ---------------------------------------------------- N4 broadened spectrum

def test_lorentzian_spectrum_closed_forms():
    rng = np.random.default_rng(8)
    om = rng.uniform(15.0, 16.0, 5)
    f = rng.uniform(0.1, 2.0, 5)
    g, shift = 0.3, -4.1
    a, b = 380.0, 460.0
    grid = np.linspace(a, b, 400001)
    I = spectrum.lorentzian_spectrum(om, f, grid, g, shift)
    # integral over [a, b]: closed form of the arctangent
    E = om * spectrum.EV_PER_EH + shift
    h = g / 2
    exact = np.sum(f * (np.arctan((b - E) / h) - np.arctan((a - E) / h))) / np.pi
    trap = np.sum(0.5 * (I[1:] + I[:-1]) * np.diff(grid))
    assert abs(trap - exact) < 1e-8 * exact
    # one line: peak 2 f / (pi g) at E, half of it at E +- g/2
    one = spectrum.lorentzian_spectrum([om[0]], [f[0]], [E[0], E[0] - h, E[0] + h], g, shift)
    assert abs(one[0] - 2 * f[0] / (np.pi * g)) < 1e-12 * one[0]
    assert np.abs(one[1:] - 0.5 * one[0]).max() < 1e-12 * one[0]
    # linear in the strengths
    I2 = spectrum.lorentzian_spectrum(om, 3 * f, grid[::1000], g, shift)
    assert np.abs(I2 - 3 * I[::1000]).max() < 1e-12 * np.abs(I2).max()
