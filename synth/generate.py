"""Seeded synthetic CVS-ADC(2) problem instances.

The paper's workloads are molecules (X2C spinor energies and Cholesky vectors
of SiCl4, Ar, MO4^n-, TiCl4, VOCl3 and a Ru complex; section "Implementation
and Computational Details" and section "Application to Medium-Sized
Complex").  None of them is available here, so seeded random inputs with the
same structure stand in for them:

* spinors are ordered [core | valence | virtual]; frozen core is already
  removed (the caller passes only correlated spinors);
* core spinor energies are metal 2p levels: 2 p1/2 at -29.5 Eh and 4 p3/2
  at -28.9 Eh per metal centre (a second centre at -27.5/-26.9 Eh), each
  with a U(-0.01, 0.01) jitter;
* valence energies come as Kramers pairs (each drawn value used twice),
  U(-1.4, -0.3);
* virtual energies are U(0.05, 2.5);
* every Cholesky vector B^P is Hermitian, B^P_pq = conj(B^P_qp), with
  N(0,1) + i N(0,1) off-diagonal entries and N(0,1) real diagonal entries,
  scaled by ``scale * exp(-P / decay)``, scale 0.3 as the named workloads
  state it.  That scale is far from perturbative (small workload: E_MP2 =
  -2e4 Eh, roots near 15 Eh with 1.7 % singles weight, far below the lowest
  M22 entry), and it gets worse with the size, because dense random
  couplings sum over all nval nvirt^2 doubles a singles state talks to.
  ``physical_scale(nval, nvirt)`` = 0.34 (max(nval, 1) nvirt^2)^(-1/4) keeps
  the coupling a singles state feels bounded, so that E_MP2 grows with the
  number of occupied spinors (extensive) and the core excitations look like
  the paper's: on the small workload the lowest roots lie 0.2 Eh below the
  bare core -> virtual gaps and 0.7 Eh below the lowest doubles, with
  singles weights of about 0.87 (a companion instance, not a named
  workload);
* the three dipole matrices use the same Hermitian construction with scale
  0.1.

Draw order for ``numpy.random.default_rng(seed)``: core jitter (ncore),
valence pair energies (nval/2), virtual energies (nvirt); then for
P = 0..naux-1 the strict upper triangle (row-major, interleaved re/im pairs)
followed by the real diagonal; then the three dipole matrices the same way.

Nothing here computes any part of the method.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# Named workload shapes: (ncore, nval, nvirt, naux, nroots)
WORKLOADS = {
    # small all-checkable case: the oracle solves it exactly
    "small": dict(ncore=6, nval=14, nvirt=40, naux=240, nroots=4),
    # medium FP64 case
    "medium": dict(ncore=6, nval=60, nvirt=300, naux=1500, nroots=8),
    # two metal L-edges, mixed precision
    "large": dict(ncore=12, nval=120, nvirt=600, naux=3000, nroots=16),
    # differentiation case
    "grad": dict(ncore=6, nval=40, nvirt=200, naux=1000, nroots=4),
}


@dataclasses.dataclass
class Instance:
    ncore: int
    nval: int
    nvirt: int
    naux: int
    eps: np.ndarray  # [n] float64
    B: np.ndarray  # [naux][n][n] complex128, each B[P] Hermitian
    dip: np.ndarray  # [3][n][n] complex128, each Hermitian
    seed: int

    @property
    def nocc(self) -> int:
        return self.ncore + self.nval

    @property
    def n(self) -> int:
        return self.ncore + self.nval + self.nvirt


def core_energies(ncore: int, rng: np.random.Generator) -> np.ndarray:
    """Metal 2p core levels with jitter; 6 spinors per metal centre."""
    centres = [(-29.5, -28.9), (-27.5, -26.9), (-25.5, -24.9), (-23.5, -22.9)]
    levels = []
    c = 0
    while len(levels) < ncore:
        p12, p32 = centres[c % len(centres)]
        levels.extend([p12] * 2 + [p32] * 4)
        c += 1
    levels = np.array(levels[:ncore], dtype=np.float64)
    jitter = rng.uniform(-0.01, 0.01, size=ncore)
    return levels + jitter


def _hermitian(rng: np.random.Generator, n: int, scale: float) -> np.ndarray:
    """One random Hermitian matrix: upper triangle first, then the diagonal."""
    iu = np.triu_indices(n, k=1)
    m = iu[0].size
    g = rng.standard_normal(2 * m)
    d = rng.standard_normal(n)
    out = np.zeros((n, n), dtype=np.complex128)
    out[iu] = (g[0::2] + 1j * g[1::2]) * scale
    out[(iu[1], iu[0])] = np.conj(out[iu])
    out[np.arange(n), np.arange(n)] = d * scale
    return out


def physical_scale(nval: int, nvirt: int) -> float:
    """The size-aware Cholesky-vector scale described above."""
    return 0.34 * (max(nval, 1) * nvirt * nvirt) ** -0.25


def make_instance(ncore: int, nval: int, nvirt: int, naux: int, seed: int = 0,
                  scale: float = 0.3, decay: float = 60.0,
                  dip_scale: float = 0.1) -> Instance:
    """Seeded synthetic instance with the structure described above."""
    if ncore < 1 or nval < 0 or nvirt < 2 or naux < 1:
        raise ValueError("bad partition sizes")
    rng = np.random.default_rng(seed)
    e_core = core_energies(ncore, rng)
    npair = (nval + 1) // 2
    pairs = rng.uniform(-1.4, -0.3, size=npair)
    e_val = np.repeat(pairs, 2)[:nval]
    e_vir = rng.uniform(0.05, 2.5, size=nvirt)
    eps = np.concatenate([e_core, e_val, e_vir]).astype(np.float64)
    n = eps.size
    B = np.empty((naux, n, n), dtype=np.complex128)
    for P in range(naux):
        B[P] = _hermitian(rng, n, scale * math.exp(-P / decay))
    dip = np.empty((3, n, n), dtype=np.complex128)
    for x in range(3):
        dip[x] = _hermitian(rng, n, dip_scale)
    return Instance(ncore, nval, nvirt, naux, eps, B, dip, seed)


def _paired_energies(rng, count, lo, hi):
    vals = rng.uniform(lo, hi, size=count // 2)
    return np.repeat(vals, 2)


def make_kramers_instance(ncore: int, nval: int, nvirt: int, naux: int,
                          seed: int = 0, scale: float = 0.3,
                          decay: float = 60.0) -> Instance:
    """Time-reversal-symmetric instance in a Kramers-paired spinor basis.

    Spinors come in pairs (2k, 2k+1) = (phi_k, theta phi_k) inside each
    partition, so every partition size must be even.  Each B^P has the
    quaternion structure [[A, C], [-conj(C), conj(A)]] (interleaved by pair)
    with A Hermitian and C antisymmetric; energies are pair-degenerate.
    """
    for s in (ncore, nval, nvirt):
        if s % 2:
            raise ValueError("Kramers instance needs even partition sizes")
    rng = np.random.default_rng(seed)
    eps = np.concatenate([
        _paired_energies(rng, ncore, -29.6, -28.8),
        _paired_energies(rng, nval, -1.4, -0.3),
        _paired_energies(rng, nvirt, 0.05, 2.5),
    ])
    n = eps.size
    m = n // 2
    B = np.zeros((naux, n, n), dtype=np.complex128)
    for P in range(naux):
        s = scale * math.exp(-P / decay)
        A = _hermitian(rng, m, s)
        C = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) * s
        C = C - C.T
        B[P, 0::2, 0::2] = A
        B[P, 0::2, 1::2] = C
        B[P, 1::2, 0::2] = -np.conj(C)
        B[P, 1::2, 1::2] = np.conj(A)
    dip = np.zeros((3, n, n), dtype=np.complex128)
    for x in range(3):
        A = _hermitian(rng, m, 0.1)
        C = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) * 0.1
        C = C - C.T
        dip[x, 0::2, 0::2] = A
        dip[x, 0::2, 1::2] = C
        dip[x, 1::2, 0::2] = -np.conj(C)
        dip[x, 1::2, 1::2] = np.conj(A)
    return Instance(ncore, nval, nvirt, naux, eps, B, dip, seed)


def make_spinfree_instance(ncore: int, nval: int, nvirt: int, naux: int,
                           seed: int = 0, scale: float = 0.3,
                           decay: float = 60.0) -> Instance:
    """Spin-free instance: spinors (2k, 2k+1) = (phi_k alpha, phi_k beta).

    Every B^P is block diagonal in spin with identical alpha-alpha and
    beta-beta blocks (a complex Hermitian spatial matrix) and energies are
    pair-degenerate, so the Hamiltonian commutes with S^2.
    """
    for s in (ncore, nval, nvirt):
        if s % 2:
            raise ValueError("spin-free instance needs even partition sizes")
    rng = np.random.default_rng(seed)
    eps = np.concatenate([
        _paired_energies(rng, ncore, -29.6, -28.8),
        _paired_energies(rng, nval, -1.4, -0.3),
        _paired_energies(rng, nvirt, 0.05, 2.5),
    ])
    n = eps.size
    m = n // 2
    B = np.zeros((naux, n, n), dtype=np.complex128)
    for P in range(naux):
        A = _hermitian(rng, m, scale * math.exp(-P / decay))
        B[P, 0::2, 0::2] = A
        B[P, 1::2, 1::2] = A
    dip = np.zeros((3, n, n), dtype=np.complex128)
    for x in range(3):
        A = _hermitian(rng, m, 0.1)
        dip[x, 0::2, 0::2] = A
        dip[x, 1::2, 1::2] = A
    return Instance(ncore, nval, nvirt, naux, eps, B, dip, seed)


def batched_shapes(count: int = 48, seed: int = 0):
    """Ragged batch of instance shapes: ncore 6, nval ~ U{20..80} (even),
    nvirt ~ U{100..400}, naux = 5 * nvirt.  Instance i uses seed 1000+i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nval = int(rng.integers(10, 41)) * 2
        nvirt = int(rng.integers(100, 401))
        out.append(dict(ncore=6, nval=nval, nvirt=nvirt, naux=5 * nvirt,
                        nroots=4, seed=1000 + i))
    return out
