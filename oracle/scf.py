"""Restricted Hartree-Fock SCF on the oracle side (paper Sec. 3.2 and 3.2.1).

TEST INFRASTRUCTURE ONLY.  Follows the paper's cycle step by step:
  1. core-Hamiltonian guess: diagonalise H in the orthogonal basis   (Sec. 3.2)
  2. H = T + V, S
  3. symmetric orthogonalisation X = U s^{-1/2} U^T
  4. loop: G(D) -> F = H + G -> (DIIS) -> F' = X^T F X -> diagonalise ->
     C = X C' -> D = 2 C_occ C_occ^T -> energy + convergence test
DIIS (Sec. 3.2.1, Algorithm 1): error e_i = F_i D_i S - S D_i F_i; B_ij =
Tr(e_i^T e_j) bordered by -1 with a zero corner; right-hand side (0,...,0,-1);
F_DIIS = sum_i c_i F_i.
Readings where the paper is silent (also listed in the design notes):
  * E_elec = 1/2 Tr[D (H + F(D))] with the un-extrapolated F of the same D;
  * convergence needs |dE| < conv_dE AND rms(dD) < conv_dD;
  * DIIS extrapolates once two error matrices are stored, keeps the last 8;
  * aufbau: the nelec/2 lowest orbitals, ties to the lower index.
Eigenpairs come from the oracle's cyclic Jacobi routine.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from .oracle import jacobi_eigh


def orthogonaliser(S: np.ndarray) -> tuple:
    """X = U s^{-1/2} U^T and the smallest overlap eigenvalue."""
    s, U = jacobi_eigh(S)
    return (U * (1.0 / np.sqrt(s))) @ U.T, float(s[0])


def density_from_fock(F: np.ndarray, X: np.ndarray, nocc: int) -> tuple:
    """F' = X^T F X, diagonalise, C = X C', D = 2 C_occ C_occ^T."""
    Fp = X.T @ F @ X
    eps, Cp = jacobi_eigh(0.5 * (Fp + Fp.T))
    Cmo = X @ Cp
    Cocc = Cmo[:, :nocc]
    return 2.0 * Cocc @ Cocc.T, eps, Cmo


def core_guess_density(S, H, nocc):
    X, _ = orthogonaliser(S)
    D, _, _ = density_from_fock(H, X, nocc)
    return D


@dataclass
class SCFResult:
    e_total: float
    e_elec: float
    e_nuc: float
    iters: int
    converged: bool
    D: np.ndarray
    F: np.ndarray
    energies: list = field(default_factory=list)
    times: list = field(default_factory=list)
    min_s_eig: float = 0.0


def diis_extrapolate(Fs: list, es: list) -> np.ndarray:
    """Algorithm 1 (Sec. 3.2.1): bordered B system, F_DIIS = sum c_i F_i."""
    m = len(Fs)
    Bm = np.zeros((m + 1, m + 1))
    for i in range(m):
        for j in range(m):
            Bm[i, j] = float(np.sum(es[i] * es[j]))  # Re Tr(e_i^T e_j)
    Bm[:m, m] = -1.0
    Bm[m, :m] = -1.0
    Bm[m, m] = 0.0
    rhs = np.zeros(m + 1)
    rhs[m] = -1.0
    x = np.linalg.solve(Bm, rhs)
    return sum(x[i] * Fs[i] for i in range(m))


def rhf(S, H, jk, nelec: int, e_nuc: float, max_iter: int = 100, conv_dE: float = 1e-10,
        conv_dD: float = 1e-7, diis: bool = True, diis_size: int = 8, D0=None) -> SCFResult:
    """jk(D) -> (J, K).  Returns the converged (or last) state."""
    t0 = time.perf_counter()
    nocc = nelec // 2
    X, smin = orthogonaliser(S)
    D = density_from_fock(H, X, nocc)[0] if D0 is None else np.array(D0, dtype=np.float64)
    E_old = None
    Fs, es = [], []
    energies, times = [], []
    converged = False
    F = H
    it = 0
    E_elec = 0.0
    for it in range(1, max_iter + 1):
        J, K = jk(D)
        F = H + J - 0.5 * K
        E_elec = 0.5 * float(np.sum(D * (H + F)))
        energies.append(E_elec + e_nuc)
        times.append(time.perf_counter() - t0)
        F_use = F
        if diis:
            Fs.append(F)
            es.append(F @ D @ S - S @ D @ F)
            if len(Fs) > diis_size:
                Fs.pop(0)
                es.pop(0)
            if len(Fs) >= 2:
                F_use = diis_extrapolate(Fs, es)
        D_new = density_from_fock(F_use, X, nocc)[0]
        dD = float(np.sqrt(np.mean((D_new - D) ** 2)))
        if E_old is not None and abs(E_elec - E_old) < conv_dE and dD < conv_dD:
            converged = True
            break
        E_old = E_elec
        D = D_new
    return SCFResult(E_elec + e_nuc, E_elec, e_nuc, it, converged, D, F, energies, times, smin)
