"""Orbital optimisation from the engine's reduced density matrices.

With a finite bond dimension D the DMRG energy depends on the orbital basis.
The 1- and 2-particle reduced density matrices that tns_rdm returns (the
derivatives of the energy with respect to the integrals, by Hellmann-Feynman)
give the gradient of the energy with respect to an orbital rotation, which is
what an orbital optimisation around DMRG needs (the RDMs of the
differentiation form; the paper names DMRG-RAS-X, Sec. "Massively parallel
DMRG-RAS-X method", as the method this kind of post-processing feeds).

Conventions (those of include/tns.h): H = sum_ij h_ij E_ij + 1/2 sum_ijkl
(ij|kl) e_ijkl, gamma_ij = dE/dh_ij (symmetrised), Gamma = 2 dE/dv averaged
over the eight index permutations of (ij|kl).  An orbital rotation is
phi'_i = sum_p U_pi phi_p with U = expm(kappa), kappa antisymmetric:
    h'_ij = sum_pq U_pi U_qj h_pq,
    (ij|kl)' = sum_pqrs U_pi U_qj U_rk U_sl (pq|rs).
To first order in kappa, with the state's RDMs held fixed,
    dE = 2 sum_pi kappa_pi F_pi,  F_pi = sum_j h_pj gamma_ij + sum_jkl (pj|kl) Gamma_ijkl,
so dE/dkappa_pq (p < q, kappa_qp = -kappa_pq) = 2 (F_pq - F_qp).  The
orbit-averaged Gamma is exact here because the first-order change of (ij|kl)
keeps its eight-fold symmetry, and only orbit sums of dE/dv enter.

The driver alternates DMRG sweeps in the current orbitals with one orbital
step: a minimisation of the fixed-RDM energy functional
    E(kappa) = sum h'(kappa) gamma + 1/2 sum v'(kappa) Gamma
along the steepest-descent direction (a few halvings of a trust step), the
integrals rotated, the MPS kept as it is (it now represents a state in the
rotated orbitals) and swept again.  Host-side numpy: an N^5 transformation
per step, outside the H_eff*psi hot path, which stays in the library.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def rotate_integrals(h: np.ndarray, v: np.ndarray, U: np.ndarray):
    """h' = U^T h U and (ij|kl)' = sum U_pi U_qj U_rk U_sl (pq|rs)."""
    h2 = U.T @ h @ U
    v2 = np.einsum("pqrs,pi->iqrs", v, U, optimize=True)
    v2 = np.einsum("iqrs,qj->ijrs", v2, U, optimize=True)
    v2 = np.einsum("ijrs,rk->ijks", v2, U, optimize=True)
    v2 = np.einsum("ijks,sl->ijkl", v2, U, optimize=True)
    # restore the exact eight-fold symmetry lost to rounding
    v2 = (v2 + v2.transpose(1, 0, 2, 3)) / 2
    v2 = (v2 + v2.transpose(0, 1, 3, 2)) / 2
    v2 = (v2 + v2.transpose(2, 3, 0, 1)) / 2
    return (h2 + h2.T) / 2, v2


def generalized_fock(h: np.ndarray, v: np.ndarray, gamma: np.ndarray, Gamma: np.ndarray) -> np.ndarray:
    """F_pi = sum_j h_pj gamma_ij + sum_jkl (pj|kl) Gamma_ijkl."""
    return h @ gamma.T + np.einsum("pjkl,ijkl->pi", v, Gamma, optimize=True)


def orbital_gradient(h, v, gamma, Gamma) -> np.ndarray:
    """G with G_pq = dE/dkappa_pq = 2 (F_pq - F_qp) (antisymmetric)."""
    F = generalized_fock(h, v, gamma, Gamma)
    return 2.0 * (F - F.T)


def rdm_energy(h, v, gamma, Gamma, e_core: float = 0.0) -> float:
    """E = sum h gamma + 1/2 sum v Gamma (+ e_core)."""
    return float(np.sum(h * gamma) + 0.5 * np.sum(v * Gamma) + e_core)


def orbital_step(h, v, gamma, Gamma, max_step: float = 0.2, tries: int = 8):
    """One steepest-descent step on the fixed-RDM energy functional.

    Returns (U, h', v', predicted energy change).  The step kappa = -t G/|G|
    starts at t = max_step (radians) and is halved until the functional
    decreases."""
    G = orbital_gradient(h, v, gamma, Gamma)
    gn = float(np.linalg.norm(G))
    N = h.shape[0]
    if gn == 0.0:
        return np.eye(N), h, v, 0.0
    e0 = rdm_energy(h, v, gamma, Gamma)
    t = max_step
    for _ in range(tries):
        U = sla.expm(-t * G / gn)
        h2, v2 = rotate_integrals(h, v, U)
        de = rdm_energy(h2, v2, gamma, Gamma) - e0
        if de < 0.0:
            return U, h2, v2, de
        t *= 0.5
    return np.eye(N), h, v, 0.0


def ground_state_rdms(ctx, site: int, N: int, precision: int, tol: float = 1e-9):
    """RDMs of the lowest eigenstate of H_eff at step (site, site+1) of the
    context's current MPS (device Davidson, then tns_rdm)."""
    import torch
    ctx.build_env(site)
    L = ctx.psi_guess(site)
    x0 = torch.empty(L, dtype=torch.float64, pin_memory=True)
    ctx.psi_guess(site, x0.data_ptr())
    x = x0.to("cuda")
    e, _, _ = ctx.davidson_ptr(site, x.data_ptr(), tol=tol, max_iter=400, precision=precision)
    gamma, Gamma = ctx.rdm_ptr(site, x.data_ptr(), N)
    return e, gamma, Gamma


def optimise(ctx, h, v, N: int, D: int, macro: int = 4, sweeps: int = 2, precision: int = 0,
             e_core: float = 0.0, tol: float = 1e-9, max_step: float = 0.2, site: int = 1):
    """DMRG with orbital optimisation: `macro` rounds of (sweeps in the current
    orbitals, RDMs at step (site, site+1), one orbital step, integrals
    rotated).  A sweep ends right to left at step (1, 2), where sites 0 and
    3.. are left- and right-canonical: the default site=1 is a step at which
    H_eff is the projected Hamiltonian.  The context must hold an MPS for
    (h, v).  Returns (history, U_total, h, v) with history entries {energy,
    grad_norm, predicted}."""
    U_tot = np.eye(N)
    hist = []
    for _ in range(macro):
        ctx.sweep(sweeps, D, tol=tol, max_iter=200, precision=precision)
        e, gamma, Gamma = ground_state_rdms(ctx, site, N, precision, tol)
        G = orbital_gradient(h, v, gamma, Gamma)
        U, h2, v2, de = orbital_step(h, v, gamma, Gamma, max_step=max_step)
        hist.append({"energy": e, "grad_norm": float(np.linalg.norm(G)), "predicted": de})
        if de == 0.0:
            break
        h, v = h2, v2
        U_tot = U_tot @ U
        ctx.load_integrals(h, v, e_core)
    return hist, U_tot, h, v
