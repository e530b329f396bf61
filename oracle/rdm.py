"""O4: one- and two-particle reduced density matrices of a state on the Fock
space (test infrastructure; imported only by tests and the benchmark's
baseline leg).

For the spin-free Hamiltonian of Eq. (1), written as
    H = sum_ij h_ij sum_s a+_is a_js + 1/2 sum_ijkl (ij|kl) sum_st a+_is a+_kt a_lt a_js,
the energy of a normalised state Phi is
    E = sum_ij h_ij gamma_ij + 1/2 sum_ijkl (ij|kl) Gamma_ijkl
with gamma_ij = sum_s <a+_is a_js> and Gamma_ijkl = sum_st <a+_is a+_kt a_lt a_js>.
With the MPS isometries frozen, H_eff at a fixed two-site step is linear in
(h, v), so by Hellmann-Feynman dE/dh_ij = gamma_ij and dE/d(ij|kl) =
Gamma_ijkl / 2 (each stored entry treated as independent).

Everything here is a brute-force definition on the 4^N Fock space (N <= 8).
Parity pinned (tests/test_oracle_rdm.py): Wick's theorem on determinants,
trace and partial-trace identities, and the energy identity against the
Fock-space Hamiltonian of O2.
"""
from __future__ import annotations

import numpy as np

from .fock import cdag_ops, left_basis, right_basis, _offsets


def mps_state(bonds, sites, k: int, X: dict, n_elec: int, two_sz: int, N: int) -> np.ndarray:
    """Fock vector of the MPS with left-canonical sites 0..k-1, right-canonical
    sites k+2..N-1 and the two-site blocks X {(q_l, s1, s2, q_r): m x n}
    (q_r = particle content of the right block)."""
    Lb = left_basis(bonds, sites, k)
    Rb = right_basis(bonds, sites, k + 2, N)
    offl, _ = _offsets(bonds[k])
    offr, o = {}, 0
    for q, d in bonds[k + 2]:
        offr[(n_elec - q[0], two_sz - q[1])] = o
        o += d
    nl, nr = Lb.shape[0], Rb.shape[0]
    Phi = np.zeros((nl, 4, 4, nr))
    for (ql, s1, s2, qr), blk in X.items():
        a, c = offl[ql], offr[qr]
        m, n = blk.shape
        Phi[:, s1, s2, :] += Lb[:, a:a + m] @ blk @ Rb[:, c:c + n].T
    return Phi.ravel()


def rdm1(phi: np.ndarray, N: int) -> np.ndarray:
    """gamma_ij = sum_s <phi| a+_is a_js |phi> = sum_s <a_is phi, a_js phi>."""
    cd = cdag_ops(N)
    anni = [(cd[p].T @ phi) for p in range(2 * N)]
    g = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            g[i, j] = sum(anni[2 * i + s] @ anni[2 * j + s] for s in range(2))
    return g


def rdm2(phi: np.ndarray, N: int) -> np.ndarray:
    """Gamma_ijkl = sum_st <phi| a+_is a+_kt a_lt a_js |phi>
                  = sum_st < a_kt a_is phi , a_lt a_js phi >."""
    cd = cdag_ops(N)
    c = [x.T.tocsr() for x in cd]
    M = 2 * N
    # w[(p, q)] = a_q a_p phi for spin-orbitals p, q
    one = [c[p] @ phi for p in range(M)]
    w = np.zeros((M, M, phi.size))
    for p in range(M):
        for q in range(M):
            w[p, q] = c[q] @ one[p]
    G = np.zeros((N, N, N, N))
    for s in range(2):
        for t in range(2):
            # rows (i, k): a_kt a_is phi ; cols (j, l): a_lt a_js phi
            A = w[s::2, t::2].reshape(N * N, -1)   # index (i, k)
            G += (A @ A.T).reshape(N, N, N, N).transpose(0, 2, 1, 3)
    return G


def energy_from_rdms(h: np.ndarray, v: np.ndarray, g: np.ndarray, G: np.ndarray) -> float:
    """E = sum h gamma + 1/2 sum (ij|kl) Gamma_ijkl."""
    return float(np.sum(h * g) + 0.5 * np.sum(v * G))
