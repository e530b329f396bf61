"""Fermionic building blocks of the oracle (Eq. (1), Sec. III).

Site basis (one spatial orbital): |0>, |up>, |dn>, |updn> with
|updn> = c+_up c+_dn |0>; Jordan-Wigner order (0up, 0dn, 1up, 1dn, ...).

Hamiltonian of Eq. (1), read as the spin-free quantum-chemistry operator
    H = sum_ij h_ij sum_s c+_is c_js
      + 1/2 sum_ijkl (ij|kl) sum_st c+_is c+_kt c_lt c_js,
i.e. T_ij^{ab} = h_ij d_ab and, over spin-orbitals p=(i,s),
    H = sum_pq t_pq c+_p c_q + 1/2 sum_pqrs W_pqrs c+_p c+_q c_r c_s,
    t_pq   = h(i_p, i_q) d(s_p, s_q),
    W_pqrs = (i_p i_s | i_q i_r) d(s_p, s_s) d(s_q, s_r).
"""
from __future__ import annotations

import numpy as np

# creation operators on one orbital, index 0 = up, 1 = dn
CDAG = np.zeros((2, 4, 4))
CDAG[0][1, 0] = 1.0   # c+_up |0>  = |up>
CDAG[0][3, 2] = 1.0   # c+_up |dn> = c+_up c+_dn |0> = |updn>
CDAG[1][2, 0] = 1.0   # c+_dn |0>  = |dn>
CDAG[1][3, 1] = -1.0  # c+_dn |up> = c+_dn c+_up |0> = -|updn>
PAR = np.diag([1.0, -1.0, -1.0, 1.0])      # (-1)^n on one orbital
N_SITE = np.array([0, 1, 1, 2])
SZ2_SITE = np.array([0, 1, -1, 0])


def spin_orbital_integrals(h: np.ndarray, v: np.ndarray):
    """t (2N,2N) and W (2N)^4 over spin-orbitals p = 2*i + s (see module doc)."""
    N = h.shape[0]
    M = 2 * N
    t = np.zeros((M, M))
    for s in range(2):
        t[s::2, s::2] = h
    W = np.zeros((M, M, M, M))
    # W[p,q,r,s] = v[i_p, i_s, i_q, i_r] when s_p == s_s and s_q == s_r
    vt = np.transpose(v, (0, 2, 3, 1))  # vt[i,k,l,j] = v[i,j,k,l]
    for sp in range(2):
        for sq in range(2):
            W[sp::2, sq::2, sq::2, sp::2] = vt
    return t, W
