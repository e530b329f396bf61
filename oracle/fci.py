"""O1: full configuration interaction (exact definition of Eq. (1)).

Determinants |alpha string, beta string> = A+(alpha) B+(beta) |vac>, all alpha
creators (ascending orbital) before all beta creators.  The Hamiltonian is
written with the spin-summed excitation operators E_ij = sum_s a+_is a_js:

    H = sum_ij h_ij E_ij + 1/2 sum_ijkl (ij|kl) (E_ij E_kl - d_jk E_il)

which equals the normal-ordered two-body form of Eq. (1) (anticommute
a_js past a+_kt).  E_ij acting on a string gives the textbook sign
(-1)^(occupied orbitals passed).  Parity pinned (tests/test_oracle_fci.py):
one electron -> eig(h); v = 0 -> aufbau sum; Hubbard dimer closed form;
agreement with the independent Fock-space oracle (O2).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def strings(N: int, n: int):
    """All n-electron occupation bit strings of N orbitals, ascending."""
    out = []
    for occ in itertools.combinations(range(N), n):
        m = 0
        for o in occ:
            m |= 1 << o
        out.append(m)
    return out


def _excitation(N: int, strs):
    """Sparse matrices e[i][j] = a+_i a_j on the string space."""
    index = {s: k for k, s in enumerate(strs)}
    n = len(strs)
    mats = [[None] * N for _ in range(N)]
    for i in range(N):
        for j in range(N):
            rows, cols, vals = [], [], []
            for k, s in enumerate(strs):
                if not (s >> j) & 1:
                    continue
                sign = (-1) ** bin(s & ((1 << j) - 1)).count("1")
                s1 = s & ~(1 << j)
                if (s1 >> i) & 1:
                    continue
                sign *= (-1) ** bin(s1 & ((1 << i) - 1)).count("1")
                s2 = s1 | (1 << i)
                rows.append(index[s2])
                cols.append(k)
                vals.append(float(sign))
            mats[i][j] = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return mats


def fci_hamiltonian(h: np.ndarray, v: np.ndarray, n_alpha: int, n_beta: int, e_core: float = 0.0):
    """Sparse FCI Hamiltonian over |alpha,beta> determinants (index ia*nb + ib)."""
    N = h.shape[0]
    sa, sb = strings(N, n_alpha), strings(N, n_beta)
    ea, eb = _excitation(N, sa), _excitation(N, sb)
    Ia = sp.identity(len(sa), format="csr")
    Ib = sp.identity(len(sb), format="csr")
    E = [[sp.kron(ea[i][j], Ib, format="csr") + sp.kron(Ia, eb[i][j], format="csr")
          for j in range(N)] for i in range(N)]
    dim = len(sa) * len(sb)
    H = sp.csr_matrix((dim, dim))
    for i in range(N):
        for j in range(N):
            H = H + h[i, j] * E[i][j]
    # 1/2 sum_kl (sum_ij (ij|kl) E_ij) E_kl  -  1/2 sum_il (sum_j (ij|jl)) E_il
    for k in range(N):
        for l in range(N):
            F = sp.csr_matrix((dim, dim))
            for i in range(N):
                for j in range(N):
                    if v[i, j, k, l] != 0.0:
                        F = F + v[i, j, k, l] * E[i][j]
            H = H + 0.5 * (F @ E[k][l])
    x = np.einsum("ijjl->il", v)
    for i in range(N):
        for l in range(N):
            H = H - 0.5 * x[i, l] * E[i][l]
    if e_core:
        H = H + e_core * sp.identity(dim)
    return H.tocsr()


def fci_energy(h, v, n_elec: int, two_sz: int, nroots: int = 1, e_core: float = 0.0):
    """Lowest eigenvalue(s) of H in the (n_elec, 2Sz) sector."""
    na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
    H = fci_hamiltonian(h, v, na, nb, e_core)
    dim = H.shape[0]
    if dim <= 3000:
        w = np.linalg.eigvalsh(H.toarray())
        return w[:nroots] if nroots > 1 else float(w[0])
    w = spla.eigsh(H, k=nroots, which="SA", tol=1e-14, maxiter=100000)[0]
    w = np.sort(w)
    return w if nroots > 1 else float(w[0])
