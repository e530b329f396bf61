"""O2: Jordan-Wigner Fock-space Hamiltonian and the projected H_eff = P^T H P.

No block operators and no complementary operators: the two-site effective
Hamiltonian is the full Hamiltonian of Eq. (1) restricted to the basis
|l>_L |s1> |s2> |r>_R spanned by a given MPS (the four-subsystem two-site
topology of Sec. III.A.2).  Left/right block basis states are built as explicit
Fock vectors from the site tensors, so H_eff*psi = P^T (H (P psi)).

Fock index: kron order, site 0 most significant; site basis |0>,|up>,|dn>,
|updn>.  Usable up to ~8 orbitals (4^8 = 65536 states).
Parity pinned (tests/test_oracle_fock.py): canonical anticommutators, the
direct c+c+cc construction at 3 orbitals, lowest eigenvalue = FCI (O1), and
the exactness of H_eff at full bond dimension.
"""
from __future__ import annotations

from functools import reduce

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fermion import CDAG, PAR, N_SITE, SZ2_SITE

SITE_QN = list(zip(N_SITE.tolist(), SZ2_SITE.tolist()))


def _kron_all(mats):
    return reduce(lambda a, b: sp.kron(a, b, format="csr"), mats)


def cdag_ops(nsites: int):
    """Sparse c+_p on the 4^nsites Fock space with JW strings, p = 2*i + s."""
    I4 = sp.identity(4, format="csr")
    P4 = sp.csr_matrix(PAR)
    ops = []
    for i in range(nsites):
        for s in range(2):
            mats = [P4] * i + [sp.csr_matrix(CDAG[s])] + [I4] * (nsites - i - 1)
            ops.append(_kron_all(mats) if nsites > 1 else sp.csr_matrix(CDAG[s]))
    return ops


def fock_hamiltonian(h: np.ndarray, v: np.ndarray, e_core: float = 0.0):
    """H of Eq. (1) on the full Fock space via E_ij = sum_s c+_is c_js."""
    N = h.shape[0]
    cd = cdag_ops(N)
    E = [[cd[2 * i] @ cd[2 * j].T + cd[2 * i + 1] @ cd[2 * j + 1].T for j in range(N)] for i in range(N)]
    dim = 4 ** N
    H = sp.csr_matrix((dim, dim))
    for i in range(N):
        for j in range(N):
            if h[i, j] != 0.0:
                H = H + h[i, j] * E[i][j]
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
            if x[i, l] != 0.0:
                H = H - 0.5 * x[i, l] * E[i][l]
    if e_core:
        H = H + e_core * sp.identity(dim)
    return H.tocsr()


def fock_hamiltonian_direct(h: np.ndarray, v: np.ndarray):
    """H from the spin-orbital normal-ordered sum (slow; tiny N only)."""
    N = h.shape[0]
    cd = cdag_ops(N)
    c = [x.T.tocsr() for x in cd]
    dim = 4 ** N
    H = sp.csr_matrix((dim, dim))
    for i in range(N):
        for j in range(N):
            for s in range(2):
                H = H + h[i, j] * (cd[2 * i + s] @ c[2 * j + s])
    for i in range(N):
        for j in range(N):
            for k in range(N):
                for l in range(N):
                    if v[i, j, k, l] == 0.0:
                        continue
                    for s in range(2):
                        for t in range(2):
                            H = H + 0.5 * v[i, j, k, l] * (cd[2 * i + s] @ cd[2 * k + t] @ c[2 * l + t] @ c[2 * j + s])
    return H.tocsr()


def sector_indices(N: int, n: int, two_sz: int):
    """Fock indices of all states with particle number n and 2Sz = two_sz."""
    nn = np.zeros(1, dtype=int)
    ss = np.zeros(1, dtype=int)
    for _ in range(N):
        nn = (nn[:, None] + N_SITE[None, :]).ravel()
        ss = (ss[:, None] + SZ2_SITE[None, :]).ravel()
    return np.nonzero((nn == n) & (ss == two_sz))[0]


def sector_ground_energy(H, N: int, n: int, two_sz: int) -> float:
    idx = sector_indices(N, n, two_sz)
    Hs = H[idx][:, idx]
    if Hs.shape[0] <= 3000:
        return float(np.linalg.eigvalsh(Hs.toarray())[0])
    return float(spla.eigsh(Hs, k=1, which="SA", tol=1e-14)[0][0])


# ---------------------------------------------------------------------------
# explicit MPS basis vectors
# ---------------------------------------------------------------------------
def _offsets(bond):
    off, o = {}, 0
    for q, d in bond:
        off[q] = o
        o += d
    return off, o


def left_basis(bonds, sites, k: int):
    """Lb (4^k x D_k): column j = Fock vector of left state j of bond k."""
    Lb = np.ones((1, 1))
    for b in range(k):
        offl, dl = _offsets(bonds[b])
        offr, dr = _offsets(bonds[b + 1])
        new = np.zeros((Lb.shape[0] * 4, dr))
        for (ql, s), blk in sites[b].items():
            qr = (ql[0] + SITE_QN[s][0], ql[1] + SITE_QN[s][1])
            if ql not in offl or qr not in offr:
                continue
            a, m = offl[ql], blk.shape[0]
            c, n = offr[qr], blk.shape[1]
            # rows (x, s) = x*4 + s
            new[s::4, c:c + n] += Lb[:, a:a + m] @ blk
        Lb = new
    return Lb


def right_basis(bonds, sites, k: int, N: int):
    """Rb (4^(N-k) x D_k): column j = Fock vector of the right state j of bond k
    (sites k..N-1), for right-canonical site tensors."""
    Rb = np.ones((1, 1))
    for b in range(N - 1, k - 1, -1):
        offl, dl = _offsets(bonds[b])
        offr, dr = _offsets(bonds[b + 1])
        ny = Rb.shape[0]
        new = np.zeros((4 * ny, dl))
        for (ql, s), blk in sites[b].items():
            qr = (ql[0] + SITE_QN[s][0], ql[1] + SITE_QN[s][1])
            if ql not in offl or qr not in offr:
                continue
            a, m = offl[ql], blk.shape[0]
            c, n = offr[qr], blk.shape[1]
            # rows (s, y) = s*ny + y
            new[s * ny:(s + 1) * ny, a:a + m] += Rb[:, c:c + n] @ blk.T
        Rb = new
    return Rb


class FockHeff:
    """H_eff = P^T H P at the two-site step (k, k+1) of an N-orbital MPS."""

    def __init__(self, h, v, bonds, sites, k: int, n_elec: int, two_sz: int, H=None):
        N = h.shape[0]
        self.N, self.k = N, k
        self.target = (n_elec, two_sz)
        self.H = fock_hamiltonian(h, v) if H is None else H
        self.Lb = left_basis(bonds, sites, k)
        self.Rb = right_basis(bonds, sites, k + 2, N)
        self.offl, _ = _offsets(bonds[k])
        # right states of bond k+2 are labelled by their own content target - q
        self.offr = {}
        o = 0
        for q, d in bonds[k + 2]:
            self.offr[(n_elec - q[0], two_sz - q[1])] = o
            o += d

    def _to_fock(self, X: dict):
        nl, nr = self.Lb.shape[0], self.Rb.shape[0]
        Phi = np.zeros((nl, 4, 4, nr))
        for (ql, s1, s2, qr), blk in X.items():
            a, c = self.offl[ql], self.offr[qr]
            m, n = blk.shape
            Phi[:, s1, s2, :] += self.Lb[:, a:a + m] @ blk @ self.Rb[:, c:c + n].T
        return Phi.ravel()

    def _from_fock(self, phi, keys):
        nl, nr = self.Lb.shape[0], self.Rb.shape[0]
        Phi = phi.reshape(nl, 4, 4, nr)
        out = {}
        for (ql, s1, s2, qr), (m, n) in keys:
            a, c = self.offl[ql], self.offr[qr]
            out[(ql, s1, s2, qr)] = self.Lb[:, a:a + m].T @ Phi[:, s1, s2, :] @ self.Rb[:, c:c + n]
        return out

    def apply(self, X: dict) -> dict:
        keys = [(key, blk.shape) for key, blk in X.items()]
        return self._from_fock(self.H @ self._to_fock(X), keys)

    def ground_energy(self, keys) -> float:
        """Lowest eigenvalue of H_eff on the block space ``keys``."""
        sizes = [m * n for _, (m, n) in keys]
        tot = sum(sizes)

        def unpack(x):
            out, o = {}, 0
            for (key, (m, n)) in keys:
                out[key] = x[o:o + m * n].reshape(m, n)
                o += m * n
            return out

        def mv(x):
            y = self.apply(unpack(np.asarray(x).ravel()))
            return np.concatenate([y[key].ravel() for key, _ in keys])

        if tot <= 2500:
            Hm = np.column_stack([mv(e) for e in np.eye(tot)])
            return float(np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[0])
        op = spla.LinearOperator((tot, tot), matvec=mv, dtype=float)
        return float(spla.eigsh(op, k=1, which="SA", tol=1e-13)[0][0])
