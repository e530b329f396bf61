"""O3: dense-operator two-site DMRG with normal/complementary operators.

Plain FP64 numpy.  Block operators are dense D x D matrices in the block
basis; symmetry is used only to label states (no blocking), so every formula
below can be read against the derivation it comes from.

Partition (Sec. III.A.2): left block L (orbitals 0..k-1), dot k, dot k+1,
right block R (orbitals k+2..N-1).  The Hamiltonian of Eq. (1) is split at
the bond between the enlarged blocks LL = L+dot k and RR = dot k+1 + R:

  H = H_LL + H_RR + sum_{a in LL} [c+_a S_a + h.c.] + sum_{x in RR} [T_x c_x + h.c.]
      + sum_{a<b in LL} [A_ab P_ab + h.c.] + sum_{a,b in LL} B_ab Q_ab          (*)

with normal operators on the left (c+_a, A_ab = c+_a c+_b, B_ab = c+_a c_b) and
complementary operators (partial summations over the integrals, which bring
the operator count from N^4 to N^2) on the right:
  S_a  = sum_{qru in R} W_aqru c+_q c_r c_u + sum_{x in R} t_ax c_x
  P_ab = sum_{ru in R} W_abru c_r c_u              (a < b)
  Q_ab = sum_{qr in R} (W_aqrb - W_aqbr) c+_q c_r
and on the left, for x right of the block,
  T_x  = sum_{pqr in L} W_pqrx c+_p c+_q c_r.
Spin-orbital integrals t, W: see ``fermion``.

Operators are block-local (Jordan-Wigner string inside the block only).  A
product (X)_left (Y)_right of full-space operators on two adjacent parts is
(X P_left^{|Y|}) (x) Y, P = (-1)^n the parity of the left part and |Y| the
fermionic parity of Y.  Enlarged ops are np.kron(X, y) with index l*4+s for
LL and np.kron(y, X) with index s*D_R+r for RR.  Renormalisation is
O' = A^T O A (left) and O' = B O B^T (right), Sec. III (blocking).
Parity pinned (tests/test_oracle_dmrg.py) against O2 (H_eff*psi, block
operators by definition) and O1 (energies).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .fermion import CDAG, PAR, N_SITE, SZ2_SITE, spin_orbital_integrals

SITE_QN = list(zip(N_SITE.tolist(), SZ2_SITE.tolist()))
I4 = np.eye(4)
CD = [CDAG[0], CDAG[1]]   # c+_up, c+_dn on one orbital
C = [CDAG[0].T, CDAG[1].T]


class Block:
    """A block: basis labels (n, 2Sz per state) and a dict of dense operators."""

    def __init__(self, n, sz, ops):
        self.n = np.asarray(n, dtype=int)
        self.sz = np.asarray(sz, dtype=int)
        self.ops = ops

    @property
    def dim(self):
        return len(self.n)

    @property
    def P(self):
        return np.diag((-1.0) ** self.n)


class Integrals:
    def __init__(self, h, v):
        self.h = np.asarray(h, float)
        self.v = np.asarray(v, float)
        self.N = self.h.shape[0]
        self.t, self.W = spin_orbital_integrals(self.h, self.v)


def _site_ops(s):
    """spin-orbital index -> (c+, c) on its own orbital."""
    return CD[s % 2], C[s % 2]


def site_hamiltonian(ints: Integrals, i: int):
    t, W = ints.t, ints.W
    ms = (2 * i, 2 * i + 1)
    h = np.zeros((4, 4))
    for p in ms:
        for q in ms:
            h += t[p, q] * CD[p % 2] @ C[q % 2]
    for p in ms:
        for q in ms:
            for r in ms:
                for s in ms:
                    if W[p, q, r, s] != 0.0:
                        h += 0.5 * W[p, q, r, s] * CD[p % 2] @ CD[q % 2] @ C[r % 2] @ C[s % 2]
    return h


# ---------------------------------------------------------------------------
# empty blocks
# ---------------------------------------------------------------------------
def empty_left(ints: Integrals) -> Block:
    M = 2 * ints.N
    ops = {"H": np.zeros((1, 1))}
    for x in range(M):
        ops[("T", x)] = np.zeros((1, 1))
    return Block([0], [0], ops)


def empty_right(ints: Integrals) -> Block:
    M = 2 * ints.N
    ops = {"H": np.zeros((1, 1))}
    for a in range(M):
        ops[("S", a)] = np.zeros((1, 1))
        for b in range(M):
            ops[("Q", a, b)] = np.zeros((1, 1))
            if a < b:
                ops[("P", a, b)] = np.zeros((1, 1))
    return Block([0], [0], ops)


def _keys(block, tag):
    return [k for k in block.ops if isinstance(k, tuple) and k[0] == tag]


# ---------------------------------------------------------------------------
# blocking: LL = L (x) site i   (site i = the orbital right of L)
# ---------------------------------------------------------------------------
def enlarge_left(L: Block, i: int, ints: Integrals) -> Block:
    t, W = ints.t, ints.W
    M = 2 * ints.N
    D = L.dim
    IL, PL = np.eye(D), L.P
    ms = (2 * i, 2 * i + 1)
    Lc = {k[1]: L.ops[k] for k in _keys(L, "c")}
    LA = {(k[1], k[2]): L.ops[k] for k in _keys(L, "A")}
    LB = {(k[1], k[2]): L.ops[k] for k in _keys(L, "B")}
    LT = {k[1]: L.ops[k] for k in _keys(L, "T")}
    inL = sorted(Lc)
    ops = {}
    # creation operators
    for a in inL:
        ops[("c", a)] = np.kron(Lc[a], I4)
    for m in ms:
        ops[("c", m)] = np.kron(PL, CD[m % 2])
    # pair operators A_ab = c+_a c+_b, a < b
    for (a, b), X in LA.items():
        ops[("A", a, b)] = np.kron(X, I4)
    for a in inL:
        for m in ms:
            ops[("A", a, m)] = np.kron(Lc[a] @ PL, CD[m % 2])
    ops[("A", ms[0], ms[1])] = np.kron(IL, CD[0] @ CD[1])
    # B_ab = c+_a c_b
    for (a, b), X in LB.items():
        ops[("B", a, b)] = np.kron(X, I4)
    for a in inL:
        for m in ms:
            ops[("B", a, m)] = np.kron(Lc[a] @ PL, C[m % 2])
            ops[("B", m, a)] = -np.kron(Lc[a].T @ PL, CD[m % 2])
    for m in ms:
        for n in ms:
            ops[("B", m, n)] = np.kron(IL, CD[m % 2] @ C[n % 2])
    # three-index complementary T_x for x right of LL
    for x in range(2 * i + 2, M):
        T = np.kron(LT[x], I4)
        for m in ms:
            Bs = np.zeros((D, D))
            for (q, r), X in LB.items():
                Bs += (W[m, q, r, x] - W[q, m, r, x]) * X
            T += np.kron(Bs @ PL, CD[m % 2])
            As = np.zeros((D, D))
            for (p, q), X in LA.items():
                As += (W[p, q, m, x] - W[q, p, m, x]) * X
            T += np.kron(As @ PL, C[m % 2])
        for a in inL:
            y1 = np.zeros((4, 4))   # c_a (x) c+_p c+_q   (p, q on the site)
            y2 = np.zeros((4, 4))   # c+_a (x) c+_q c_r
            for p in ms:
                for q in ms:
                    y1 += W[p, q, a, x] * CD[p % 2] @ CD[q % 2]
                    y2 += (W[a, p, q, x] - W[p, a, q, x]) * CD[p % 2] @ C[q % 2]
            T += np.kron(Lc[a].T, y1) + np.kron(Lc[a], y2)
        y3 = np.zeros((4, 4))
        for p in ms:
            for q in ms:
                for r in ms:
                    y3 += W[p, q, r, x] * CD[p % 2] @ CD[q % 2] @ C[r % 2]
        T += np.kron(PL, y3)
        ops[("T", x)] = T
    # Hamiltonian of LL: H_L + h_site + cross terms of the L | site bipartition
    H = np.kron(L.ops["H"], I4) + np.kron(IL, site_hamiltonian(ints, i))
    for a in inL:
        S = np.zeros((4, 4))
        for q in ms:
            S += t[a, q] * C[q % 2]
            for r in ms:
                for u in ms:
                    S += W[a, q, r, u] * CD[q % 2] @ C[r % 2] @ C[u % 2]
        H += np.kron(Lc[a] @ PL, S) - np.kron(Lc[a].T @ PL, S.T)
    for m in ms:
        H += np.kron(LT[m] @ PL, C[m % 2]) - np.kron(LT[m].T @ PL, CD[m % 2])
    for (a, b), X in LA.items():
        Pp = np.zeros((4, 4))
        for r in ms:
            for u in ms:
                Pp += W[a, b, r, u] * C[r % 2] @ C[u % 2]
        H += np.kron(X, Pp) + np.kron(X.T, Pp.T)
    for (a, b), X in LB.items():
        Q = np.zeros((4, 4))
        for q in ms:
            for r in ms:
                Q += (W[a, q, r, b] - W[a, q, b, r]) * CD[q % 2] @ C[r % 2]
        H += np.kron(X, Q)
    ops["H"] = H
    n = (L.n[:, None] + N_SITE[None, :]).ravel()
    sz = (L.sz[:, None] + SZ2_SITE[None, :]).ravel()
    return Block(n, sz, ops)


# ---------------------------------------------------------------------------
# blocking: RR = site i (x) R   (site i = the orbital left of R)
# ---------------------------------------------------------------------------
def enlarge_right(R: Block, i: int, ints: Integrals) -> Block:
    t, W = ints.t, ints.W
    D = R.dim
    IR = np.eye(D)
    P4 = PAR
    ms = (2 * i, 2 * i + 1)
    Rc = {k[1]: R.ops[k] for k in _keys(R, "c")}
    RS = {k[1]: R.ops[k] for k in _keys(R, "S")}
    RP = {(k[1], k[2]): R.ops[k] for k in _keys(R, "P")}
    RQ = {(k[1], k[2]): R.ops[k] for k in _keys(R, "Q")}
    inR = sorted(Rc)
    outside = range(0, 2 * i)
    ops = {}
    for m in ms:
        ops[("c", m)] = np.kron(CD[m % 2], IR)
    for x in inR:
        ops[("c", x)] = np.kron(P4, Rc[x])
    # S_a for a left of RR
    for a in outside:
        S = np.kron(P4, RS[a])
        for m in ms:
            S += np.kron(CD[m % 2], RP[(a, m)])
            S += np.kron(C[m % 2], RQ[(a, m)])
            S += t[a, m] * np.kron(C[m % 2], IR)
        for x in inR:
            y1 = np.zeros((4, 4))  # (c+_q c_r P) (x) c_x
            y3 = np.zeros((4, 4))  # (c_r c_u P) (x) c+_x
            for q in ms:
                for r in ms:
                    y1 += (W[a, q, r, x] - W[a, q, x, r]) * CD[q % 2] @ C[r % 2]
                    y3 += W[a, x, q, r] * C[q % 2] @ C[r % 2]
            S += np.kron(y1 @ P4, Rc[x].T) + np.kron(y3 @ P4, Rc[x])
        y = np.zeros((4, 4))
        for q in ms:
            for r in ms:
                for u in ms:
                    y += W[a, q, r, u] * CD[q % 2] @ C[r % 2] @ C[u % 2]
        S += np.kron(y, IR)
        ops[("S", a)] = S
    # P_ab, Q_ab for a, b left of RR
    for a in outside:
        for b in outside:
            Q = np.kron(I4, RQ[(a, b)])
            for m in ms:
                for x in inR:
                    cqr = W[a, m, x, b] - W[a, m, b, x]   # c+_m c_x
                    crq = W[a, x, m, b] - W[a, x, b, m]   # c+_x c_m
                    if cqr:
                        Q += cqr * np.kron(CD[m % 2] @ P4, Rc[x].T)
                    if crq:
                        Q -= crq * np.kron(C[m % 2] @ P4, Rc[x])
            y = np.zeros((4, 4))
            for q in ms:
                for r in ms:
                    y += (W[a, q, r, b] - W[a, q, b, r]) * CD[q % 2] @ C[r % 2]
            Q += np.kron(y, IR)
            ops[("Q", a, b)] = Q
            if a < b:
                Pm = np.kron(I4, RP[(a, b)])
                for m in ms:
                    for x in inR:
                        cf = W[a, b, m, x] - W[a, b, x, m]
                        if cf:
                            Pm += cf * np.kron(C[m % 2] @ P4, Rc[x].T)
                y = np.zeros((4, 4))
                for r in ms:
                    for u in ms:
                        y += W[a, b, r, u] * C[r % 2] @ C[u % 2]
                Pm += np.kron(y, IR)
                ops[("P", a, b)] = Pm
    # Hamiltonian of RR: h_site + H_R + cross terms of the site | R bipartition
    H = np.kron(site_hamiltonian(ints, i), IR) + np.kron(I4, R.ops["H"])
    for m in ms:
        H += np.kron(CD[m % 2] @ P4, RS[m]) - np.kron(C[m % 2] @ P4, RS[m].T)
    for x in inR:
        Ts = np.zeros((4, 4))
        for p in ms:
            for q in ms:
                for r in ms:
                    Ts += W[p, q, r, x] * CD[p % 2] @ CD[q % 2] @ C[r % 2]
        H += np.kron(Ts @ P4, Rc[x].T) - np.kron(Ts.T @ P4, Rc[x])
    As = CD[0] @ CD[1]
    H += np.kron(As, RP[ms]) + np.kron(As.T, RP[ms].T)
    for m in ms:
        for n in ms:
            H += np.kron(CD[m % 2] @ C[n % 2], RQ[(m, n)])
    ops["H"] = H
    n = (N_SITE[:, None] + R.n[None, :]).ravel()
    sz = (SZ2_SITE[:, None] + R.sz[None, :]).ravel()
    return Block(n, sz, ops)


# ---------------------------------------------------------------------------
# renormalisation
# ---------------------------------------------------------------------------
def rotate_left(LL: Block, A: np.ndarray, n_new, sz_new) -> Block:
    """A: (D_L*4, D') isometry (rows l*4+s)."""
    return Block(n_new, sz_new, {k: A.T @ X @ A for k, X in LL.ops.items()})


def rotate_right(RR: Block, B: np.ndarray, n_new, sz_new) -> Block:
    """B: (D', 4*D_R) isometry (columns s*D_R+r)."""
    return Block(n_new, sz_new, {k: B @ X @ B.T for k, X in RR.ops.items()})


# ---------------------------------------------------------------------------
# H_eff * psi at the LL | RR bond, formula (*)
# ---------------------------------------------------------------------------
def heff_apply(LL: Block, RR: Block, Psi: np.ndarray) -> np.ndarray:
    """Psi: (dim LL, dim RR) matrix, rows (l, s1), cols (s2, r)."""
    PLL = LL.P
    Y = LL.ops["H"] @ Psi + Psi @ RR.ops["H"].T
    for k in _keys(LL, "c"):
        a = k[1]
        X = LL.ops[k]
        S = RR.ops[("S", a)]
        Y += (X @ PLL) @ Psi @ S.T - (X.T @ PLL) @ Psi @ S
    for k in _keys(RR, "c"):
        x = k[1]
        T = LL.ops[("T", x)]
        cx = RR.ops[k]
        Y += (T @ PLL) @ Psi @ cx - (T.T @ PLL) @ Psi @ cx.T
    for k in _keys(LL, "A"):
        X = LL.ops[k]
        P = RR.ops[("P", k[1], k[2])]
        Y += X @ Psi @ P.T + X.T @ Psi @ P
    for k in _keys(LL, "B"):
        Y += LL.ops[k] @ Psi @ RR.ops[("Q", k[1], k[2])].T
    return Y


def heff_apply_abs(LL: Block, RR: Block, Psi: np.ndarray) -> np.ndarray:
    """Error-bound helper (not the method): the term sum of ``heff_apply`` with
    every operator and Psi replaced by its elementwise absolute value,
    sum_a |O_a^LL| |Psi| |O_a^RR|^T.  The forward error of a sum of matrix
    products whose operands and partial results carry a relative rounding u is
    bounded elementwise by a small multiple of u times this sum."""
    A = np.abs
    Pa = A(Psi)
    Y = A(LL.ops["H"]) @ Pa + Pa @ A(RR.ops["H"]).T
    for k in _keys(LL, "c"):
        X, S = A(LL.ops[k]), A(RR.ops[("S", k[1])])
        Y += X @ Pa @ S.T + X.T @ Pa @ S
    for k in _keys(RR, "c"):
        T, cx = A(LL.ops[("T", k[1])]), A(RR.ops[k])
        Y += T @ Pa @ cx + T.T @ Pa @ cx.T
    for k in _keys(LL, "A"):
        X, P = A(LL.ops[k]), A(RR.ops[("P", k[1], k[2])])
        Y += X @ Pa @ P.T + X.T @ Pa @ P
    for k in _keys(LL, "B"):
        Y += A(LL.ops[k]) @ Pa @ A(RR.ops[("Q", k[1], k[2])]).T
    return Y


# ---------------------------------------------------------------------------
# block-sparse MPS <-> dense helpers
# ---------------------------------------------------------------------------
def bond_labels(bond):
    n, sz, off = [], [], {}
    o = 0
    for q, d in bond:
        off[q] = o
        n += [q[0]] * d
        sz += [q[1]] * d
        o += d
    return np.array(n, int), np.array(sz, int), off


def dense_site(bonds, sites, b):
    """(D_b, 4, D_{b+1}) dense tensor from blocks."""
    nl, _, offl = bond_labels(bonds[b])
    nr, _, offr = bond_labels(bonds[b + 1])
    A = np.zeros((len(nl), 4, len(nr)))
    for (ql, s), blk in sites[b].items():
        qr = (ql[0] + SITE_QN[s][0], ql[1] + SITE_QN[s][1])
        if ql in offl and qr in offr:
            A[offl[ql]:offl[ql] + blk.shape[0], s, offr[qr]:offr[qr] + blk.shape[1]] = blk
    return A


def right_counted(n_elec, two_sz, bond):
    return [((n_elec - q[0], two_sz - q[1]), d) for q, d in bond]


def build_left(ints: Integrals, bonds, sites, k: int) -> Block:
    """Left block L_k (orbitals 0..k-1) by repeated blocking + renormalisation."""
    L = empty_left(ints)
    for b in range(k):
        LL = enlarge_left(L, b, ints)
        A = dense_site(bonds, sites, b).reshape(-1, sum(d for _, d in bonds[b + 1]))
        n, sz, _ = bond_labels(bonds[b + 1])
        L = rotate_left(LL, A, n, sz)
    return L


def build_right(ints: Integrals, bonds, sites, k: int, n_elec: int, two_sz: int) -> Block:
    """Right block R_k (orbitals k..N-1); labels are its own particle content."""
    N = ints.N
    R = empty_right(ints)
    for b in range(N - 1, k - 1, -1):
        RR = enlarge_right(R, b, ints)
        A = dense_site(bonds, sites, b)
        B = A.reshape(A.shape[0], -1)   # (D_b, 4*D_{b+1}) -> columns s*D+r
        n, sz, _ = bond_labels(right_counted(n_elec, two_sz, bonds[b]))
        R = rotate_right(RR, B, n, sz)
    return R


class DenseHeff:
    """H_eff at step (k, k+1) built from dense blocks; X/Y as block dicts."""

    def __init__(self, ints: Integrals, bonds, sites, k, n_elec, two_sz, L=None, R=None):
        self.ints = ints
        self.k = k
        self.target = (n_elec, two_sz)
        L = build_left(ints, bonds, sites, k) if L is None else L
        R = build_right(ints, bonds, sites, k + 2, n_elec, two_sz) if R is None else R
        self.L, self.R = L, R
        self.LL = enlarge_left(L, k, ints)
        self.RR = enlarge_right(R, k + 1, ints)
        _, _, self.offl = bond_labels(bonds[k])
        _, _, self.offr = bond_labels(right_counted(n_elec, two_sz, bonds[k + 2]))
        self.DL, self.DR = L.dim, R.dim

    def to_matrix(self, X: dict):
        Psi = np.zeros((self.DL * 4, 4 * self.DR))
        for (ql, s1, s2, qr), blk in X.items():
            a, c = self.offl[ql], self.offr[qr]
            m, n = blk.shape
            Psi[a * 4 + s1:(a + m) * 4:4, s2 * self.DR + c:s2 * self.DR + c + n] = blk
        return Psi

    def from_matrix(self, Y, keys):
        out = {}
        for (ql, s1, s2, qr), (m, n) in keys:
            a, c = self.offl[ql], self.offr[qr]
            out[(ql, s1, s2, qr)] = Y[a * 4 + s1:(a + m) * 4:4, s2 * self.DR + c:s2 * self.DR + c + n].copy()
        return out

    def apply(self, X: dict) -> dict:
        keys = [(key, blk.shape) for key, blk in X.items()]
        Y = heff_apply(self.LL, self.RR, self.to_matrix(X))
        return self.from_matrix(Y, keys)

    def apply_matrix(self, Psi):
        return heff_apply(self.LL, self.RR, Psi)

    def apply_abs(self, X: dict) -> dict:
        """sum_a |O_a^LL| |X| |O_a^RR|^T (error-bound helper, see heff_apply_abs)."""
        keys = [(key, blk.shape) for key, blk in X.items()]
        return self.from_matrix(heff_apply_abs(self.LL, self.RR, self.to_matrix(X)), keys)

    def sector_mask(self):
        n = (self.LL.n[:, None] + self.RR.n[None, :])
        sz = (self.LL.sz[:, None] + self.RR.sz[None, :])
        return (n == self.target[0]) & (sz == self.target[1])


# ---------------------------------------------------------------------------
# full sweep (oracle DMRG)
# ---------------------------------------------------------------------------
def _lowest(Hop, x0, tol):
    n = x0.size
    if n <= 1500:
        Hm = np.column_stack([Hop(e) for e in np.eye(n)])
        w, V = np.linalg.eigh(0.5 * (Hm + Hm.T))
        return w[0], V[:, 0]
    op = spla.LinearOperator((n, n), matvec=Hop, dtype=float)
    w, V = spla.eigsh(op, k=1, which="SA", v0=x0, tol=tol)
    return w[0], V[:, 0]


def _truncate(theta_mat, nrow, szrow, ncol, szcol, D, left_to_right):
    """SVD per middle-bond sector (labelled by the row content), keep top D."""
    sectors = sorted(set(zip(nrow.tolist(), szrow.tolist())))
    parts = []
    for q in sectors:
        ri = np.nonzero((nrow == q[0]) & (szrow == q[1]))[0]
        ci = np.nonzero((ncol == q[0]) & (szcol == q[1]))[0]   # cols labelled by matching content
        if len(ri) == 0 or len(ci) == 0:
            continue
        U, s, Vt = np.linalg.svd(theta_mat[np.ix_(ri, ci)], full_matrices=False)
        parts.append((q, ri, ci, U, s, Vt))
    allsv = []
    for pi, (q, ri, ci, U, s, Vt) in enumerate(parts):
        for j, x in enumerate(s):
            allsv.append((-x, pi, j))
    allsv.sort()
    keep = [e for e in allsv if -e[0] > 1e-14][:D]
    discarded = sum(e[0] ** 2 for e in allsv) - sum(e[0] ** 2 for e in keep)
    kept = {}
    for _, pi, j in keep:
        kept.setdefault(pi, []).append(j)
    return parts, kept, discarded


def dmrg(h, v, n_elec, two_sz, D, nsweeps, seed=0, tol=1e-12, verbose=False):
    """Plain two-site DMRG with dense operators; returns (energy, history).

    Start: random right-canonical MPS (synthetic input, all sites right
    canonical).  Each step: blocking, H_eff lowest eigenpair, SVD truncation
    to at most D states, renormalisation.  Sweeps L->R then R->L.
    """
    import synth  # seeded inputs only (random start); no method arithmetic
    ints = Integrals(h, v)
    N = ints.N
    bonds, sites = synth.random_mps(N, n_elec, two_sz, D, center=-1, seed=seed)
    dense = [dense_site(bonds, sites, b) for b in range(N)]
    labels = [bond_labels(bd)[:2] for bd in bonds]   # left-counted labels per bond
    # right blocks R_b for b = N..2
    Rb = {N: empty_right(ints)}
    for b in range(N - 1, 1, -1):
        RR = enlarge_right(Rb[b + 1], b, ints)
        n, sz = labels[b]
        Rb[b] = rotate_right(RR, dense[b].reshape(dense[b].shape[0], -1), n_elec - n, two_sz - sz)
    Lb = {0: empty_left(ints)}
    hist = []
    E = None
    psi_guess = None
    for sweep in range(nsweeps):
        for direction in (+1, -1):
            ks = range(0, N - 1) if direction > 0 else range(N - 2, -1, -1)
            for k in ks:
                if direction > 0 and k == N - 2 and sweep > 0:
                    pass
                LL = enlarge_left(Lb[k], k, ints)
                RR = enlarge_right(Rb[k + 2], k + 1, ints)
                mask = ((LL.n[:, None] + RR.n[None, :]) == n_elec) & ((LL.sz[:, None] + RR.sz[None, :]) == two_sz)
                idx = np.nonzero(mask.ravel())[0]
                shape = mask.shape

                def Hop(x):
                    Psi = np.zeros(shape)
                    Psi.ravel()[idx] = x
                    return heff_apply(LL, RR, Psi).ravel()[idx]

                x0 = np.random.default_rng(seed + 17 * k + sweep).standard_normal(idx.size)
                E, x = _lowest(Hop, x0, tol)
                Psi = np.zeros(shape)
                Psi.ravel()[idx] = x
                # SVD: rows = LL states (content q), cols = RR states (content target-q)
                parts, kept, disc = _truncate(Psi, LL.n, LL.sz, n_elec - RR.n, two_sz - RR.sz, D, direction > 0)
                qs, cols_l, cols_r = [], [], []
                for pi in sorted(kept):
                    q, ri, ci, U, s, Vt = parts[pi]
                    for j in kept[pi]:
                        u = np.zeros(shape[0]); u[ri] = U[:, j]
                        w = np.zeros(shape[1]); w[ci] = Vt[j, :]
                        cols_l.append(u); cols_r.append(w); qs.append(q)
                Um = np.array(cols_l).T          # (dim LL, D')
                Vm = np.array(cols_r)            # (D', dim RR)
                nq = np.array([q[0] for q in qs]); szq = np.array([q[1] for q in qs])
                if direction > 0:
                    Lb[k + 1] = rotate_left(LL, Um, nq, szq)
                else:
                    Rb[k + 1] = rotate_right(RR, Vm, n_elec - nq, two_sz - szq)
                hist.append((sweep, direction, k, E, disc))
                if verbose:
                    print(sweep, direction, k, E, disc)
    return E, hist


def useful_flops(heff: "DenseHeff") -> float:
    """Useful flop count of one H_eff*psi in the block-sparse form: over every
    term of formula (*), every dot block (s' <- s) of its left and right
    enlarged operators and every symmetry block of psi, the cheaper chain of
    the product L_blk X_blk R_blk^T: min(2mr(n+q), 2qn(m+r)).  Identity
    factors cost one product.  Pure counting over the nonzero blocks of the
    oracle's own dense operators (no arithmetic of the method)."""
    LL, RR = heff.LL, heff.RR
    DL, DR = heff.DL, heff.DR

    def sectors(n, sz):
        lab = list(zip(n.tolist(), sz.tolist()))
        out = {}
        for i, q in enumerate(lab):
            out.setdefault(q, []).append(i)
        return out

    # D-basis sector index sets of the two blocks
    secL = sectors(heff.L.n, heff.L.sz)
    secR = sectors(heff.R.n, heff.R.sz)

    def blocks(E, dim, left, sec):
        """{(s', s): [(q_out, q_in, is_identity)]} of the nonzero D-basis blocks."""
        out = {}
        for so in range(4):
            for si in range(4):
                if left:
                    M = E[so::4, si::4]
                else:
                    M = E[so * dim:(so + 1) * dim, si * dim:(si + 1) * dim]
                if not M.any():
                    continue
                lst = []
                ident = np.allclose(M, M[0, 0] * np.eye(dim)) if M[0, 0] != 0 else False
                for qo, io in sec.items():
                    for qi, ii in sec.items():
                        if M[np.ix_(io, ii)].any():
                            lst.append((qo, qi, ident and qo == qi))
                out[(so, si)] = lst
        return out

    terms = [(LL.ops["H"], None), (None, RR.ops["H"])]
    for k in _keys(LL, "c"):
        terms += [(LL.ops[k], RR.ops[("S", k[1])]), (LL.ops[k].T, RR.ops[("S", k[1])].T)]
    for k in _keys(RR, "c"):
        terms += [(LL.ops[("T", k[1])], RR.ops[k].T), (LL.ops[("T", k[1])].T, RR.ops[k])]
    for k in _keys(LL, "A"):
        P = RR.ops[("P", k[1], k[2])]
        terms += [(LL.ops[k], P), (LL.ops[k].T, P.T)]
    for k in _keys(LL, "B"):
        terms += [(LL.ops[k], RR.ops[("Q", k[1], k[2])])]
    eyeL = np.eye(4 * DL)
    eyeR = np.eye(4 * DR)
    dimL = {q: len(i) for q, i in secL.items()}
    dimR = {q: len(i) for q, i in secR.items()}
    tot = 0.0
    for El, Er in terms:
        bl = blocks(eyeL if El is None else El, DL, True, secL)
        br = blocks(eyeR if Er is None else Er, DR, False, secR)
        for (s1o, s1i), lb in bl.items():
            for (s2o, s2i), rb in br.items():
                for (qlo, qli, li) in lb:
                    for (qro, qri, ri) in rb:
                        # psi block (qli, s1i, s2i, qri) must be in the target sector
                        q, m = dimL[qlo], dimL[qli]
                        n, r = dimR[qri], dimR[qro]
                        nl = qli[0] + int(N_SITE[s1i]) + int(N_SITE[s2i]) + qri[0]
                        sl = qli[1] + int(SZ2_SITE[s1i]) + int(SZ2_SITE[s2i]) + qri[1]
                        if (nl, sl) != heff.target:
                            continue
                        if li and ri:
                            tot += 2.0 * m * n
                        elif li:
                            tot += 2.0 * m * n * r
                        elif ri:
                            tot += 2.0 * q * m * n
                        else:
                            tot += min(2.0 * m * r * (n + q), 2.0 * q * n * (m + r))
    return tot
