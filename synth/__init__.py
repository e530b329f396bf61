"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and lays them out; it holds none of the
DMRG arithmetic (no operators, no contractions, no eigen/SVD steps of the
method).  Both sides of every parity test receive the arrays made here.

Contents
--------
* ``integrals(N, lam, seed)`` -- random quantum-chemistry integrals standing in
  for the molecular integrals of the paper's F2 / FeMoco runs (Sec. IV.A):
  h_ij symmetric with entries N(0,1)*exp(-|i-j|/lam); v_ijkl in chemist order
  (ij|kl) with the 8-fold permutational symmetry, entries
  N(0,0.5)*exp(-(|i-j|+|k-l|)/lam), plus 1.0 on every (ii|ii).
* ``bond_sectors`` / ``random_mps`` -- a random matrix product state with
  U(1)xU(1) (particle number, 2*S_z) block structure, orthonormalised per
  symmetry block (left-canonical left of the two-site centre, right-canonical
  right of it).  Used as the shared input that fixes H_eff for parity tests.
* ``random_psi(keys, dims, seed)`` -- random two-site wavefunction blocks.

Conventions (shared with the C ABI, ``include/tns.h``):
  * site basis order |0>, |up>, |dn>, |updn>; quantum numbers (n, 2S_z) =
    (0,0), (1,1), (1,-1), (2,0);
  * bond b (0..N) carries the quantum numbers of sites 0..b-1 ("left counted");
  * a site tensor block (q_l, s) maps the bond-b sector q_l to the bond-(b+1)
    sector q_l + qn(s); it is a dim(q_l) x dim(q_l+qn(s)) row-major array.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

SITE_QN = ((0, 0), (1, 1), (1, -1), (2, 0))

Sector = Tuple[int, int]


# ---------------------------------------------------------------------------
# integrals
# ---------------------------------------------------------------------------
def integrals(N: int, lam: float, seed: int, diag_coulomb: float = 1.0):
    """Random (h, v) with the symmetry of real molecular integrals.

    Draw order: one ``numpy.random.default_rng(seed)`` stream; h for i<=j in
    row-major order, then v for the canonical quadruples i>=j, k>=l,
    ij>=kl (compound index i*(i+1)/2+j) in lexicographic (i,j,k,l) order.
    The decay factor exp(-(|i-j|+|k-l|)/lam) is invariant under the eight
    index permutations, so filling the images keeps the symmetry exact.
    Returns h (N,N) and v (N,N,N,N) float64, v[i,j,k,l] = (ij|kl).
    """
    rng = np.random.default_rng(seed)
    h = np.zeros((N, N))
    for i in range(N):
        for j in range(i, N):
            x = rng.standard_normal() * math.exp(-abs(i - j) / lam)
            h[i, j] = h[j, i] = x
    v = np.zeros((N, N, N, N))
    for i in range(N):
        for j in range(i + 1):
            ij = i * (i + 1) // 2 + j
            for k in range(N):
                for l in range(k + 1):
                    kl = k * (k + 1) // 2 + l
                    if kl > ij:
                        continue
                    x = 0.5 * rng.standard_normal() * math.exp(-(abs(i - j) + abs(k - l)) / lam)
                    for (a, b) in ((i, j), (j, i)):
                        for (c, d) in ((k, l), (l, k)):
                            v[a, b, c, d] = x
                            v[c, d, a, b] = x
    for i in range(N):
        v[i, i, i, i] += diag_coulomb
    return h, v


# ---------------------------------------------------------------------------
# bond sector tables of a random MPS
# ---------------------------------------------------------------------------
def _count(nsites: int, n: int, s2: int) -> int:
    """Number of determinants of ``nsites`` orbitals with n electrons, 2Sz=s2."""
    if (n + s2) % 2:
        return 0
    nu, nd = (n + s2) // 2, (n - s2) // 2
    if nu < 0 or nd < 0 or nu > nsites or nd > nsites:
        return 0
    return math.comb(nsites, nu) * math.comb(nsites, nd)


def bond_sectors(N: int, n_elec: int, two_sz: int, D: int,
                 max_sectors: int = 0) -> List[List[Tuple[Sector, int]]]:
    """Per bond b=0..N, the list of (sector, dim), sectors sorted by (n, 2Sz).

    dim = min(#left determinants, #right determinants) (the Schmidt-rank
    bound), scaled down proportionally when the total exceeds D, then made
    consistent so that every site tensor can be orthonormalised both ways.
    max_sectors > 0 keeps only that many sectors per bond (those with the
    largest bound, ties by sector), which concentrates D in a few large
    sectors.
    """
    target = (n_elec, two_sz)
    dims: List[Dict[Sector, int]] = []
    for b in range(N + 1):
        full = {}
        for n in range(0, 2 * b + 1):
            for s2 in range(-b, b + 1):
                cl = _count(b, n, s2)
                cr = _count(N - b, target[0] - n, target[1] - s2)
                if cl and cr:
                    full[(n, s2)] = min(cl, cr)
        if max_sectors > 0 and len(full) > max_sectors:
            keep = sorted(full, key=lambda q: (-full[q], q))[:max_sectors]
            full = {q: full[q] for q in keep}
        tot = sum(full.values())
        if tot > D:
            # proportional share, remainder to the largest fractional parts
            share = {q: D * f / tot for q, f in full.items()}
            alloc = {q: int(x) for q, x in share.items()}
            rest = D - sum(alloc.values())
            for q in sorted(share, key=lambda q: (-(share[q] - alloc[q]), q))[:rest]:
                alloc[q] += 1
            full = alloc
        dims.append(full)
    changed = True
    while changed:
        changed = False
        for b in range(1, N + 1):  # dim_b(q) <= sum_s dim_{b-1}(q - s)
            for q in list(dims[b]):
                avail = sum(dims[b - 1].get((q[0] - a, q[1] - c), 0) for a, c in SITE_QN)
                if dims[b][q] > avail:
                    dims[b][q] = avail
                    changed = True
        for b in range(N - 1, -1, -1):  # dim_b(q) <= sum_s dim_{b+1}(q + s)
            for q in list(dims[b]):
                avail = sum(dims[b + 1].get((q[0] + a, q[1] + c), 0) for a, c in SITE_QN)
                if dims[b][q] > avail:
                    dims[b][q] = avail
                    changed = True
    return [sorted(((q, d) for q, d in db.items() if d > 0)) for db in dims]


def random_mps(N: int, n_elec: int, two_sz: int, D: int, center: int, seed: int, max_sectors: int = 0):
    """Random block-sparse MPS, left-canonical on sites <= center and
    right-canonical on sites >= center+1.

    Returns (bonds, sites): ``bonds[b]`` = [(sector, dim)], ``sites[b]`` =
    {(q_l, s): ndarray(dim_b(q_l), dim_{b+1}(q_l+qn(s)))}.
    Orthonormalisation uses numpy QR on Gaussian matrices (input generation,
    not part of the method).
    """
    rng = np.random.default_rng(seed)
    bonds = bond_sectors(N, n_elec, two_sz, D, max_sectors)
    sites = []
    for b in range(N):
        left = dict(bonds[b])
        right = dict(bonds[b + 1])
        blocks = {}
        if b <= center:
            for qr, dr in bonds[b + 1]:
                parts = []
                for s, (a, c) in enumerate(SITE_QN):
                    ql = (qr[0] - a, qr[1] - c)
                    if ql in left:
                        parts.append((ql, s, left[ql]))
                rows = sum(p[2] for p in parts)
                g = rng.standard_normal((rows, dr))
                qm, _ = np.linalg.qr(g)
                r0 = 0
                for ql, s, dl in parts:
                    blocks[(ql, s)] = np.ascontiguousarray(qm[r0:r0 + dl, :])
                    r0 += dl
        else:
            for ql, dl in bonds[b]:
                parts = []
                for s, (a, c) in enumerate(SITE_QN):
                    qr = (ql[0] + a, ql[1] + c)
                    if qr in right:
                        parts.append((qr, s, right[qr]))
                cols = sum(p[2] for p in parts)
                g = rng.standard_normal((cols, dl))
                qm, _ = np.linalg.qr(g)
                qt = qm.T
                c0 = 0
                for qr, s, dr in parts:
                    blocks[(ql, s)] = np.ascontiguousarray(qt[:, c0:c0 + dr])
                    c0 += dr
        sites.append(blocks)
    return bonds, sites


def psi_keys(bonds, N: int, n_elec: int, two_sz: int, k: int):
    """Keys (q_l, s1, s2, q_r) of the two-site wavefunction at sites (k, k+1).

    q_l is a bond-k sector (left counted), q_r is the particle content of sites
    k+2..N-1 ("right counted", = target - bond-(k+2) sector)."""
    target = (n_elec, two_sz)
    left = bonds[k]
    right = [((target[0] - q[0], target[1] - q[1]), d) for q, d in bonds[k + 2]]
    keys = []
    for ql, dl in left:
        for s1, (a1, c1) in enumerate(SITE_QN):
            for s2, (a2, c2) in enumerate(SITE_QN):
                for qr, dr in right:
                    if (ql[0] + a1 + a2 + qr[0], ql[1] + c1 + c2 + qr[1]) == target:
                        keys.append(((ql, s1, s2, qr), (dl, dr)))
    return keys


def random_psi(keys, seed: int, nvec: int = 1):
    """Gaussian blocks for each (key, (m, n)); returns list of dicts (one per vector)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nvec):
        out.append({key: rng.standard_normal(dims) for key, dims in keys})
    return out


# workloads (sizes follow the five benchmark systems; the decay length of the
# 40- and 30-orbital systems is not stated and is taken as 5)
WORKLOADS = {
    "n8":  dict(N=8,  n_elec=8,   two_sz=0, lam=3.0, seed=0, D=256),
    "n24": dict(N=24, n_elec=24,  two_sz=0, lam=5.0, seed=1, D=512),
    "n40": dict(N=40, n_elec=40,  two_sz=0, lam=5.0, seed=2, D=1024),
    "n30": dict(N=30, n_elec=30,  two_sz=0, lam=5.0, seed=3, D=512),
    "n76": dict(N=76, n_elec=113, two_sz=1, lam=8.0, seed=4, D=2048),
}
