"""Pins of O3 (dense-operator DMRG with complementary operators) against O2 and O1."""
import numpy as np
import pytest

import synth
from oracle import dmrg as O3
from oracle.fci import fci_energy
from oracle.fock import FockHeff, fock_hamiltonian


def _rel(a, b):
    num = sum(np.sum((a[k] - b[k]) ** 2) for k in a)
    den = sum(np.sum(b[k] ** 2) for k in b)
    return np.sqrt(num / den)


@pytest.mark.parametrize("N,n,s2,D,k", [(5, 5, 1, 8, 0), (5, 4, 0, 8, 1), (6, 6, 0, 12, 2),
                                         (6, 5, -1, 9, 3), (6, 6, 2, 16, 4)])
def test_heff_matches_projected_fock(N, n, s2, D, k):
    h, v = synth.integrals(N, 2.0, 100 + N + k)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k + 1)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=3)[0]
    ref = FockHeff(h, v, bonds, sites, k, n, s2).apply(X)
    ints = O3.Integrals(h, v)
    got = O3.DenseHeff(ints, bonds, sites, k, n, s2).apply(X)
    assert _rel(got, ref) < 1e-13


def test_heff_hermitian_and_sector_closed():
    N, n, s2, D, k = 6, 6, 0, 20, 2
    h, v = synth.integrals(N, 2.0, 9)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=2)
    heff = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
    rng = np.random.default_rng(0)
    mask = heff.sector_mask()
    x = rng.standard_normal(mask.shape) * mask
    y = rng.standard_normal(mask.shape) * mask
    Hx, Hy = heff.apply_matrix(x), heff.apply_matrix(y)
    assert abs(np.sum(x * Hy) - np.sum(Hx * y)) < 1e-12 * np.abs(Hx).max() * x.size
    assert np.abs(Hx[~mask]).max() < 1e-13


def test_block_operators_by_definition():
    """L_k and R_k catalogue operators equal their defining sums in the Fock space."""
    from oracle.fock import cdag_ops, left_basis, right_basis
    N, n, s2, D, k = 5, 5, 1, 10, 2
    h, v = synth.integrals(N, 2.0, 31)
    ints = O3.Integrals(h, v)
    t, W = ints.t, ints.W
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=4)
    L = O3.build_left(ints, bonds, sites, k)
    Lb = left_basis(bonds, sites, k)
    cdL = cdag_ops(k)
    cL = [x.T for x in cdL]
    for a in range(2 * k):
        assert np.allclose(Lb.T @ (cdL[a] @ Lb), L.ops[("c", a)], atol=1e-13)
    for x in range(2 * k, 2 * N):
        T = sum(W[p, q, r, x] * (cdL[p] @ cdL[q] @ cL[r]).toarray()
                for p in range(2 * k) for q in range(2 * k) for r in range(2 * k))
        assert np.allclose(Lb.T @ T @ Lb, L.ops[("T", x)], atol=1e-12)
    kr = 3
    R = O3.build_right(ints, bonds, sites, kr, n, s2)
    Rb = right_basis(bonds, sites, kr, N)
    nr = N - kr
    cdR = cdag_ops(nr)
    cR = [x.T for x in cdR]
    off = 2 * kr
    for a in range(0, 2 * kr):
        S = sum(W[a, q + off, r + off, u + off] * (cdR[q] @ cR[r] @ cR[u]).toarray()
                for q in range(2 * nr) for r in range(2 * nr) for u in range(2 * nr))
        S = S + sum(t[a, x + off] * cR[x].toarray() for x in range(2 * nr))
        assert np.allclose(Rb.T @ S @ Rb, R.ops[("S", a)], atol=1e-12)
        for b in range(0, 2 * kr):
            Q = sum((W[a, q + off, r + off, b] - W[a, q + off, b, r + off]) * (cdR[q] @ cR[r]).toarray()
                    for q in range(2 * nr) for r in range(2 * nr))
            assert np.allclose(Rb.T @ Q @ Rb, R.ops[("Q", a, b)], atol=1e-12)
            if a < b:
                P = sum(W[a, b, r + off, u + off] * (cR[r] @ cR[u]).toarray()
                        for r in range(2 * nr) for u in range(2 * nr))
                assert np.allclose(Rb.T @ P @ Rb, R.ops[("P", a, b)], atol=1e-12)


@pytest.mark.slow
def test_dmrg_exact_bond_dimension_reaches_fci_n6():
    N, n, s2 = 6, 6, 0
    h, v = synth.integrals(N, 3.0, 0)
    e, _ = O3.dmrg(h, v, n, s2, D=64, nsweeps=3)
    assert abs(e - fci_energy(h, v, n, s2)) < 1e-10


def test_dmrg_energy_monotone_in_D():
    N, n, s2 = 6, 6, 0
    h, v = synth.integrals(N, 3.0, 1)
    es = [O3.dmrg(h, v, n, s2, D=D, nsweeps=3)[0] for D in (4, 8, 16)]
    efci = fci_energy(h, v, n, s2)
    assert es[0] >= es[1] - 1e-9 >= es[2] - 2e-9
    assert es[2] >= efci - 1e-9


def test_apply_abs_bounds_the_product():
    """The error-bound helper dominates the product elementwise and is linear
    in |psi|."""
    N, n, s2, D, k = 6, 6, 0, 12, 2
    h, v = synth.integrals(N, 2.0, 9)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=2)
    heff = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=4)[0]
    Y, Ya = heff.apply(X), heff.apply_abs(X)
    for q in Y:
        assert np.all(np.abs(Y[q]) <= Ya[q] + 1e-12)
    X2 = {q: 2.0 * np.abs(b) for q, b in X.items()}
    Ya2 = heff.apply_abs(X2)
    for q in Y:
        assert np.allclose(Ya2[q], 2.0 * Ya[q], rtol=1e-13, atol=0)
