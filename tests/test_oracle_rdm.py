"""Pins of the oracle's reduced density matrices (O4) against facts that do not
come from the oracle itself: Wick's theorem for single determinants, the
particle-number trace and partial-trace identities, index symmetries of a real
state, and the energy identity against the Fock-space Hamiltonian (O2)."""
import numpy as np
import pytest

import synth
from oracle import fock as O2
from oracle import rdm as O4
from oracle.fci import fci_energy


def _det_state(N, occ):
    """Fock basis vector of the determinant with spin-orbital occupations occ[(i, s)]."""
    # site state index: 0 empty, 1 up, 2 down, 3 up+down
    idx = 0
    for i in range(N):
        st = occ[i][0] * 1 + occ[i][1] * 2
        st = {0: 0, 1: 1, 2: 2, 3: 3}[st]
        idx = idx * 4 + st
    phi = np.zeros(4 ** N)
    phi[idx] = 1.0
    return phi


@pytest.mark.parametrize("occ", [[(1, 1), (1, 0), (0, 0)], [(0, 1), (1, 1), (1, 0), (0, 0)],
                                 [(1, 1), (1, 1), (0, 1)]])
def test_wick_on_determinants(occ):
    N = len(occ)
    phi = _det_state(N, occ)
    g = O4.rdm1(phi, N)
    G = O4.rdm2(phi, N)
    n = np.array(occ, dtype=float)          # n[i, s]
    Ni = n.sum(axis=1)
    assert np.allclose(g, np.diag(Ni), atol=0, rtol=0)
    ref = np.zeros((N, N, N, N))
    for i in range(N):
        for k in range(N):
            ref[i, i, k, k] += Ni[i] * Ni[k]
            ref[i, k, k, i] -= n[i] @ n[k]
    assert np.array_equal(G, ref)


def _random_state(N, n_elec, two_sz, seed):
    rng = np.random.default_rng(seed)
    idx = O2.sector_indices(N, n_elec, two_sz)
    phi = np.zeros(4 ** N)
    phi[idx] = rng.standard_normal(idx.size)
    return phi / np.linalg.norm(phi)


@pytest.mark.parametrize("N,n,s2", [(3, 3, 1), (4, 4, 0), (4, 3, -1)])
def test_traces_and_symmetries(N, n, s2):
    phi = _random_state(N, n, s2, N + n)
    g = O4.rdm1(phi, N)
    G = O4.rdm2(phi, N)
    assert abs(np.trace(g) - n) < 1e-12
    assert np.allclose(np.einsum("ijkk->ij", G), (n - 1) * g, atol=1e-12)
    assert np.allclose(g, g.T, atol=1e-13)
    assert np.allclose(G, G.transpose(2, 3, 0, 1), atol=1e-13)   # electron exchange
    assert np.allclose(G, G.transpose(1, 0, 3, 2), atol=1e-13)   # real state (hermiticity)
    # Sz: number of up electrons from the spin-resolved trace is not needed; total pairs
    assert abs(np.einsum("iikk->", G) - n * (n - 1)) < 1e-11


@pytest.mark.parametrize("N,n,s2", [(4, 4, 0), (5, 5, 1)])
def test_energy_identity_against_fock_hamiltonian(N, n, s2):
    h, v = synth.integrals(N, 2.0, 70 + N)
    H = O2.fock_hamiltonian(h, v)
    phi = _random_state(N, n, s2, 3)
    e_direct = float(phi @ (H @ phi))
    g = O4.rdm1(phi, N)
    G = O4.rdm2(phi, N)
    assert abs(O4.energy_from_rdms(h, v, g, G) - e_direct) < 1e-11 * max(1.0, abs(e_direct))


def test_ground_state_energy_identity_matches_fci():
    N, n, s2 = 4, 4, 0
    h, v = synth.integrals(N, 2.0, 5)
    H = O2.fock_hamiltonian(h, v)
    idx = O2.sector_indices(N, n, s2)
    w, U = np.linalg.eigh(H[idx][:, idx].toarray())
    phi = np.zeros(4 ** N)
    phi[idx] = U[:, 0]
    e = O4.energy_from_rdms(h, v, O4.rdm1(phi, N), O4.rdm2(phi, N))
    assert abs(e - fci_energy(h, v, n, s2)) < 1e-10


def test_mps_state_matches_fock_heff_embedding():
    N, n, s2, D, k = 6, 6, 0, 12, 2
    h, v = synth.integrals(N, 2.0, 9)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=1)
    F = O2.FockHeff(h, v, bonds, sites, k, n, s2)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=4)[0]
    phi = O4.mps_state(bonds, sites, k, X, n, s2, N)
    assert np.allclose(phi, F._to_fock(X), atol=1e-14)
    # the embedded state has the norm of X (isometric left/right bases)
    assert abs(phi @ phi - sum(np.sum(b * b) for b in X.values())) < 1e-12
