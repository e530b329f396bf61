"""Orbital optimisation from the RDMs (paper_2305_05581_gb300.orbopt), pinned
on CPU against facts that do not come from the code itself:
  * the FCI energy is invariant under orbital rotations (rotated integrals
    give the same FCI energy, oracle O1);
  * at the FCI ground state (all orbitals active) the orbital gradient
    vanishes, with RDMs from the oracle's Fock-space state (O2, O4);
  * away from stationarity the gradient equals central finite differences of
    the fixed-RDM energy functional, evaluated with the oracle's full 2-RDM
    while the gradient uses its eight-fold orbit average (which the engine
    returns);
  * one orbital step lowers the functional.
The GPU test (DMRG with orbital optimisation at a truncated bond dimension)
is in test_gpu_orbopt.py."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import fock as O2
from oracle import rdm as O4
from oracle.fci import fci_energy
from paper_2305_05581_gb300 import orbopt as OO


def _orbit_average(G):
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
             (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    return sum(G.transpose(p) for p in perms) / 8.0


def _random_rotation(N, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    K = rng.standard_normal((N, N)) * scale
    return sla.expm(K - K.T)


def test_fci_energy_invariant_under_rotation():
    N, n, s2 = 4, 4, 0
    h, v = synth.integrals(N, 2.0, 3)
    U = _random_rotation(N, 1)
    h2, v2 = OO.rotate_integrals(h, v, U)
    assert np.allclose(U.T @ U, np.eye(N), atol=1e-13)
    assert abs(fci_energy(h2, v2, n, s2) - fci_energy(h, v, n, s2)) < 1e-10


def _ground_rdms(h, v, N, n, s2):
    H = O2.fock_hamiltonian(h, v)
    idx = O2.sector_indices(N, n, s2)
    Hs = H[np.ix_(idx, idx)].toarray() if hasattr(H, "toarray") else H[np.ix_(idx, idx)]
    w, V = np.linalg.eigh(Hs)
    phi = np.zeros(4 ** N)
    phi[idx] = V[:, 0]
    return w[0], O4.rdm1(phi, N), O4.rdm2(phi, N), phi


def test_gradient_vanishes_at_fci():
    N, n, s2 = 4, 4, 0
    h, v = synth.integrals(N, 2.0, 5)
    e, g, G, _ = _ground_rdms(h, v, N, n, s2)
    assert abs(OO.rdm_energy(h, v, g, G) - e) < 1e-10
    grad = OO.orbital_gradient(h, v, g, _orbit_average(G))
    assert np.max(np.abs(grad)) < 1e-9
    assert np.allclose(grad, -grad.T)


def test_gradient_matches_finite_differences():
    N, n, s2 = 4, 3, 1
    h, v = synth.integrals(N, 2.0, 7)
    # a state that is not stationary: the ground state of other integrals
    hb, vb = synth.integrals(N, 2.0, 8)
    _, g, G, _ = _ground_rdms(hb, vb, N, n, s2)
    grad = OO.orbital_gradient(h, v, g, _orbit_average(G))
    assert np.max(np.abs(grad)) > 1e-2
    d = 1e-5
    for p, q in [(0, 1), (1, 3), (0, 3), (2, 3)]:
        K = np.zeros((N, N))
        K[p, q], K[q, p] = 1.0, -1.0
        ep = OO.rdm_energy(*OO.rotate_integrals(h, v, sla.expm(d * K)), g, G)
        em = OO.rdm_energy(*OO.rotate_integrals(h, v, sla.expm(-d * K)), g, G)
        assert abs((ep - em) / (2 * d) - grad[p, q]) < 1e-6 * max(1.0, abs(grad[p, q]))


def test_orbital_step_lowers_the_functional():
    N, n, s2 = 4, 4, 0
    h, v = synth.integrals(N, 2.0, 11)
    hb, vb = synth.integrals(N, 2.0, 12)
    _, g, G, _ = _ground_rdms(hb, vb, N, n, s2)
    Ga = _orbit_average(G)
    U, h2, v2, de = OO.orbital_step(h, v, g, Ga)
    assert de < 0.0
    assert abs(OO.rdm_energy(h2, v2, g, Ga) - OO.rdm_energy(h, v, g, Ga) - de) < 1e-12
    assert np.allclose(U.T @ U, np.eye(N), atol=1e-12)
