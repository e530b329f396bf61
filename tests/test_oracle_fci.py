"""Pins of O1 (full CI of Eq. (1)) against closed forms and special cases."""
import math

import numpy as np
import pytest

import synth
from oracle.fci import fci_energy, fci_hamiltonian


def test_integral_symmetry():
    h, v = synth.integrals(6, 3.0, 0)
    assert np.array_equal(h, h.T)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.array_equal(v, np.transpose(v, perm))
    # the diagonal Coulomb shift of the recipe
    h2, v2 = synth.integrals(6, 3.0, 0, diag_coulomb=0.0)
    d = v - v2
    expect = np.zeros_like(d)
    for i in range(6):
        expect[i, i, i, i] = 1.0
    assert np.allclose(d, expect)


def test_one_electron_is_eig_h():
    h, v = synth.integrals(5, 2.0, 7)
    e = fci_energy(h, v, 1, 1)
    assert abs(e - np.linalg.eigvalsh(h)[0]) < 1e-12


def test_noninteracting_aufbau():
    h, _ = synth.integrals(6, 3.0, 3)
    v = np.zeros((6,) * 4)
    eps = np.linalg.eigvalsh(h)
    for n_elec, two_sz in [(4, 0), (5, 1), (3, -1), (6, 2)]:
        na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
        assert abs(fci_energy(h, v, n_elec, two_sz) - (eps[:na].sum() + eps[:nb].sum())) < 1e-11


def test_hubbard_dimer_closed_form():
    # two sites, hopping -t, on-site U: singlet ground state (U - sqrt(U^2+16t^2))/2
    for t, U in [(1.0, 4.0), (0.7, 1.3), (1.0, 0.0)]:
        h = np.array([[0.0, -t], [-t, 0.0]])
        v = np.zeros((2, 2, 2, 2))
        v[0, 0, 0, 0] = v[1, 1, 1, 1] = U
        e = fci_energy(h, v, 2, 0)
        assert abs(e - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def test_triplet_coulomb_minus_exchange():
    # two up electrons in two orbitals: one determinant, E = h00 + h11 + J - K
    h, v = synth.integrals(2, 1.5, 11)
    e = fci_energy(h, v, 2, 2)
    J, K = v[0, 0, 1, 1], v[0, 1, 1, 0]
    assert abs(e - (h[0, 0] + h[1, 1] + J - K)) < 1e-12


def test_single_determinant_energy_closed_form():
    # diagonal element of a closed-shell determinant: 2 sum h_ii + sum (2J_ij - K_ij)
    h, v = synth.integrals(4, 2.0, 5)
    H = fci_hamiltonian(h, v, 2, 2).toarray()
    occ = [0, 1]  # first alpha and beta strings occupy orbitals 0,1
    e = sum(2 * h[i, i] for i in occ) + sum(2 * v[i, i, j, j] - v[i, j, j, i] for i in occ for j in occ)
    assert abs(H[0, 0] - e) < 1e-12


def test_fci_dimension_and_hermitian():
    h, v = synth.integrals(8, 3.0, 0)
    H = fci_hamiltonian(h, v, 4, 4)
    assert H.shape == (4900, 4900)
    assert abs(H - H.T).max() < 1e-13
