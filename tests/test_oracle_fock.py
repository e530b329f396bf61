"""Pins of O2 (Fock-space H and projected H_eff) against algebra, O1 and exactness."""
import numpy as np
import pytest

import synth
from oracle.fci import fci_energy
from oracle.fock import (FockHeff, cdag_ops, fock_hamiltonian, fock_hamiltonian_direct,
                         sector_ground_energy)


def test_canonical_anticommutators():
    cd = cdag_ops(3)
    n = len(cd)
    I = np.eye(4 ** 3)
    for p in range(n):
        for q in range(n):
            a = (cd[p].T @ cd[q] + cd[q] @ cd[p].T).toarray()
            assert np.allclose(a, I if p == q else 0.0)
            b = (cd[p] @ cd[q] + cd[q] @ cd[p]).toarray()
            assert np.allclose(b, 0.0)


def test_excitation_form_equals_normal_ordered_sum():
    h, v = synth.integrals(3, 2.0, 4)
    A = fock_hamiltonian(h, v)
    B = fock_hamiltonian_direct(h, v)
    assert abs(A - B).max() < 1e-12


@pytest.mark.parametrize("N,n,s2", [(4, 4, 0), (5, 4, 2), (5, 5, 1)])
def test_fock_sector_energy_equals_fci(N, n, s2):
    h, v = synth.integrals(N, 2.5, 20 + N)
    H = fock_hamiltonian(h, v)
    assert abs(sector_ground_energy(H, N, n, s2) - fci_energy(h, v, n, s2)) < 1e-10


def test_projected_heff_exact_at_full_bond_dimension():
    N, n, s2 = 6, 6, 0
    h, v = synth.integrals(N, 3.0, 2)
    k = 2
    bonds, sites = synth.random_mps(N, n, s2, 10 ** 6, center=k, seed=5)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    heff = FockHeff(h, v, bonds, sites, k, n, s2)
    e = heff.ground_energy(keys)
    assert abs(e - fci_energy(h, v, n, s2)) < 1e-10
