"""Pins of the oracle's useful-flop count (oracle/dmrg.py useful_flops) on
cases small enough to count by hand.

The count follows the reading of the per-product cost of Eq. (2) with the
cheaper chain of Sec. III.B: one product per term of the operator expansion,
per pair of nonzero dot blocks and per X symmetry block in the target sector,
costing min(2mr(n+q), 2qn(m+r)); a factor that is a multiple of the block
identity costs nothing (2mnr, 2qmn, or 2mn when both are).  In both cases
below every block basis has one-state sectors, so each product costs 2 flops
and the count is twice the number of products.
"""
import synth
from oracle import dmrg as O3


def _flops(N, n, s2, D, k, lam, seed):
    h, v = synth.integrals(N, lam, seed)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=1)
    return O3.useful_flops(O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2))


def test_two_orbitals_two_electrons():
    """N = 2, two electrons, S_z = 0, step (0, 1): both blocks are empty, so
    every operator block is 1 x 1 (a multiple of the identity).  psi blocks
    (s1, s2): (0, ud), (u, d), (d, u), (ud, 0).  Products by term:
      H_LL x 1 and 1 x H_RR: the on-site Hamiltonian is diagonal and zero on
        the empty dot, so s = u, d, ud on the dot it acts on: 3 + 3;
      c+_a S_a + h.c., a in {0u, 0d}: c+_0u maps 0->u, d->ud and S_0u
        (= t c_1u + W n_1d c_1u) maps u->0, ud->d on dot 1: X in {(0, ud), (d, u)}
        for the term and {(u, d), (ud, 0)} for its conjugate: 4 per a, 8;
      T_x c_x + h.c., x in {1u, 1d}: T_1u = W c+_0u c+_0d c_0d maps d->ud only,
        so one X block for the term and one for its conjugate: 2 per x, 4;
      A_ab P_ab + h.c., (a, b) = (0u, 0d): 0->ud on dot 0 with ud->0 on dot 1
        and the conjugate: 2;
      B_ab Q_ab over the four (a, b) in {0u, 0d}^2: one X block each: 4.
    24 products x 2 flops = 48."""
    assert _flops(2, 2, 0, 4, 0, 2.0, 5) == 48.0


def test_three_orbitals_one_electron():
    """N = 3, one up electron, step (0, 1): the left block is empty, the right
    block (orbital 2) holds |0> and |u>.  psi blocks (s1, s2, right state):
    (u, 0, 0), (0, u, 0), (0, 0, u).  Products by term:
      H_LL x 1: only the dot-0 state u has a nonzero on-site energy: 1;
      1 x H_RR: from (0, u, 0) to (0, u, 0) (t_11) and (0, 0, u) (t_12), from
        (0, 0, u) to (0, u, 0) (t_21) and (0, 0, u) (t_22); (u, 0, 0) meets the
        vacuum of orbitals 1-2, where H_RR is zero: 4;
      c+_0u S_0u + h.c.: S_0u = t_01 c_1u + t_02 c_2u on one-particle states,
        two X blocks for the term and two for the conjugate; a = 0d finds no
        down electron: 4;
      T_x c_x, A_ab P_ab, B_ab Q_ab: each needs two electrons (or a particle in
        orbitals 1-2 where the left factor acts on dot-0 state u): 0.
    9 products x 2 flops = 18."""
    assert _flops(3, 1, 1, 4, 0, 2.0, 6) == 18.0
