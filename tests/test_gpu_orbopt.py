"""DMRG with orbital optimisation from the engine's RDMs (GPU): at a
truncated bond dimension the energy depends on the orbitals, and the orbital
steps lower it towards (never below) the full-CI energy; with all orbitals
active and an exact bond dimension the orbital gradient vanishes (the FCI
energy is invariant under rotations)."""
import numpy as np
import pytest

import synth
from oracle.fci import fci_energy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(h, v, N, n, s2, D):
    from paper_2305_05581_gb300 import Context
    ctx = Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_integrals(h, v)
    ctx.mps_init(N, n, s2, D, seed=1)
    return ctx


def test_orbital_optimisation_lowers_truncated_energy():
    from paper_2305_05581_gb300 import orbopt as OO, TNS_FP64
    c = synth.WORKLOADS["n8"]
    N, n, s2 = c["N"], c["n_elec"], c["two_sz"]
    h, v = synth.integrals(N, c["lam"], c["seed"])
    D = 12
    ctx = _ctx(h, v, N, n, s2, D)
    hist, U, h2, v2 = OO.optimise(ctx, h, v, N, D, macro=4, sweeps=2, precision=TNS_FP64, max_step=0.3)
    e = [x["energy"] for x in hist]
    efci = fci_energy(h, v, n, s2)
    assert e[-1] < e[0] - 1e-6
    assert min(e) > efci - 1e-9
    assert np.allclose(U.T @ U, np.eye(N), atol=1e-10)
    # the rotated problem has the same full-CI energy
    assert abs(fci_energy(h2, v2, n, s2) - efci) < 1e-8
    ctx.close()


def test_orbital_gradient_vanishes_at_exact_bond_dimension():
    from paper_2305_05581_gb300 import orbopt as OO, TNS_FP64
    c = synth.WORKLOADS["n8"]
    N, n, s2, D = c["N"], c["n_elec"], c["two_sz"], c["D"]
    h, v = synth.integrals(N, c["lam"], c["seed"])
    ctx = _ctx(h, v, N, n, s2, D)
    ctx.sweep(3, D, tol=1e-10, max_iter=200, precision=TNS_FP64)
    # a sweep ends at step (1, 2), where the MPS is canonical around the two sites
    e, gamma, Gamma = OO.ground_state_rdms(ctx, 1, N, TNS_FP64, tol=1e-10)
    assert abs(e - fci_energy(h, v, n, s2)) < 1e-9
    assert abs(OO.rdm_energy(h, v, gamma, Gamma) - e) < 1e-8
    assert np.max(np.abs(OO.orbital_gradient(h, v, gamma, Gamma))) < 1e-6
    ctx.close()
