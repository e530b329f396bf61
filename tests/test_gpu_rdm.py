"""Differentiation form on the GPU: integral gradients (tns_rdm) against the
oracle's brute-force RDMs, against central finite differences of the energy
with the MPS fixed, and against the trace and energy identities at the
30-orbital workload."""
import os

import numpy as np
import pytest

import synth
from oracle import rdm as O4

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_05581_gb300 import Context, DEFAULT_LIB, TNS_FP64, blocks_to_vector  # noqa: E402

PERMS = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0),
         (3, 2, 1, 0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(DEFAULT_LIB):
        from paper_2305_05581_gb300 import build as b
        b.build()


def _setup(N, n, s2, D, k, seed, lam=3.0):
    h, v = synth.integrals(N, lam, seed)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=seed + 1)
    ctx = Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    return ctx, h, v, bonds, sites


def _energy(ctx, k, x):
    y = torch.empty_like(x)
    ctx.heff_apply_ptr(k, x.data_ptr(), y.data_ptr(), 1, TNS_FP64)
    torch.cuda.synchronize()
    return float(torch.dot(x, y) / torch.dot(x, x))


def test_rdm_matches_oracle_n8():
    N, n, s2, D, k = 8, 8, 0, 40, 3
    ctx, h, v, bonds, sites = _setup(N, n, s2, D, k, 61)
    desc, length = ctx.psi_layout(k)
    X = synth.random_psi(synth.psi_keys(bonds, N, n, s2, k), seed=9)[0]
    x = torch.tensor(blocks_to_vector(desc, length, X), device="cuda")
    gamma, Gamma = ctx.rdm_ptr(k, x.data_ptr(), N)
    phi = O4.mps_state(bonds, sites, k, X, n, s2, N)
    n2 = float(phi @ phi)
    g_ref = O4.rdm1(phi, N) / n2
    G = O4.rdm2(phi, N) / n2
    assert np.max(np.abs(gamma - g_ref)) < 1e-10
    # Gamma holds orbit averages: its sum over an orbit equals the oracle's
    for idx in [(0, 1, 2, 3), (1, 1, 2, 2), (3, 0, 3, 0), (2, 5, 7, 4), (6, 6, 6, 6), (7, 2, 2, 7)]:
        imgs = {tuple(idx[p] for p in perm) for perm in PERMS}
        assert abs(sum(Gamma[i] for i in imgs) - sum(G[i] for i in imgs)) < 1e-10
    assert abs(np.trace(gamma) - n) < 1e-10
    e = _energy(ctx, k, x)
    assert abs(e - (np.sum(h * gamma) + 0.5 * np.sum(v * Gamma))) < 1e-10 * abs(e)


def test_rdm_finite_differences():
    """Central differences (step 1e-5) of E(theta) = <psi|H_eff(theta)|psi>/<psi|psi>, the MPS
    fixed, along symmetric perturbations of h and v: relative error <= 1e-6."""
    N, n, s2, D, k = 12, 12, 0, 60, 5
    ctx, h, v, bonds, sites = _setup(N, n, s2, D, k, 71, lam=5.0)
    desc, length = ctx.psi_layout(k)
    g = torch.Generator(device="cuda").manual_seed(4)
    x = torch.randn(length, device="cuda", dtype=torch.float64, generator=g)
    gamma, Gamma = ctx.rdm_ptr(k, x.data_ptr(), N)
    d = 1e-5

    def energy_at(hh, vv):
        ctx.load_integrals(hh, vv)
        ctx.mps_import(N, n, s2, D, bonds, sites)
        ctx.build_env(k)
        return _energy(ctx, k, x)

    for (i, j) in [(0, 0), (2, 7), (5, 6), (11, 1)]:
        e = np.zeros((N, N))
        e[i, j] += 1.0
        if i != j:
            e[j, i] += 1.0
        fd = (energy_at(h + d * e, v) - energy_at(h - d * e, v)) / (2 * d)
        an = float(np.sum(e * gamma))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (i, j, fd, an)
    for idx in [(0, 0, 0, 0), (1, 2, 3, 4), (5, 5, 6, 6), (2, 9, 2, 9), (7, 1, 10, 3)]:
        imgs = {tuple(idx[p] for p in perm) for perm in PERMS}
        e = np.zeros((N, N, N, N))
        for im in imgs:
            e[im] = 1.0
        fd = (energy_at(h, v + d * e) - energy_at(h, v - d * e)) / (2 * d)
        an = 0.5 * float(np.sum(e * Gamma))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (idx, fd, an)


def test_rdm_identities_n30():
    """30 orbitals, 30 electrons (the differentiation-form workload's shape; random
    MPS at D=128): particle number, pair count and energy identities."""
    c = synth.WORKLOADS["n30"]
    N, n, s2 = c["N"], c["n_elec"], c["two_sz"]
    D, k = 128, N // 2 - 1
    ctx, h, v, bonds, sites = _setup(N, n, s2, D, k, c["seed"], lam=c["lam"])
    desc, length = ctx.psi_layout(k)
    g = torch.Generator(device="cuda").manual_seed(2)
    x = torch.randn(length, device="cuda", dtype=torch.float64, generator=g)
    gamma, Gamma = ctx.rdm_ptr(k, x.data_ptr(), N)
    assert abs(np.trace(gamma) - n) < 1e-9 * n
    assert abs(np.einsum("iikk->", Gamma) - n * (n - 1)) < 1e-8 * n * n
    assert np.max(np.abs(gamma - gamma.T)) < 1e-12
    e = _energy(ctx, k, x)
    assert abs(e - (np.sum(h * gamma) + 0.5 * np.sum(v * Gamma))) < 1e-9 * abs(e)


def test_rdm_finite_differences_n30_d512():
    """The differentiation-form workload (30 orbitals, 30 electrons, D = 512, random
    MPS at the middle bond): dE/dh and dE/dv through the torch.autograd.Function
    over the library (tns_rdm in backward) against central differences (step
    1e-5) of E(theta) = <psi|H_eff(theta)|psi>/<psi|psi>, the MPS fixed, on two
    entries of h and two orbits of (ij|kl): relative error <= 1e-6."""
    from paper_2305_05581_gb300.autograd import integral_energy
    c = synth.WORKLOADS["n30"]
    N, n, s2, D = c["N"], c["n_elec"], c["two_sz"], c["D"]
    k = N // 2 - 1
    ctx, h, v, bonds, sites = _setup(N, n, s2, D, k, c["seed"], lam=c["lam"])
    desc, length = ctx.psi_layout(k)
    g = torch.Generator(device="cuda").manual_seed(6)
    x = torch.randn(length, device="cuda", dtype=torch.float64, generator=g)
    ht = torch.tensor(h, requires_grad=True)
    vt = torch.tensor(v, requires_grad=True)
    e = integral_energy(ht, vt, x, ctx, k)
    gh, gv = torch.autograd.grad(e, (ht, vt))
    gh, gv = gh.numpy(), gv.numpy()
    d = 1e-5

    def energy_at(hh, vv):
        ctx.load_integrals(hh, vv)
        ctx.build_env(k)
        return _energy(ctx, k, x)

    for (i, j) in [(3, 3), (14, 16)]:
        p = np.zeros((N, N))
        p[i, j] += 1.0
        if i != j:
            p[j, i] += 1.0
        fd = (energy_at(h + d * p, v) - energy_at(h - d * p, v)) / (2 * d)
        an = float(np.sum(p * gh))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (i, j, fd, an)
    for idx in [(14, 14, 15, 15), (13, 16, 14, 15)]:
        imgs = {tuple(idx[q] for q in perm) for perm in PERMS}
        p = np.zeros((N, N, N, N))
        for im in imgs:
            p[im] = 1.0
        fd = (energy_at(h, v + d * p) - energy_at(h, v - d * p)) / (2 * d)
        an = float(np.sum(p * gv))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (idx, fd, an)
