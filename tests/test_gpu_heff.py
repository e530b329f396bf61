"""GPU parity of the FP64 path (CUDA kernels through the C ABI) against the oracle."""
import os

import numpy as np
import pytest

import synth
from oracle import dmrg as O3
from oracle.fci import fci_energy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_05581_gb300 import (Context, TNS_FP64, blocks_to_vector,  # noqa: E402
                                    vector_to_blocks, DEFAULT_LIB)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(DEFAULT_LIB):
        from paper_2305_05581_gb300 import build as b
        b.build()


def _ctx(fixed_schedule=False):
    """Context on the torch stream; fixed_schedule turns the online schedule
    autotuner off (one schedule throughout: bitwise-reproducible results)."""
    if not fixed_schedule:
        return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    os.environ["TNS_AUTOTUNE"] = "0"
    try:
        return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        del os.environ["TNS_AUTOTUNE"]


def _rel(a, b):
    num = sum(np.sum((a[k] - b[k]) ** 2) for k in b)
    den = sum(np.sum(b[k] ** 2) for k in b)
    return float(np.sqrt(num / den))


def _gpu_heff(ctx, k, X, desc, length, nvec=1, precision=TNS_FP64):
    x = torch.tensor(blocks_to_vector(desc, length, X), device="cuda", dtype=torch.float64)
    y = torch.empty_like(x)
    ctx.heff_apply_ptr(k, x.data_ptr(), y.data_ptr(), nvec, precision)
    torch.cuda.synchronize()
    return vector_to_blocks(desc, y.cpu().numpy())


CASES = [(5, 5, 1, 8, 0), (6, 6, 0, 12, 2), (6, 5, -1, 9, 3), (6, 6, 2, 16, 4), (8, 8, 0, 40, 3),
         (8, 7, 1, 30, 1), (8, 8, 0, 256, 3), (8, 8, 0, 24, 6), (10, 10, 0, 120, 4), (10, 9, 1, 90, 7)]


@pytest.mark.parametrize("N,n,s2,D,k", CASES)
def test_heff_fp64_matches_oracle(N, n, s2, D, k):
    """Element-wise H_eff*psi vs the dense-operator oracle, relative error <= 1e-12."""
    h, v = synth.integrals(N, 3.0, 200 + N + k)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k + 5)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=11)[0]
    ref = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2).apply(X)
    ctx = _ctx()
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    got = _gpu_heff(ctx, k, X, desc, length)
    assert _rel(got, ref) < 1e-12


def test_heff_diag_matches_oracle():
    N, n, s2, D, k = 6, 6, 0, 12, 2
    h, v = synth.integrals(N, 2.0, 42)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=7)
    ctx = _ctx()
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    d = torch.zeros(length, device="cuda", dtype=torch.float64)
    ctx.heff_diag_ptr(k, d.data_ptr())
    torch.cuda.synchronize()
    heff = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
    ref = np.zeros(length)
    for i in range(length):
        e = np.zeros(length)
        e[i] = 1.0
        M = heff.to_matrix(vector_to_blocks(desc, e))
        ref[i] = heff.apply_matrix(M)[np.nonzero(M)][0]
    assert np.max(np.abs(d.cpu().numpy() - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_multivector_and_determinism():
    N, n, s2, D, k = 8, 8, 0, 60, 3
    h, v = synth.integrals(N, 3.0, 5)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=3)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    Xs = synth.random_psi(keys, seed=4, nvec=3)
    ctx = _ctx(fixed_schedule=True)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    x = torch.tensor(np.concatenate([blocks_to_vector(desc, length, X) for X in Xs]), device="cuda")
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    ctx.heff_apply_ptr(k, x.data_ptr(), y1.data_ptr(), 3)
    ctx.heff_apply_ptr(k, x.data_ptr(), y2.data_ptr(), 3)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)  # fixed-order accumulation: bitwise reproducible
    heff = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
    for j in range(3):
        got = vector_to_blocks(desc, y1[j * length:(j + 1) * length].cpu().numpy())
        assert _rel(got, heff.apply(Xs[j])) < 1e-12


@pytest.mark.parametrize("wl", ["n24"])
def test_full_size_hermitian(wl):
    """Workload size (24 orbitals, D=512, middle bond): <x,Hy> = <Hx,y> and
    H_eff*psi is linear; properties that hold at any size."""
    c = synth.WORKLOADS[wl]
    N, n, s2, D = c["N"], c["n_elec"], c["two_sz"], c["D"]
    k = N // 2 - 1
    h, v = synth.integrals(N, c["lam"], c["seed"])
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=c["seed"])
    ctx = _ctx()
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(length, device="cuda", dtype=torch.float64, generator=g)
    y = torch.randn(length, device="cuda", dtype=torch.float64, generator=g)
    Hx = torch.empty_like(x)
    Hy = torch.empty_like(x)
    ctx.heff_apply_ptr(k, x.data_ptr(), Hx.data_ptr())
    ctx.heff_apply_ptr(k, y.data_ptr(), Hy.data_ptr())
    torch.cuda.synchronize()
    a = float(torch.dot(x, Hy))
    b = float(torch.dot(Hx, y))
    scale = float(torch.linalg.norm(x) * torch.linalg.norm(Hy))
    assert abs(a - b) < 1e-12 * scale
    z = 0.3 * x - 1.7 * y
    Hz = torch.empty_like(z)
    ctx.heff_apply_ptr(k, z.data_ptr(), Hz.data_ptr())
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(Hz - (0.3 * Hx - 1.7 * Hy))) < 1e-12 * float(torch.linalg.norm(Hz))


def test_davidson_exact_space_is_fci():
    """At full bond dimension the middle-bond H_eff spans the sector: lowest
    eigenvalue from the device Davidson = FCI (O1) within 1e-10 Ha."""
    N, n, s2 = 8, 8, 0
    h, v = synth.integrals(N, 3.0, 0)
    k = 3
    bonds, sites = synth.random_mps(N, n, s2, 10 ** 6, center=k, seed=1)
    ctx = _ctx()
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, 10 ** 6, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    x = torch.zeros(length, device="cuda", dtype=torch.float64)
    e, its, ok = ctx.davidson_ptr(k, x.data_ptr(), tol=1e-9, max_iter=400)
    assert ok
    assert abs(e - fci_energy(h, v, n, s2)) < 1e-10


def test_sweep_reaches_fci_n8():
    """8 orbitals, 8 electrons, D=256 (exact): four sweeps reach FCI to 1e-10 Ha."""
    c = synth.WORKLOADS["n8"]
    h, v = synth.integrals(c["N"], c["lam"], c["seed"])
    ctx = _ctx()
    ctx.load_integrals(h, v)
    ctx.mps_init(c["N"], c["n_elec"], c["two_sz"], c["D"], seed=1)
    e, st = ctx.sweep(4, c["D"], tol=1e-9, max_iter=200)
    assert abs(e - fci_energy(h, v, c["n_elec"], c["two_sz"])) < 1e-10
    assert st.steps == 4 * (2 * c["N"] - 4)
