"""Host logic of the engine (operator catalogues, partial sums, work lists)
executed by the test-only plain-loop executor and compared with the oracle.

This checks the symbolic layer of the product (engine.cpp) on CPU; the CUDA
kernels that execute the same work lists on the GPU are checked in
test_gpu_*.py.
"""
import os
import subprocess

import numpy as np
import pytest

import synth
from oracle import dmrg as O3
from paper_2305_05581_gb300.binding import Context, blocks_to_vector, vector_to_blocks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "_build", "libtns_hostcheck.so")


@pytest.fixture(scope="module")
def hostlib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    src = [os.path.join(ROOT, "tests", "hostcheck", "hostcheck.cpp"),
           os.path.join(ROOT, "paper_2305_05581_gb300", "csrc", "engine.cpp")]
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", LIB] + src)
    return LIB


def _ctx(hostlib):
    return Context(path=hostlib, prefix="tnshc_")


def _rel(a, b):
    num = sum(np.sum((a[k] - b[k]) ** 2) for k in b)
    den = sum(np.sum(b[k] ** 2) for k in b)
    return np.sqrt(num / den)


CASES = [(5, 5, 1, 8, 0), (6, 6, 0, 12, 2), (6, 5, -1, 9, 3), (6, 6, 2, 16, 4), (8, 8, 0, 40, 3),
         (8, 7, 1, 30, 1), (8, 8, 0, 24, 6)]


@pytest.mark.parametrize("N,n,s2,D,k", CASES)
def test_heff_matches_oracle(hostlib, N, n, s2, D, k):
    h, v = synth.integrals(N, 2.0, 100 + N + k)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k + 1)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=3)[0]
    ref = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2).apply(X)
    ctx = _ctx(hostlib)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    assert len(desc) == len(keys)
    x = blocks_to_vector(desc, length, X)
    y = np.zeros(length)
    ctx.heff_apply_ptr(k, x.ctypes.data, y.ctypes.data)
    got = vector_to_blocks(desc, y)
    assert _rel(got, ref) < 1e-12


def test_heff_diag_matches_oracle(hostlib):
    N, n, s2, D, k = 6, 6, 0, 12, 2
    h, v = synth.integrals(N, 2.0, 42)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=7)
    ctx = _ctx(hostlib)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    d = np.zeros(length)
    ctx.heff_diag_ptr(k, d.ctypes.data)
    heff = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
    ref = np.zeros(length)
    for i in range(length):
        e = np.zeros(length)
        e[i] = 1.0
        ref[i] = heff.apply_matrix(heff.to_matrix(vector_to_blocks(desc, e)))[
            np.nonzero(heff.to_matrix(vector_to_blocks(desc, e)))][0]
    assert np.max(np.abs(d - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_layout_and_flops(hostlib):
    N, n, s2, D, k = 8, 8, 0, 40, 3
    h, v = synth.integrals(N, 2.0, 1)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=2)
    ctx = _ctx(hostlib)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    assert length == int(sum(r[6] * r[7] for r in desc))
    offs = desc[:, 8]
    assert np.all(np.diff(offs) > 0)
    f, nprod = ctx.heff_flops(k)
    assert f > 0 and nprod > 0


# edge bonds (k = 0: empty left block; k = N-2: empty right block), 2S_z != 0,
# identity factors (the enlarged blocks of the empty blocks are identities)
FLOP_CASES = [(3, 3, 1, 4, 0), (4, 4, 0, 16, 0), (4, 4, 0, 16, 1), (5, 5, 1, 8, 0), (6, 6, 0, 12, 2),
              (6, 5, -1, 9, 3), (6, 6, 2, 16, 4), (8, 8, 0, 40, 3), (8, 7, 1, 30, 1)]


@pytest.mark.parametrize("N,n,s2,D,k", FLOP_CASES)
def test_heff_flops_equal_oracle(hostlib, N, n, s2, D, k):
    """The engine's useful-flop count (structural work list plus the identically
    zero operator blocks it detects) equals the oracle's count over its dense
    operators exactly: every throughput figure divides this number."""
    h, v = synth.integrals(N, 2.0, 100 + N + k)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k + 1)
    ctx = _ctx(hostlib)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    f, nprod = ctx.heff_flops(k)
    ref = O3.useful_flops(O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2))
    assert f == ref


def test_bad_arguments(hostlib):
    from paper_2305_05581_gb300.binding import TnsError
    ctx = _ctx(hostlib)
    h, v = synth.integrals(4, 2.0, 1)
    v2 = v.copy()
    v2[0, 1, 2, 3] += 1e-3
    with pytest.raises(TnsError) as e:
        ctx.load_integrals(h, v2)
    assert "TNS_ERR_ARG" in str(e.value)
    with pytest.raises(TnsError):
        ctx.build_env(0)   # no integrals / MPS yet
