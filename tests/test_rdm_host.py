"""Integral gradients of the differentiation form (tns_rdm) through the
host-logic check library: dE/dh and 2 dE/dv of <psi|H_eff|psi>/<psi|psi> with
the MPS fixed equal the oracle's brute-force 1-RDM and (orbit-averaged) 2-RDM
of the embedded Fock-space state (O4), for random MPS and random psi."""
import os
import subprocess

import numpy as np
import pytest

import synth
from oracle import rdm as O4
from paper_2305_05581_gb300.binding import Context, blocks_to_vector

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "_build", "libtns_hostcheck.so")


@pytest.fixture(scope="module")
def hostlib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    src = [os.path.join(ROOT, "tests", "hostcheck", "hostcheck.cpp"),
           os.path.join(ROOT, "paper_2305_05581_gb300", "csrc", "engine.cpp")]
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", LIB] + src)
    return LIB


def orbit_average(G):
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0),
             (3, 2, 1, 0)]
    N = G.shape[0]
    out = np.zeros_like(G)
    for idx in np.ndindex(*G.shape):
        imgs = {tuple(idx[p] for p in perm) for perm in perms}
        out[idx] = np.mean([G[i] for i in imgs])
    return out


@pytest.mark.parametrize("N,n,s2,D,k", [(4, 4, 0, 16, 1), (5, 5, 1, 8, 1), (5, 4, 0, 12, 2), (6, 6, 0, 12, 2)])
def test_rdm_matches_oracle(hostlib, N, n, s2, D, k):
    h, v = synth.integrals(N, 2.0, 800 + N + k)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k + 11)
    ctx = Context(path=hostlib, prefix="tnshc_")
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=3)[0]
    x = blocks_to_vector(desc, length, X)
    gamma, Gamma = ctx.rdm_ptr(k, x.ctypes.data, N)
    phi = O4.mps_state(bonds, sites, k, X, n, s2, N)
    n2 = float(phi @ phi)
    g_ref = O4.rdm1(phi, N) / n2
    G_ref = orbit_average(O4.rdm2(phi, N) / n2)
    assert np.max(np.abs(gamma - g_ref)) < 1e-10
    assert np.max(np.abs(Gamma - G_ref)) < 1e-10
    # the energy identity with the gradients
    e = float(x @ _heff(ctx, k, x, length)) / float(x @ x)
    assert abs(np.sum(h * gamma) + 0.5 * np.sum(v * Gamma) - e) < 1e-10 * max(1.0, abs(e))


def _heff(ctx, k, x, length):
    y = np.zeros(length)
    ctx.heff_apply_ptr(k, x.ctypes.data, y.ctypes.data)
    return y
