"""Adjoint of the grouped triple product (differentiation form), host logic:
gradients of <Ybar, H_eff X> with respect to X and to every element of the
left/right operator arenas, checked by central finite differences through the
test-only plain-loop executor of the same work lists."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth
from paper_2305_05581_gb300.binding import Context

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "_build", "libtns_hostcheck.so")


@pytest.fixture(scope="module")
def hostlib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    src = [os.path.join(ROOT, "tests", "hostcheck", "hostcheck.cpp"),
           os.path.join(ROOT, "paper_2305_05581_gb300", "csrc", "engine.cpp")]
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", LIB] + src)
    return LIB


def _arena(ctx, k, side):
    p, n = ctx.env_arena(k, side)
    return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_double)), shape=(n,))


@pytest.mark.parametrize("N,n,s2,D,k", [(5, 5, 1, 8, 1), (6, 6, 0, 12, 2), (6, 5, -1, 9, 3)])
def test_adjoint_matches_finite_differences(hostlib, N, n, s2, D, k):
    h, v = synth.integrals(N, 2.0, 500 + N + k)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k + 3)
    ctx = Context(path=hostlib, prefix="tnshc_")
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    _, length = ctx.psi_layout(k)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(length)
    yb = rng.standard_normal(length)
    L = _arena(ctx, k, 0)
    R = _arena(ctx, k, 1)
    xb = np.zeros(length)
    lb = np.zeros(L.size)
    rb = np.zeros(R.size)
    ctx.heff_adjoint_ptr(k, x.ctypes.data, yb.ctypes.data, xb.ctypes.data, lb.ctypes.data, rb.ctypes.data)

    def energy():
        y = np.zeros(length)
        ctx.heff_apply_ptr(k, x.ctypes.data, y.ctypes.data)
        return float(yb @ y)

    # X: H_eff is symmetric, so Xbar = H_eff Ybar
    hy = np.zeros(length)
    ctx.heff_apply_ptr(k, yb.ctypes.data, hy.ctypes.data)
    assert np.max(np.abs(xb - hy)) < 1e-10 * np.max(np.abs(hy))
    # arenas: central differences on sampled entries (linear in each entry)
    for arena, grad in ((L, lb), (R, rb)):
        nz = np.nonzero(grad)[0]
        picks = list(rng.choice(nz, size=min(12, nz.size), replace=False)) if nz.size else []
        picks += list(rng.choice(arena.size, size=min(4, arena.size), replace=False))
        scale = max(1.0, float(np.max(np.abs(grad))))
        for e in picks:
            old = arena[e]
            d = 1e-5
            arena[e] = old + d
            ctx.build_env(k)
            ep = energy()
            arena[e] = old - d
            ctx.build_env(k)
            em = energy()
            arena[e] = old
            ctx.build_env(k)
            fd = (ep - em) / (2 * d)
            assert abs(fd - grad[e]) <= 1e-6 * scale, (e, fd, grad[e])
