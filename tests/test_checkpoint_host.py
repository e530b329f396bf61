"""Checkpoint / restart of the engine's state (integrals, MPS, sweep
position) on the test-only plain-loop build: a restored context reproduces
the MPS and H_eff*psi bitwise, and damaged files are refused before the
context changes."""
import os
import subprocess

import numpy as np
import pytest

import synth
from paper_2305_05581_gb300.binding import Context, TnsError

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "_build", "libtns_hostcheck.so")
N, NE, S2, D, K = 7, 6, 2, 24, 3


@pytest.fixture(scope="module")
def hostlib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    src = [os.path.join(ROOT, "tests", "hostcheck", "hostcheck.cpp"),
           os.path.join(ROOT, "paper_2305_05581_gb300", "csrc", "engine.cpp")]
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", LIB] + src)
    return LIB


def _product(ctx):
    ctx.build_env(K)
    desc, length = ctx.psi_layout(K)
    x = np.random.default_rng(5).standard_normal(length)
    y = np.zeros(length)
    ctx.heff_apply_ptr(K, x.ctypes.data, y.ctypes.data)
    return y


def test_checkpoint_round_trip(hostlib, tmp_path):
    h, v = synth.integrals(N, 2.5, 31)
    bonds, sites = synth.random_mps(N, NE, S2, D, center=K, seed=32)
    a = Context(path=hostlib, prefix="tnshc_")
    a.load_integrals(h, v, e_core=1.25)
    a.mps_import(N, NE, S2, D, bonds, sites)
    ya = _product(a)
    path = str(tmp_path / "state.ckpt")
    a.checkpoint_save(path, site=K, left_to_right=False)
    b = Context(path=hostlib, prefix="tnshc_")
    assert b.checkpoint_load(path) == (K, False)
    for bb in range(N + 1):
        assert b.get_bond(bb) == a.get_bond(bb)
    for s in range(N):
        assert np.array_equal(b.get_site(s), a.get_site(s))
    assert np.array_equal(_product(b), ya)
    # a damaged file is refused and the context keeps its state
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(TnsError) as e:
        b.checkpoint_load(bad)
    assert "TNS_ERR_ARG" in str(e.value)
    open(bad, "wb").write(open(path, "rb").read()[:-100])
    with pytest.raises(TnsError):
        b.checkpoint_load(bad)
    assert np.array_equal(_product(b), ya)
