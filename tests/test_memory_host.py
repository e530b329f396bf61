"""Out-of-HBM environments and the step memory plan, on the test-only
plain-loop build of the engine (the allocation accounting of its host
backend stands in for the device).

The operator catalogues of a sweep grow as D^2 N^2 per block; under a device
budget the engine keeps the two catalogues of the current step, moves the
others off the device in stack order (the tree-traversal cache of Alg. 1 on
the block chain): to host memory while the host budget lasts, else it drops
them and rebuilds them by renormalisation when the sweep comes back.  A step
whose memory plan (partial sums, work list, its two catalogues) exceeds the
budget is refused with TNS_ERR_OOM before it allocates anything.
"""
import os
import subprocess

import numpy as np
import pytest

import synth
from paper_2305_05581_gb300.binding import Context, TnsError

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "_build", "libtns_hostcheck.so")

N, NE, S2, D = 10, 10, 0, 60
# a sweep-like visiting order: out to the right end, back to the left end,
# then the middle again (each block is needed again after others were built)
SEQ = [0, 1, 2, 3, 4, 5, 6, 7, 8, 7, 6, 5, 4, 3, 2, 1, 0, 4]


@pytest.fixture(scope="module")
def hostlib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    src = [os.path.join(ROOT, "tests", "hostcheck", "hostcheck.cpp"),
           os.path.join(ROOT, "paper_2305_05581_gb300", "csrc", "engine.cpp")]
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", LIB] + src)
    return LIB


def _state():
    h, v = synth.integrals(N, 2.0, 7)
    bonds, sites = synth.random_mps(N, NE, S2, D, center=4, seed=3)
    return h, v, bonds, sites


def _run(lib, budget, host, seq):
    h, v, bonds, sites = _state()
    ctx = Context(path=lib, prefix="tnshc_")
    ctx.set_memory_budget(budget, host)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, NE, S2, D, bonds, sites)
    ys, need = [], []
    for k in seq:
        ctx.build_env(k)
        _, length = ctx.psi_layout(k)
        x = np.random.default_rng(k).standard_normal(length)
        y = np.zeros(length)
        ctx.heff_apply_ptr(k, x.ctypes.data, y.ctypes.data)
        ys.append(y)
        (_, la), (_, lb) = ctx.env_arena(k, 0), ctx.env_arena(k, 1)
        need.append((la + lb) * 8 + ctx.memory_stats()["last_plan"])
    return ys, need, ctx.memory_stats()


def test_staging_and_dropping_keep_results(hostlib):
    ref, need, st0 = _run(hostlib, 0, 0, SEQ)
    assert st0["staged"] == st0["dropped"] == 0
    budget = int(1.3 * max(need))
    assert budget < st0["device_peak"]  # the budget forces catalogues off the device
    staged, _, st1 = _run(hostlib, budget, 1 << 30, SEQ)
    assert st1["staged"] > 0 and st1["restored"] > 0 and st1["dropped"] == 0
    assert st1["built"] == st0["built"]  # staged catalogues come back, nothing is rebuilt
    assert st1["device_peak"] <= budget
    dropped, _, st2 = _run(hostlib, budget, 0, SEQ)
    assert st2["dropped"] > 0 and st2["staged"] == 0
    assert st2["built"] > st0["built"]  # dropped catalogues are rebuilt
    assert st2["device_peak"] <= budget
    for a, b, c in zip(ref, staged, dropped):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_memory_plan_refuses_before_allocating(hostlib):
    k = 4
    ref, need, _ = _run(hostlib, 0, 0, [k])
    h, v, bonds, sites = _state()
    ctx = Context(path=hostlib, prefix="tnshc_")
    ctx.load_integrals(h, v)
    ctx.mps_import(N, NE, S2, D, bonds, sites)
    ctx.build_env(k - 1)  # every other block exists; step k grows one more
    ctx.set_memory_budget(need[0] - 8, 0)  # one double short of step k's plan
    ctx.memory_stats(reset=True)
    with pytest.raises(TnsError) as e:
        ctx.build_env(k)
    assert "TNS_ERR_OOM" in str(e.value) and "memory plan" in str(e.value)
    st = ctx.memory_stats()
    # the other blocks left the device to make room, then the plan was refused
    assert st["dropped"] > 0 and st["device_used"] <= need[0] - 8
    # the same context recovers once the budget allows the step
    ctx.set_memory_budget(0, 0)
    ctx.build_env(k)
    _, length = ctx.psi_layout(k)
    x = np.random.default_rng(k).standard_normal(length)
    y = np.zeros(length)
    ctx.heff_apply_ptr(k, x.ctypes.data, y.ctypes.data)
    assert np.array_equal(y, ref[0])
