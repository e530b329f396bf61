"""Operator-row split of H_eff*psi across ranks (Sec. "Independent
operational tasks": the operator-table rows are distributed, every rank
accumulates all output blocks of its rows, one sum over the ranks gives
H_eff*psi).  Run here as world_size 2 and 3 gloo process groups on CPU with
the test-only plain-loop build of the engine: every rank builds the same
step, computes its part with tns_heff_apply_part, and an all-reduce of the
partial products must equal the single-rank product and the oracle."""
import os
import socket
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import synth  # noqa: E402
from oracle import dmrg as O3  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "_build", "libtns_hostcheck.so")
CASE = (8, 7, 1, 30, 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    N, n, s2, D, k = CASE
    h, v = synth.integrals(N, 2.0, 21)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=22)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=23)[0]
    return h, v, bonds, sites, X


def _ctx(h, v, bonds, sites):
    from paper_2305_05581_gb300.binding import Context
    N, n, s2, D, k = CASE
    ctx = Context(path=LIB, prefix="tnshc_")
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    return ctx


def _worker(rank, world, port, out):
    from paper_2305_05581_gb300.binding import blocks_to_vector
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h, v, bonds, sites, X = _problem()
    ctx = _ctx(h, v, bonds, sites)
    k = CASE[4]
    desc, length = ctx.psi_layout(k)
    x = blocks_to_vector(desc, length, X)
    y = np.zeros(length)
    ctx.heff_apply_part_ptr(k, x.ctypes.data, y.ctypes.data, rank, world)
    part = torch.from_numpy(y.copy())
    total = part.clone()
    dist.all_reduce(total)  # the one exchange step: a sum of the partial products
    out[rank] = (part.numpy(), total.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def hostlib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    src = [os.path.join(ROOT, "tests", "hostcheck", "hostcheck.cpp"),
           os.path.join(ROOT, "paper_2305_05581_gb300", "csrc", "engine.cpp")]
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", LIB] + src)
    return LIB


@pytest.mark.parametrize("world", [2, 3])
def test_row_split_all_reduce_equals_full_product(hostlib, world):
    from paper_2305_05581_gb300.binding import blocks_to_vector
    h, v, bonds, sites, X = _problem()
    N, n, s2, D, k = CASE
    ctx = _ctx(h, v, bonds, sites)
    desc, length = ctx.psi_layout(k)
    x = blocks_to_vector(desc, length, X)
    full = np.zeros(length)
    ctx.heff_apply_ptr(k, x.ctypes.data, full.ctypes.data)
    ref = blocks_to_vector(desc, length, O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2).apply(X))
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    parts = [out[r][0] for r in range(world)]
    # every rank holds the same reduced product
    for r in range(world):
        assert np.array_equal(out[r][1], out[0][1])
    assert np.linalg.norm(out[0][1] - full) <= 1e-13 * np.linalg.norm(full)
    assert np.linalg.norm(out[0][1] - ref) <= 1e-12 * np.linalg.norm(ref)
    # a real split: every part holds work and none is the whole product
    for p in parts:
        assert np.linalg.norm(p) > 0 and np.linalg.norm(p - full) > 1e-6 * np.linalg.norm(full)
