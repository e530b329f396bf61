"""The small-block warp kernel of the tensor-core form (output blocks and X
blocks with every dimension <= 32; mma.sync fragments from bulk-copied
operand images) against the oracle, against the tile kernel on the same
products (TNS_TC_SMALL=0 routes every block to the tile kernel), and in a
work list that mixes both kernels: split-BF16 and TF32, one and four vectors,
every routing limit of blocks to the small kernel."""
import os

import numpy as np
import pytest

import synth
from oracle import dmrg as O3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative 2-norm bounds of one product (those of the tile kernel: the
# operands and the re-split intermediate are rounded the same way)
TOL = {1: 1e-3, 2: 2e-4}  # TNS_TF32, TNS_BF16X3


def _ctx(small=None, variant=None):
    from paper_2305_05581_gb300 import Context
    env = {}
    if small is not None:
        env["TNS_TC_SMALL"] = str(small)
    if variant is not None:
        env["TNS_TC_VARIANT"] = str(variant)
    os.environ.update(env)
    try:
        return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        for k in env:
            del os.environ[k]


def _products(ctx, h, v, N, n, s2, D, bonds, sites, k, Xs, prec):
    from paper_2305_05581_gb300 import blocks_to_vector
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    x = torch.tensor(np.concatenate([blocks_to_vector(desc, length, X) for X in Xs]), device="cuda")
    y1 = torch.empty(length, device="cuda", dtype=torch.float64)
    y4 = torch.empty(4 * length, device="cuda", dtype=torch.float64)
    for _ in range(2):  # second call: steady state (graph replay)
        ctx.heff_apply_ptr(k, x.data_ptr(), y1.data_ptr(), 1, prec)
        ctx.heff_apply_ptr(k, x.data_ptr(), y4.data_ptr(), 4, prec)
    torch.cuda.synchronize()
    return y1.cpu().numpy(), y4.cpu().numpy(), desc, length


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


_ORACLE = {}


def _system(N, n, s2, D, k, seed, ms=0):
    """Integrals, MPS, four input vectors and their oracle products (shared
    by the precisions and routing limits that use the same system)."""
    key = (N, n, s2, D, k, seed, ms)
    if key not in _ORACLE:
        h, v = synth.integrals(N, 3.0, seed)
        bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=seed + 1, max_sectors=ms)
        keys = synth.psi_keys(bonds, N, n, s2, k)
        Xs = synth.random_psi(keys, seed=seed + 2, nvec=4)
        dense = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
        _ORACLE[key] = (h, v, bonds, sites, Xs, [dense.apply(X) for X in Xs])
    return _ORACLE[key]


# sectors of 1..32 states with ragged edges (odd sizes, a single state, full 32)
# (largest sectors at the step: 3, 8, 20, 32, 31, 32 with 18, edge steps)
CASES = [(6, 6, 0, 12, 2, 0), (8, 7, 1, 60, 3, 0), (10, 10, 0, 140, 4, 0), (12, 12, 0, 330, 5, 0),
         (12, 11, 1, 320, 5, 0), (10, 9, 1, 150, 4, 5), (9, 9, 1, 90, 1, 0), (9, 9, 1, 90, 7, 0)]


@pytest.mark.parametrize("prec", [2, 1], ids=["bf16x3", "tf32"])
@pytest.mark.parametrize("N,n,s2,D,k,ms", CASES)
def test_small_kernel_matches_oracle_and_tile_kernel(prec, N, n, s2, D, k, ms):
    from paper_2305_05581_gb300 import blocks_to_vector
    h, v, bonds, sites, Xs, refs = _system(N, n, s2, D, k, 60 + N + k, ms)
    out = {}
    for small in (32, 0):
        ctx = _ctx(small=small)
        out[small] = _products(ctx, h, v, N, n, s2, D, bonds, sites, k, Xs, prec)
        ctx.close()
    y1, y4, desc, length = out[32]
    for i in range(4):
        r = blocks_to_vector(desc, length, refs[i])
        assert _rel(y4[i * length:(i + 1) * length], r) < TOL[prec]
    assert _rel(y1, blocks_to_vector(desc, length, refs[0])) < TOL[prec]
    # vector 0 of the four-vector launch equals the one-vector product bitwise
    assert np.array_equal(y4[:length], y1)
    t1, t4 = out[0][0], out[0][1]
    assert _rel(y1, t1) < TOL[prec] and _rel(y4, t4) < TOL[prec]


@pytest.mark.parametrize("prec", [2, 1], ids=["bf16x3", "tf32"])
@pytest.mark.parametrize("limit", [8, 16, 24])
def test_mixed_work_list_both_kernels(prec, limit):
    """A routing limit below the largest sector sends some output blocks to
    the small kernel and the rest to the tile kernel in the same product."""
    from paper_2305_05581_gb300 import blocks_to_vector
    N, n, s2, D, k = 12, 12, 0, 330, 5
    h, v, bonds, sites, Xs, refs = _system(N, n, s2, D, k, 71)
    dims = [d for _, d in bonds[k]] + [d for _, d in bonds[k + 2]]
    assert min(dims) <= limit < max(dims)
    ctx = _ctx(small=limit)
    y1, y4, desc, length = _products(ctx, h, v, N, n, s2, D, bonds, sites, k, Xs, prec)
    ctx.close()
    r = np.concatenate([blocks_to_vector(desc, length, R) for R in refs])
    assert _rel(y4, r) < TOL[prec]
    assert np.array_equal(y4[:length], y1)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_small_kernel_under_every_schedule_variant(variant):
    """Each autotuner variant splits the small kernel's pieces differently
    (split-K rounds 1, 2, 4; the persistent variant keeps its own split):
    all agree with the oracle."""
    from paper_2305_05581_gb300 import blocks_to_vector
    N, n, s2, D, k = 10, 10, 0, 140, 4
    h, v, bonds, sites, Xs, refs = _system(N, n, s2, D, k, 81)
    ctx = _ctx(variant=variant)
    y1, y4, desc, length = _products(ctx, h, v, N, n, s2, D, bonds, sites, k, Xs, 2)
    ctx.close()
    r = np.concatenate([blocks_to_vector(desc, length, R) for R in refs])
    assert _rel(y4, r) < TOL[2]
