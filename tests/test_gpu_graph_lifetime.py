"""CUDA graphs of a work list hold the addresses of the buffers they read and
write (operand images, partial tiles).  A product with more vectors than
before grows those buffers; the graphs captured with the smaller ones must go
with them.  Sequence per precision on one context: one-vector products until
a graph has been captured and replayed, a four-vector product (the buffers
grow), then one-vector products again (a new graph): every result equals the
oracle, and the one-vector results before and after are identical."""
import os

import numpy as np
import pytest

import synth
from oracle import dmrg as O3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-3, 2: 2e-4}


@pytest.mark.parametrize("prec", [2, 1, 0], ids=["bf16x3", "tf32", "fp64"])
def test_graphs_follow_buffer_growth(prec):
    from paper_2305_05581_gb300 import Context, blocks_to_vector
    N, n, s2, D, k = 10, 10, 0, 140, 4
    h, v = synth.integrals(N, 3.0, 91)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=92)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    Xs = synth.random_psi(keys, seed=93, nvec=4)
    os.environ["TNS_TC_VARIANT"] = "1"  # reduced precision: a fixed schedule, graphs from the first product
    try:
        ctx = Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        del os.environ["TNS_TC_VARIANT"]
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    dense = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
    ref = np.concatenate([blocks_to_vector(desc, length, dense.apply(X)) for X in Xs])
    x = torch.tensor(np.concatenate([blocks_to_vector(desc, length, X) for X in Xs]), device="cuda")
    y1 = torch.empty(length, device="cuda", dtype=torch.float64)
    y4 = torch.empty(4 * length, device="cuda", dtype=torch.float64)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    # FP64 tunes its schedule over the first 9 products, then captures
    for _ in range(12):
        ctx.heff_apply_ptr(k, x.data_ptr(), y1.data_ptr(), 1, prec)
    torch.cuda.synchronize()
    before = y1.cpu().numpy()
    assert rel(before, ref[:length]) < TOL[prec]
    for _ in range(12):
        ctx.heff_apply_ptr(k, x.data_ptr(), y4.data_ptr(), 4, prec)
    torch.cuda.synchronize()
    assert rel(y4.cpu().numpy(), ref) < TOL[prec]
    for _ in range(3):
        y1.fill_(0.0)
        ctx.heff_apply_ptr(k, x.data_ptr(), y1.data_ptr(), 1, prec)
    torch.cuda.synchronize()
    after = y1.cpu().numpy()
    assert np.array_equal(after, before)
    ctx.close()
