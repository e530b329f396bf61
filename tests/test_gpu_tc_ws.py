"""The persistent warp-specialised tensor-core kernel (schedule variant 3 of
the autotuner, forced here with TNS_TC_VARIANT) against the oracle and
against the one-CTA-per-piece kernel (variant 1): split-BF16 and TF32, one
and four vectors, small and large sectors."""
import os

import numpy as np
import pytest

import synth
from oracle import dmrg as O3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {1: 1e-3, 2: 2e-4}  # TNS_TF32, TNS_BF16X3 (relative 2-norm, as in test_gpu_tc.py)


def _ctx(variant):
    from paper_2305_05581_gb300 import Context
    os.environ["TNS_TC_VARIANT"] = str(variant)
    try:
        return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        del os.environ["TNS_TC_VARIANT"]


@pytest.mark.parametrize("prec", [2, 1], ids=["bf16x3", "tf32"])
@pytest.mark.parametrize("N,n,s2,D,k,ms", [(6, 6, 0, 12, 2, 0), (8, 7, 1, 60, 3, 0), (10, 10, 0, 140, 4, 0),
                                           (13, 13, 1, 260, 6, 3)])
def test_ws_kernel_matches_oracle_and_classic(prec, N, n, s2, D, k, ms):
    from paper_2305_05581_gb300 import blocks_to_vector
    h, v = synth.integrals(N, 3.0, 40 + N + k)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=41 + k, max_sectors=ms)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    Xs = synth.random_psi(keys, seed=42, nvec=4)
    ref = [O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2).apply(X) for X in Xs[:1]]
    out = {}
    for variant in (3, 1):
        ctx = _ctx(variant)
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
        out[variant] = (y1.cpu().numpy(), y4.cpu().numpy(), desc, length)
        ctx.close()
    y1, y4, desc, length = out[3]
    r = blocks_to_vector(desc, length, ref[0])
    assert np.linalg.norm(y1 - r) < TOL[prec] * np.linalg.norm(r)
    # four vectors in one launch: vector 0 equals the single-vector product bitwise
    assert np.array_equal(y4[:length], y1)
    c1, c4 = out[1][0], out[1][1]
    assert np.linalg.norm(y4 - c4) < TOL[prec] * np.linalg.norm(c4)
    assert np.linalg.norm(y1 - c1) < TOL[prec] * np.linalg.norm(c1)
