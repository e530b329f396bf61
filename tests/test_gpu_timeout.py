"""Failure detection of the tensor-core product without a GPU fault: every
wait of k_tasks_tc on an mbarrier is bounded in time; a wait that gives up
sets a device flag, the CTA drains its own copies and MMAs (with the full
bound) and releases its tensor memory, and the host reports the timeout.
Here the bound of the waits inside the product loop is set to zero through
TNS_TC_WAIT_NS (read when a context is created), so the first wait runs out;
the call must fail with TNS_ERR_DEVICE_TIMEOUT naming the wait, and the same
context must then still compute an FP64 product that matches the oracle."""
import os

import numpy as np
import pytest

import synth
from oracle import dmrg as O3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("small", ["0", "32"], ids=["tile-kernel", "small-block-kernel"])
def test_tensor_core_wait_timeout_is_reported_and_context_survives(small):
    from paper_2305_05581_gb300 import Context, TNS_BF16X3, TNS_FP64, blocks_to_vector, vector_to_blocks
    from paper_2305_05581_gb300.binding import TnsError
    N, n, s2, D, k = 6, 6, 0, 16, 2
    h, v = synth.integrals(N, 3.0, 11)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=4)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=5)[0]
    ref = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2).apply(X)
    os.environ["TNS_TC_WAIT_NS"] = "0"
    os.environ["TNS_TC_SMALL"] = small  # every block of this step is small: "0" keeps it on the tile kernel
    try:
        ctx = Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        del os.environ["TNS_TC_WAIT_NS"]
        del os.environ["TNS_TC_SMALL"]
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    x = torch.tensor(blocks_to_vector(desc, length, X), device="cuda", dtype=torch.float64)
    y = torch.full_like(x, 7.0)
    with pytest.raises(TnsError) as e:
        ctx.heff_apply_ptr(k, x.data_ptr(), y.data_ptr(), 1, TNS_BF16X3)
    assert "TNS_ERR_DEVICE_TIMEOUT" in str(e.value) and "wait timed out" in str(e.value)
    torch.cuda.synchronize()  # the device is still usable
    ctx.heff_apply_ptr(k, x.data_ptr(), y.data_ptr(), 1, TNS_FP64)
    torch.cuda.synchronize()
    got = vector_to_blocks(desc, y.cpu().numpy())
    num = sum(float(np.sum((got[q] - ref[q]) ** 2)) for q in ref)
    den = sum(float(np.sum(ref[q] ** 2)) for q in ref)
    assert (num / den) ** 0.5 < 1e-12
    ctx.close()
