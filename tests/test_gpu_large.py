"""Oracle parity of H_eff*psi on sectors large enough for the full-size
kernel paths (GPU).

Random MPS whose bond dimension sits in the three largest sectors per bond
(synth.random_mps(max_sectors=3)), 13 orbitals, 13 electrons, 2S_z = 1:
  * step (6, 7): left sectors up to 99 states, right sectors up to 41 -- output
    blocks up to 99 x 41 (taller than a 32-row tile: the FP64 tall class,
    several row tiles per block; GEMM2 of the tensor-core kernel runs several
    32-row K steps, GEMM1 several 32-element K chunks);
  * step (4, 5): the mirror shape, right sectors up to 99 (wide blocks).
The FP64 path must match the dense-operator oracle to 1e-12 (relative, and
element-wise against the largest entry).  The tensor-core forms are checked
against the forward error model of a sum of products: every operand and the
intermediate X R^T carry a relative rounding u (split-BF16 x = hi + lo:
u = 2^-16; TF32: u = 2^-11 per rounding, four roundings), so
|Y_tc - Y| <= c u sum_a |L_a| |X| |R_a|^T elementwise; the sum is the
oracle's heff_apply_abs and c = 8 covers the roundings of L, X, R, the
intermediate and the FP32 accumulation.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg as O3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(13, 13, 1, 260, 6, 3), (13, 13, 1, 260, 4, 3)]
U = {1: 4 * 2.0 ** -11, 2: 2.0 ** -16}  # TNS_TF32, TNS_BF16X3
C_MODEL = 8.0


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"N{c[0]}_k{c[4]}")
def case(request):
    from paper_2305_05581_gb300 import Context, blocks_to_vector
    N, n, s2, D, k, ms = request.param
    h, v = synth.integrals(N, 3.0, 2)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=1, max_sectors=ms)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=3)[0]
    heff = O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2)
    ref, ref_abs = heff.apply(X), heff.apply_abs(X)
    ctx = Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    x = torch.tensor(blocks_to_vector(desc, length, X), device="cuda", dtype=torch.float64)
    yield dict(ctx=ctx, k=k, desc=desc, length=length, x=x, ref=ref, ref_abs=ref_abs,
               dims=max(max(m for _, (m, _n) in keys), max(_n for _, (_m, _n) in keys)))
    ctx.close()


def _apply(c, prec):
    y = torch.empty_like(c["x"])
    c["ctx"].heff_apply_ptr(c["k"], c["x"].data_ptr(), y.data_ptr(), 1, prec)
    torch.cuda.synchronize()
    from paper_2305_05581_gb300 import vector_to_blocks
    return vector_to_blocks(c["desc"], y.cpu().numpy())


def test_case_has_large_sectors(case):
    assert case["dims"] >= 90


def test_fp64_matches_oracle_at_size(case):
    from paper_2305_05581_gb300 import TNS_FP64
    got, ref = _apply(case, TNS_FP64), case["ref"]
    num = sum(float(np.sum((got[q] - ref[q]) ** 2)) for q in ref)
    den = sum(float(np.sum(ref[q] ** 2)) for q in ref)
    assert (num / den) ** 0.5 < 1e-12
    ymax = max(float(np.max(np.abs(ref[q]))) for q in ref)
    assert max(float(np.max(np.abs(got[q] - ref[q]))) for q in ref) < 1e-12 * ymax


@pytest.mark.parametrize("prec", [1, 2], ids=["tf32", "bf16x3"])
def test_tensor_cores_within_error_model(case, prec):
    got, ref, ra = _apply(case, prec), case["ref"], case["ref_abs"]
    worst = 0.0
    for q in ref:
        err = np.abs(got[q] - ref[q])
        bound = C_MODEL * U[prec] * ra[q]
        worst = max(worst, float(np.max(err / np.maximum(bound, 1e-300))))
        assert np.all(err <= bound + 1e-300), f"block {q}: error above the model bound"
    # the bound is not vacuous: the error uses a visible part of it
    assert worst > 1e-3
