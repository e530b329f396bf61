"""FP64 product kernel on a state with large sectors: its tall / wide output
tiles (each product in the cheaper chain order for its tile, four tile
classes on forked streams) against the independent FP64 tensor-path kernel
(DMMA, warp tiles of 32 x 16, its own chain choice), element by element, and
the Hermiticity of H_eff.  A random MPS has only small sectors; one sweep of
the 24-orbital workload at D = 512 grows sectors of up to ~90 states, so the
output blocks run in the tall and wide classes."""
import ctypes as C
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_05581_gb300 import Context, DEFAULT_LIB, TNS_BF16X3, TNS_FP64  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(DEFAULT_LIB):
        from paper_2305_05581_gb300 import build as b
        b.build()


def _ctx(**env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _copy_state(src, dst, N, n, s2, D):
    """The MPS of src into dst through the ABI (define, bonds, site tensors)."""
    dst._check(dst._fn("mps_define")(dst._h, N, n, s2, D))
    for b in range(N + 1):
        bd = src.get_bond(b)
        sec = np.array([x for (q, _) in bd for x in q], dtype=np.int32)
        dims = np.array([d for (_, d) in bd], dtype=np.int32)
        dst._check(dst._fn("mps_set_bond")(dst._h, b, len(bd), sec.ctypes.data_as(C.POINTER(C.c_int)),
                                            dims.ctypes.data_as(C.POINTER(C.c_int))))
    for b in range(N):
        d = np.ascontiguousarray(src.get_site(b))
        dst._check(dst._fn("mps_set_site")(dst._h, b, d.ctypes.data_as(C.POINTER(C.c_double)), d.size))


def test_fp64_tiles_match_dmma_kernel_on_swept_state():
    """DFMA tile schedule vs the DMMA kernel: relative error <= 1e-13 (both
    FP64; only the summation order differs), and <x, H y> = <H x, y>."""
    c = synth.WORKLOADS["n24"]
    N, n, s2, D = c["N"], c["n_elec"], c["two_sz"], c["D"]
    k = N // 2 - 1
    h, v = synth.integrals(N, c["lam"], c["seed"])
    a = _ctx(TNS_FP64_KERNEL="dfma")
    a.load_integrals(h, v)
    a.mps_init(N, n, s2, D)
    a.sweep(1, D, tol=1e-6, max_iter=40, precision=TNS_BF16X3)
    assert max(d for _, d in a.get_bond(k)) > 32  # output blocks beyond the 32 x 32 class
    b = _ctx(TNS_FP64_KERNEL="dmma")
    b.load_integrals(h, v)
    _copy_state(a, b, N, n, s2, D)
    a.build_env(k)
    b.build_env(k)
    _, length = a.psi_layout(k)
    assert b.psi_layout(k)[1] == length
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(2 * length, device="cuda", dtype=torch.float64, generator=g)
    ya = torch.empty_like(x)
    yb = torch.empty_like(x)
    a.heff_apply_ptr(k, x.data_ptr(), ya.data_ptr(), 2, TNS_FP64)
    b.heff_apply_ptr(k, x.data_ptr(), yb.data_ptr(), 2, TNS_FP64)
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(ya - yb) / torch.linalg.norm(yb))
    assert err < 1e-13, err
    xa, xb = x[:length], x[length:]
    Ha, Hb = ya[:length], ya[length:]
    scale = float(torch.linalg.norm(xa) * torch.linalg.norm(Hb))
    assert abs(float(torch.dot(xa, Hb)) - float(torch.dot(Ha, xb))) < 1e-12 * scale
