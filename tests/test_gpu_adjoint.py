"""Differentiation form on the GPU: torch.autograd through H_eff*psi (FP64),
gradients with respect to psi and to the left/right operator arenas checked by
central finite differences (step 1e-5, relative error <= 1e-6)."""
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_05581_gb300 import Context, DEFAULT_LIB  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(DEFAULT_LIB):
        from paper_2305_05581_gb300 import build as b
        b.build()


@pytest.mark.parametrize("N,n,s2,D,k", [(6, 6, 0, 12, 2), (8, 8, 0, 40, 3), (10, 10, 0, 60, 4)])
def test_autograd_gradients_match_finite_differences(N, n, s2, D, k):
    from paper_2305_05581_gb300.autograd import arena_tensor, heff
    h, v = synth.integrals(N, 3.0, 900 + N)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k + 2)
    ctx = Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    _, length = ctx.psi_layout(k)
    g = torch.Generator(device="cuda").manual_seed(N)
    x = torch.randn(length, device="cuda", dtype=torch.float64, generator=g).requires_grad_(True)
    yb = torch.randn(length, device="cuda", dtype=torch.float64, generator=g)
    L = arena_tensor(ctx, k, 0)
    R = arena_tensor(ctx, k, 1)
    Lp = L.detach().requires_grad_(True)
    Rp = R.detach().requires_grad_(True)
    E = torch.dot(yb, heff(x, Lp, Rp, ctx, k))
    E.backward()

    def energy():
        y = torch.empty_like(x)
        ctx.heff_apply_ptr(k, x.detach().data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        return float(torch.dot(yb, y))

    # psi: linear map, gradient = H_eff^T Ybar
    d = 1e-5
    idx = torch.randint(0, length, (6,), generator=g, device="cuda").tolist()
    for e in idx:
        with torch.no_grad():
            x[e] += d
        ep = energy()
        with torch.no_grad():
            x[e] -= 2 * d
        em = energy()
        with torch.no_grad():
            x[e] += d
        assert abs((ep - em) / (2 * d) - float(x.grad[e])) <= 1e-6 * max(1.0, float(x.grad.abs().max()))
    for arena, grad in ((L, Lp.grad), (R, Rp.grad)):
        nz = torch.nonzero(grad).flatten()
        sel = nz[torch.randperm(nz.numel(), generator=torch.Generator().manual_seed(1))[:8].to(nz.device)].tolist()
        scale = max(1.0, float(grad.abs().max()))
        for e in sel:
            old = float(arena[e])
            arena[e] = old + d
            ctx.build_env(k)
            ep = energy()
            arena[e] = old - d
            ctx.build_env(k)
            em = energy()
            arena[e] = old
            ctx.build_env(k)
            assert abs((ep - em) / (2 * d) - float(grad[e])) <= 1e-6 * scale
