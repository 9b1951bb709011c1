"""The update's FP64 arithmetic helpers against CUDA's IEEE operations
(computed by PyTorch on the same GPU) and against the MC limiter's
definition: the Newton-Raphson reciprocal and quotient stay within 2 ulp,
the reciprocal square root within 2 ulp."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05061_gb300 import build, hydro

    build.build()
    hydro.load()
    return torch, hydro


def run(env, which, x, y=None):
    torch, hy = env
    out = torch.empty_like(x)
    yp = y.data_ptr() if y is not None else 0
    hy.hydro_selftest_math(which, x.data_ptr(), yp, out.data_ptr(), x.numel(),
                           torch.cuda.current_stream().cuda_stream)
    return out


def test_reciprocal_and_quotient(env):
    torch, _ = env
    g = torch.Generator(device="cuda").manual_seed(3)
    mant = torch.rand(1 << 20, device="cuda", dtype=torch.float64, generator=g) + 0.5
    expo = torch.randint(-60, 60, (1 << 20,), device="cuda", generator=g).double()
    x = mant * torch.pow(2.0, expo)
    x[::2] *= -1
    y = torch.randn(1 << 20, device="cuda", dtype=torch.float64, generator=g)
    eps = 2.0 ** -52
    r = run(env, 0, x)
    assert (torch.abs(r - 1.0 / x) / torch.abs(1.0 / x)).max().item() <= 2 * eps
    q = run(env, 1, x, y)
    ref = y / x
    assert (torch.abs(q - ref) / torch.abs(ref).clamp_min(1e-300)).max().item() <= 2 * eps
    s = run(env, 2, x.abs())
    refs = 1.0 / torch.sqrt(x.abs())
    assert (torch.abs(s - refs) / refs).max().item() <= 2 * eps


def test_mc_slope_definition(env):
    torch, _ = env
    g = torch.Generator(device="cuda").manual_seed(4)
    dl = torch.randn(1 << 16, device="cuda", dtype=torch.float64, generator=g)
    dr = torch.randn(1 << 16, device="cuda", dtype=torch.float64, generator=g)
    dl[:100] = 0.0
    dr[100:200] = 0.0
    dr[200:300] = dl[200:300]
    got = run(env, 3, dl, dr)
    a = torch.minimum(torch.minimum(2 * dl.abs(), 2 * dr.abs()), 0.5 * (dl + dr).abs())
    want = torch.where(dl * dr > 0, torch.copysign(a, dr), torch.zeros_like(a))
    assert torch.equal(got, want)
