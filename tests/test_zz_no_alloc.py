"""sigw_fft3d_noalloc (the allocation-free 3-D FFT) against the plan-based sigw_fft3d.

Callers that cannot call cudaMalloc use the allocation-free entry point; it must give the same
transform as the plan-based one, call after call, although every call reuses one static scratch array.
This file is collected last so that a run stopping at its first failure has run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_27231_gb300 import build, sigw
    build.build()
    sigw.lib()
    return torch, sigw


@pytest.mark.parametrize("N,precision", [(32, 32), (128, 32), (16, 64), (64, 64)])
def test_noalloc_matches_plan_fft_twice(env, N, precision):
    torch, sigw = env
    rdt = torch.float64 if precision == 64 else torch.float32
    cdt = torch.complex128 if precision == 64 else torch.complex64
    tol = 1e-12 if precision == 64 else 2e-6
    rng = np.random.default_rng(100 + N)
    with sigw.Plan(N, 1.0, precision=precision, n_alpha=2) as plan:
        for call in range(2):  # two calls in a row through the shared scratch
            x = torch.tensor(rng.standard_normal((N, N, N)), dtype=rdt, device="cuda")
            ref = torch.empty((N, N, N // 2 + 1), dtype=cdt, device="cuda")
            plan.fft3d(-1, x.data_ptr(), ref.data_ptr())
            plan.synchronize()
            got = torch.empty_like(ref)
            sigw.fft3d_noalloc(N, precision, -1, x.data_ptr(), got.data_ptr())
            torch.cuda.synchronize()
            scale = ref.abs().max().item()
            assert (got - ref).abs().max().item() <= tol * scale, (call, "forward")
            back_ref = torch.empty((N, N, N), dtype=rdt, device="cuda")
            plan.fft3d(+1, ref.data_ptr(), back_ref.data_ptr())
            plan.synchronize()
            back = torch.empty_like(back_ref)
            sigw.fft3d_noalloc(N, precision, +1, got.data_ptr(), back.data_ptr())
            torch.cuda.synchronize()
            scale = back_ref.abs().max().item()
            assert (back - back_ref).abs().max().item() <= tol * scale, (call, "inverse")


def test_noalloc_rejects_sizes_beyond_the_scratch(env):
    torch, sigw = env
    x = torch.zeros(8, device="cuda")
    for N, precision in ((256, 32), (128, 64), (12, 32)):
        with pytest.raises(sigw.SigwError) as e:
            sigw.fft3d_noalloc(N, precision, -1, x.data_ptr(), x.data_ptr())
        assert e.value.status == sigw.EINVAL
