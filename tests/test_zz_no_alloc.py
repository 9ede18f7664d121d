"""sigw_fft3d_noalloc (the allocation-free 3-D FFT) against numpy and against the plan-based sigw_fft3d.

Callers that cannot call cudaMalloc (a program whose pool allocator owns all device memory, or a path where a
synchronising allocation is not acceptable) use the allocation-free entry point.  It must give the same
transform as the plan-based one and as numpy, call after call, although every call reuses one static scratch
array; and its first call in a process must be correct on a non-blocking stream, which is not ordered after the
set-up's copies of the twiddle tables.
This file is collected last so that a run stopping at its first failure has run every other test.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = {32: 2e-6, 64: 1e-12}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_27231_gb300 import build, sigw
    build.build()
    sigw.lib()
    return torch, sigw


def _dtypes(torch, precision):
    return (torch.float64, torch.complex128) if precision == 64 else (torch.float32, torch.complex64)


@pytest.mark.parametrize("N,precision", [(8, 32), (16, 32), (32, 32), (64, 32), (128, 32), (8, 64), (16, 64),
                                         (64, 64)])
def test_noalloc_matches_numpy_twice(env, N, precision):
    """Forward transform against numpy.fft.rfftn and the round trip back, on two calls in a row."""
    torch, sigw = env
    rdt, cdt = _dtypes(torch, precision)
    tol = TOL[precision] * np.sqrt(np.log2(N ** 3))
    rng = np.random.default_rng(200 + N + precision)
    for call in range(2):
        x = rng.standard_normal((N, N, N))
        xd = torch.tensor(x, dtype=rdt, device="cuda")
        Xd = torch.empty((N, N, N // 2 + 1), dtype=cdt, device="cuda")
        sigw.fft3d_noalloc(N, precision, -1, xd.data_ptr(), Xd.data_ptr())
        yd = torch.empty((N, N, N), dtype=rdt, device="cuda")
        sigw.fft3d_noalloc(N, precision, +1, Xd.data_ptr(), yd.data_ptr())
        torch.cuda.synchronize()
        ref = np.fft.rfftn(x)
        X = Xd.cpu().numpy()
        assert np.abs(X - ref).max() <= tol * np.abs(ref).max(), (call, "forward")
        y = yd.cpu().numpy() / N ** 3
        assert np.abs(y - x).max() <= 10 * tol * np.abs(x).max(), (call, "inverse")


@pytest.mark.parametrize("N,precision", [(32, 32), (128, 32), (16, 64), (64, 64)])
def test_noalloc_matches_plan_fft_twice(env, N, precision):
    torch, sigw = env
    rdt, cdt = _dtypes(torch, precision)
    tol = TOL[precision]
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


def test_noalloc_first_call_on_a_nonblocking_stream(env):
    """In a fresh process, the very first call (which sets the device up) runs on a torch stream, which is a
    non-blocking stream; its result must match numpy, so the twiddle tables were on the device in time."""
    script = textwrap.dedent("""
        import sys
        import numpy as np
        import torch
        sys.path.insert(0, %r)
        from paper_2605_27231_gb300 import sigw
        N = 64
        rng = np.random.default_rng(7)
        x = rng.standard_normal((N, N, N))
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            xd = torch.tensor(x, dtype=torch.float32, device="cuda")
            Xd = torch.empty((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        st.synchronize()
        sigw.fft3d_noalloc(N, 32, -1, xd.data_ptr(), Xd.data_ptr(), stream=st.cuda_stream)
        st.synchronize()
        ref = np.fft.rfftn(x)
        err = np.abs(Xd.cpu().numpy() - ref).max() / np.abs(ref).max()
        print("ERR", err)
        sys.exit(0 if err <= 2e-6 * np.sqrt(np.log2(N ** 3)) else 1)
    """ % ROOT)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr


def test_noalloc_rejects_sizes_beyond_the_scratch(env):
    torch, sigw = env
    x = torch.zeros(8, device="cuda")
    for N, precision in ((256, 32), (128, 64), (12, 32)):
        with pytest.raises(sigw.SigwError) as e:
            sigw.fft3d_noalloc(N, precision, -1, x.data_ptr(), x.data_ptr())
        assert e.value.status == sigw.EINVAL
