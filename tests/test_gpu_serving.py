"""Serving and batched synthesis through the C ABI: every result is the same alone and in the mix.

Tolerance: FP32 path, 1e-4 relative per shell bin (the stated FP32 bound).  Members of a batch that share
kernels with the single call are compared more tightly.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_27231_gb300 import build, sigw
    build.build()
    sigw.lib()
    return sigw


def _spec(N, kind, seed, F=0.0, sigma=0.5):
    return workloads.Spec(N=N, L=1.0, A=1e-2, sigma=sigma, kstar=(N // 8) * 2 * np.pi, kind=kind,
                          F_NL=F, seed=seed)


def _alone(lib, spec):
    with lib.Plan(spec.N, spec.L, precision=32) as p:
        p.generate_spec(spec)
        return p.spectrum()["omega"][0]


def test_generate_batch_matches_single_calls(lib):
    specs = [_spec(32, "gauss", 11), _spec(32, "local", 12, F=3.0, sigma=0.7), _spec(32, "usr", 13, sigma=0.3)]
    with lib.Plan(32, 1.0, precision=32, max_batch=3) as p:
        p.generate_batch(specs)
        mixed = p.spectrum()["omega"]
    for i, s in enumerate(specs):
        np.testing.assert_allclose(mixed[i], _alone(lib, s), rtol=1e-4)
    # non-Gaussian members run the same kernels alone and in the batch
    np.testing.assert_array_equal(mixed[1], _alone(lib, specs[1]))


def test_server_results_equal_alone(lib):
    specs = []
    seed = 100
    for N in (16, 32, 64):
        for kind, F in (("gauss", 0.0), ("local", 2.0), ("usr", 0.0)):
            specs.append(_spec(N, kind, seed, F=F))
            seed += 1
    with lib.Server(40e9, max_slots=3, max_batch=2, precision=32) as srv:
        tickets = [srv.submit(s) for s in specs]
        results = [srv.wait(t, timeout_s=300) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(specs) and st["failed"] == 0
    assert st["batches"] <= len(specs)
    for s, (om, lat) in zip(specs, results):
        assert lat > 0
        np.testing.assert_allclose(om, _alone(lib, s), rtol=1e-4)


def test_server_admission_under_small_budget(lib):
    fp64_budget = lib.footprint(64, lib.default_opts(max_batch=1)) * 1.2
    with lib.Server(fp64_budget, max_slots=2, max_batch=1, precision=32) as srv:
        specs = [_spec(64, "local", 200 + i, F=1.0) for i in range(3)] + [_spec(32, "gauss", 210)]
        tickets = [srv.submit(s) for s in specs]
        with pytest.raises(lib.SigwError) as e:
            srv.submit(_spec(128, "gauss", 1))
        assert e.value.status == lib.EBUSY
        results = [srv.wait(t, timeout_s=300) for t in tickets]
        st = srv.stats()
    assert st["completed"] == 4
    assert st["hbm_peak"] <= fp64_budget
    for s, (om, _) in zip(specs, results):
        np.testing.assert_allclose(om, _alone(lib, s), rtol=1e-4)


def test_server_wait_timeout_then_result(lib):
    with lib.Server(40e9, max_slots=1, precision=32) as srv:
        t = srv.submit(_spec(128, "gauss", 7))
        with pytest.raises(lib.SigwError) as e:
            srv.wait(t, timeout_s=1e-4)
        assert e.value.status == lib.ETIMEOUT
        om, lat = srv.wait(t, timeout_s=300)
        assert np.all(np.isfinite(om)) and lat > 0
        with pytest.raises(lib.SigwError):
            srv.poll(t)  # ticket consumed


def test_express_slot_serves_small_requests_beside_a_large_batch(lib):
    """With one general slot busy on a 128^3 request, the express slot (N <= 32) takes the small requests that
    arrive behind it; every result still equals its single-plan value."""
    big = _spec(128, "local", 300, F=2.0)
    small = [_spec(16, "gauss", 301), _spec(32, "usr", 302), _spec(16, "local", 303, F=1.0)]
    with lib.Server(40e9, max_slots=1, max_batch=2, precision=32) as srv:
        srv.set_express(1, 32)
        with pytest.raises(lib.SigwError) as e:
            srv.set_express(1, 32)
        assert e.value.status == lib.ESTATE
        tb = srv.submit(big)
        ts = [srv.submit(s) for s in small]
        res_small = [srv.wait(t, timeout_s=300) for t in ts]
        om_big, _ = srv.wait(tb, timeout_s=300)
        st = srv.stats()
    assert st["completed"] == 4 and st["failed"] == 0 and st["express_batches"] >= 1
    np.testing.assert_allclose(om_big, _alone(lib, big), rtol=1e-4)
    for s, (om, lat) in zip(small, res_small):
        np.testing.assert_allclose(om, _alone(lib, s), rtol=1e-4)


def test_queue_head_is_not_starved_by_small_requests(lib):
    """A 64^3 request whose plan fits the budget only after an idle 32^3 plan is evicted, queued ahead of a stream of
    32^3 requests that an express slot could serve: while it cannot be admitted, no later request starts, so it
    completes before the small stream does (instead of after it), and every result equals its single-plan value."""
    import time
    fp32 = lib.footprint(32, lib.default_opts(max_batch=2))
    fp64 = lib.footprint(64, lib.default_opts(max_batch=2))
    first = [_spec(32, "gauss", 400 + i) for i in range(2)]
    big = _spec(64, "local", 410, F=1.5)
    stream = [_spec(32, "usr", 420 + i, sigma=0.4) for i in range(24)]
    with lib.Server(fp64 + 0.5 * fp32, max_slots=1, max_batch=2, precision=32) as srv:
        srv.set_express(1, 32)
        tf = [(time.perf_counter(), srv.submit(s)) for s in first]
        tb = (time.perf_counter(), srv.submit(big))
        ts = [(time.perf_counter(), srv.submit(s)) for s in stream]
        res_first = [srv.wait(t, timeout_s=300) for _, t in tf]
        om_big, lat_big = srv.wait(tb[1], timeout_s=300)
        res_stream = [srv.wait(t, timeout_s=300) for _, t in ts]
        st = srv.stats()
    assert st["completed"] == 27 and st["failed"] == 0 and st["plans_evicted"] >= 1
    big_done = tb[0] + lat_big
    last_small_done = max(t0 + lat for (t0, _), (_, lat) in zip(ts, res_stream))
    assert big_done < last_small_done
    np.testing.assert_allclose(om_big, _alone(lib, big), rtol=1e-4)
    for s, (om, _) in zip(first + stream, res_first + res_stream):
        np.testing.assert_allclose(om, _alone(lib, s), rtol=1e-4)
