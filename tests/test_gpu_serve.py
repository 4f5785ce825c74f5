"""Continuous batching: requests of mixed grid sizes and accuracies, admitted while
others run, give the same result as the same solve alone; the device-memory budget
bounds what the server holds; an invalid request fails alone."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, serve, workloads as W  # noqa: E402

SIZES = (32, 64, 96)


def _density(n, seed, precision):
    dt = torch.float32 if precision == "fp32" else torch.float64
    return torch.from_numpy(W.gaussian_mixture(n, -1.0, 1.0, seed)).to(dt).pin_memory()


def test_results_in_the_mix_equal_alone():
    srv = serve.Server(budget_bytes=8e9, max_batch=4, slots=3).start()
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(48):
        n = int(SIZES[rng.integers(3)])
        acc = (1e-6, 1e-12)[int(rng.integers(2))]
        rho = _density(n, i, serve.precision_for(acc))
        reqs.append((n, acc, rho, srv.submit(rho, acc)))
        if i % 8 == 7:
            time.sleep(0.002)  # arrivals in bursts, while earlier batches run
    results = [f.result(timeout=120) for *_, f in reqs]
    srv.stop()
    plans = {}
    for (n, acc, rho, _), u in zip(reqs, results):
        key = (n, serve.precision_for(acc))
        if key not in plans:
            plans[key] = Plan(n, -1.0, 1.0, precision=key[1])
        alone = plans[key].solve(rho.cuda()).cpu()
        assert torch.equal(u, alone), key
    for p in plans.values():
        p.close()


def test_budget_bounds_resident_plans_and_bad_request_fails_alone():
    # room for one 96^3 plan only: the 64^3 and 96^3 keys must take turns (eviction)
    one = serve.entry_bytes(96, "df32", 2)
    srv = serve.Server(budget_bytes=int(1.1 * one), max_batch=2, slots=2).start()
    futs = []
    for i in range(12):
        n = (64, 96)[i % 2]
        acc = 1e-12
        futs.append(srv.submit(_density(n, i, "df32"), acc))
    bad = srv.submit(torch.zeros((64, 64, 64), dtype=torch.float32).pin_memory(), 1e-12)  # wrong dtype
    for f in futs:
        assert f.result(timeout=120).shape[0] in (64, 96)
    with pytest.raises(ValueError):
        bad.result(timeout=120)
    too_big = srv.submit(_density(128, 0, "df32"), 1e-12)
    with pytest.raises(MemoryError):
        too_big.result(timeout=120)
    srv.stop()
    assert srv.peak_bytes <= int(1.1 * one)


def test_results_into_caller_buffers():
    # results land in the pinned buffers the caller passes; a wrongly shaped buffer fails
    # its request alone
    srv = serve.Server(budget_bytes=4e9, max_batch=4, slots=2).start()
    rhos = [_density(64, i, "df32") for i in range(6)]
    outs = [torch.full(r.shape, float("nan"), dtype=r.dtype).pin_memory() for r in rhos]
    futs = [srv.submit(r, 1e-12, out=o) for r, o in zip(rhos, outs)]
    bad = srv.submit(rhos[0], 1e-12, out=torch.empty((8, 8, 8), dtype=torch.float64))
    got = [f.result(timeout=120) for f in futs]
    with pytest.raises(ValueError):
        bad.result(timeout=120)
    srv.stop()
    plan = Plan(64, -1.0, 1.0, precision="df32")
    for r, o, g in zip(rhos, outs, got):
        assert g.data_ptr() == o.data_ptr()
        assert torch.equal(o, plan.solve(r.cuda()).cpu())
    plan.close()


def test_large_sizes_in_the_mix_equal_alone():
    # the served sizes where the latency tail lives (128^3, 192^3, 256^3) mixed with small
    # ones, both accuracies: each result equals the same solve alone, bit for bit
    srv = serve.Server(budget_bytes=40e9, max_batch=4, slots=4).start()
    rng = np.random.default_rng(1)
    sizes = (32, 128, 192, 256)
    reqs = []
    for i in range(24):
        n = int(sizes[rng.integers(len(sizes))])
        acc = (1e-6, 1e-12)[int(rng.integers(2))]
        rho = _density(n, 100 + i, serve.precision_for(acc))
        reqs.append((n, acc, rho, srv.submit(rho, acc)))
        if i % 6 == 5:
            time.sleep(0.005)
    results = [f.result(timeout=300) for *_, f in reqs]
    srv.stop()
    plans = {}
    for (n, acc, rho, _), u in zip(reqs, results):
        key = (n, serve.precision_for(acc))
        if key not in plans:
            plans[key] = Plan(n, -1.0, 1.0, precision=key[1])
        assert torch.equal(u, plans[key].solve(rho.cuda()).cpu()), key
    for p in plans.values():
        p.close()


def test_replayed_stream_completes_with_results_equal_alone():
    # a seeded Poisson stream submitted by the library at the arrival times (the bench's
    # load generator): every request completes, latencies are stamped on the monotonic
    # clock after their arrivals, and sampled results equal the solve alone
    srv = serve.Server(budget_bytes=20e9, max_batch=4, slots=3).start()
    sizes = (32, 64, 96)
    dens = {}
    for n in sizes:
        for prec in ("fp32", "df32"):
            dens[(n, prec)] = _density(n, n, prec)
    outputs = {k: [v.new_empty(v.shape).pin_memory() for _ in range(2)] for k, v in dens.items()}
    t0 = time.monotonic() + 0.05
    kept = serve.poisson_stream(srv, rate=400.0, duration=0.2, sizes=sizes, accuracies=(1e-6, 1e-12), seed=3,
                                densities=dens, warmup=0.05, outputs=outputs, t0=t0)
    recs = srv.completed
    assert len(recs) >= len(kept) > 10
    assert all(r.done_at > r.arrival >= t0 - 1e-6 for r in recs)
    s = serve.latency_summary(srv, t0 + 0.05, t0 + 0.25)
    assert s["requests"] == len(kept) and s["p99_ms"] > 0
    for key in ((32, "fp32"), (96, "df32")):
        plan = Plan(key[0], -1.0, 1.0, precision=key[1])
        want = plan.solve(dens[key].cuda()).cpu()
        out = torch.empty_like(dens[key]).pin_memory()
        assert torch.equal(srv.submit(dens[key], 1e-6 if key[1] == "fp32" else 1e-12, out=out).result(timeout=60),
                           want)
        plan.close()
    srv.stop()


def test_waiting_requests_are_batched():
    # one slot and one plan: requests that arrive while a batch runs wait for it and are
    # then solved together (at most max_batch at a time); each result equals the solve alone
    srv = serve.Server(budget_bytes=8e9, max_batch=4, slots=1, plans_per_key=1).start()
    key = (128, "df32")
    rhos = [_density(128, 200 + i, "df32") for i in range(12)]
    outs = [torch.empty_like(r).pin_memory() for r in rhos]
    t0 = time.monotonic() + 0.05
    futs = srv.replay([t0] * len(rhos), [key] * len(rhos), rhos, outs)
    got = [f.result(timeout=120) for f in futs]
    srv.stop()
    assert srv.batches <= 1 + (len(rhos) - 1 + 3) // 4  # the first alone, then batches of up to 4
    plan = Plan(128, -1.0, 1.0, precision="df32")
    for r, g in zip(rhos, got):
        assert torch.equal(g, plan.solve(r.cuda()).cpu())
    plan.close()
