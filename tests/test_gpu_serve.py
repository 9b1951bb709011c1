"""Continuous-batching server: requests join and leave the batch between
steps, admission is bounded by slots and an HBM budget, and every served
result equals the same solve run alone (bit for bit: the per-cell arithmetic
does not depend on which other solves share the launch)."""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05061_gb300 import build, hydro, serve

    build.build()
    hydro.load()
    return torch, hydro, serve


def small_requests(serve):
    # all arrive at once, so that slots and the memory budget decide admission
    specs = [("kh2d", 48, 12), ("rt3d", 16, 9), ("kh2d", 37, 15), ("rt3d", 24, 6),
             ("kh2d", 64, 7), ("rt3d", 20, 11), ("kh2d", 33, 5)]
    reqs = []
    for i, (fam, n, steps) in enumerate(specs):
        r = serve.Request(id=i, arrival=0.0, family=fam, n=n, steps=steps, seed=151005063 + i)
        reqs.append(serve.make_payload(r))
    return reqs


def solo_state(hydro, req):
    sim = hydro.Simulation(req.prob, req.W)
    sim.run_steps(req.steps)
    out = sim.get_state()
    sim.close()
    return out


def test_served_results_equal_solo_and_budget_binds(env):
    torch, hydro, serve = env
    reqs = small_requests(serve)
    probe = serve.Server(budget_bytes=1e12, max_active=8, max_items3d=200000, max_items2d=20000)
    sizes = [probe.request_bytes(r) for r in reqs]
    probe.close()
    budget = 2.2 * max(sizes)            # at most a few solves fit at once
    srv = serve.Server(budget_bytes=budget, max_active=8, max_items3d=200000, max_items2d=20000)
    peak = {"n": 0, "mixed": False}
    orig_advance = srv.advance

    def advance(keep):
        peak["n"] = max(peak["n"], len(srv.active))
        fams = {r.family for r in srv.active.values()}
        peak["mixed"] |= len(fams) == 2
        assert srv.used <= budget
        return orig_advance(keep)

    srv.advance = advance
    stats = srv.run(reqs, keep_results=lambda r: True)
    srv.close()
    assert stats["requests"] == len(reqs)
    assert 2 <= peak["n"] < len(reqs)     # solves overlapped, and the budget held some back
    assert peak["mixed"]                  # 2D and 3D solves shared ticks
    assert stats["p99_latency_s"] >= stats["p50_latency_s"] > 0
    for r in reqs:
        assert np.array_equal(r.result, solo_state(hydro, r)), r.id


def test_slot_limit_and_reuse(env):
    torch, hydro, serve = env
    reqs = small_requests(serve)[:5]
    srv = serve.Server(budget_bytes=1e12, max_active=2, max_items3d=200000, max_items2d=20000)
    seen = []
    orig = srv.advance

    def advance(keep):
        seen.append(len(srv.active))
        return orig(keep)

    srv.advance = advance
    stats = srv.run(reqs, keep_results=lambda r: True)
    srv.close()
    assert max(seen) <= 2 and stats["requests"] == 5
    for r in reqs:
        assert np.array_equal(r.result, solo_state(hydro, r)), r.id


def test_lazy_payloads_match_eager(env):
    """A stream whose payloads are built by the background prefetcher gives
    the same results as one built up front."""
    torch, hydro, serve = env
    kw = dict(count=6, rate=1e6, seed=7, kh2d=(32, 48), rt3d=(16, 24), steps=(3, 5))
    eager = serve.requests_from_inputs(**kw)
    lazy = serve.requests_from_inputs(lazy=True, **kw)
    assert all(r.prob is None for r in lazy)
    out = []
    for reqs in (eager, lazy):
        srv = serve.Server(budget_bytes=2e9, max_active=3, max_items3d=4096, max_items2d=4096)
        srv.run(reqs, keep_results=lambda r: True)
        srv.close()
        out.append({r.id: r.result for r in reqs})
    assert all(r.W is None for r in lazy)
    for i in out[0]:
        assert np.array_equal(out[0][i], out[1][i])


def test_served_results_match_the_oracle(env):
    """A served FP32 result against the FP64 oracle: density within the
    FP32 accuracy bound (L1-relative 1e-4) after the request's steps."""
    import oracle

    torch, hydro, serve = env
    reqs = small_requests(serve)[:4]
    srv = serve.Server(budget_bytes=1e12, max_active=4, max_items3d=200000, max_items2d=20000)
    srv.run(reqs, keep_results=lambda r: True)
    srv.close()
    oracle.build()
    for r in reqs:
        o = oracle.Oracle(r.prob.replace(precision=inputs.FP64))
        V, _, s, _ = o.run(o.state_from_prim(r.W), max_steps=r.steps)
        assert s == r.steps
        rho = o.total(V)[0]
        rho_gpu = o.total(r.result.astype(np.float64))[0]
        err = float(np.abs(rho_gpu - rho).sum() / np.abs(rho).sum())
        assert err <= 1e-4, (r.id, err)


def test_server_loop_never_waits_for_the_whole_stream(env, monkeypatch):
    """Steps, admissions and retirements are enqueued without synchronising
    the stream; the host only polls (or waits on) its own marks."""
    torch, hydro, serve = env
    reqs = small_requests(serve)
    calls = {"n": 0}

    def counted(orig):
        def f(*a, **k):
            calls["n"] += 1
            return orig(*a, **k)
        return f

    srv = serve.Server(budget_bytes=1e12, max_active=3, max_items3d=200000, max_items2d=20000)
    monkeypatch.setattr(srv.stream, "synchronize", counted(srv.stream.synchronize))
    monkeypatch.setattr(torch.cuda, "synchronize", counted(torch.cuda.synchronize))
    stats = srv.run(reqs, keep_results=lambda r: True)
    srv.close()
    assert stats["requests"] == len(reqs)
    assert calls["n"] <= 1            # the statistics' final synchronisation only
    for r in reqs:
        assert np.array_equal(r.result, solo_state(hydro, r)), r.id


def test_queue_survives_an_empty_list_between_launches(env):
    """The claim counters of a list reset themselves at the end of every
    launch, so a list may sit empty (its launches skipped) while the other
    one runs, and fill again: a 3D solve that leaves, 2D steps with no 3D
    instance, a new 3D solve -- each result equals its solo run."""
    torch, hydro, serve = env
    mk = lambda i, fam, n, steps: serve.make_payload(serve.Request(id=i, arrival=0.0, family=fam, n=n, steps=steps,
                                                                   seed=151005063 + i))
    a, b, c = mk(0, "rt3d", 20, 4), mk(1, "kh2d", 40, 15), mk(2, "rt3d", 18, 5)
    srv = serve.Server(budget_bytes=1e12, max_active=4, max_items3d=200000, max_items2d=20000)
    keep = lambda r: True
    assert srv.try_admit(a, 0.0) and srv.try_admit(b, 0.0)
    done = []
    while a.id in {r.id for r in srv.active.values()}:
        done += srv.advance(keep)
    for _ in range(3):                      # 2D only: the 3D launches are skipped
        done += srv.advance(keep)
    assert all(r.prob.ndim == 2 for r in srv.active.values())
    assert srv.try_admit(c, 0.0)
    while srv.active:
        done += srv.advance(keep)
    done += srv.poll(block=True)
    while srv._marks:
        done += srv.poll(block=True)
    srv.close()
    assert {r.id for r in done} == {0, 1, 2}
    for r in (a, b, c):
        assert np.array_equal(r.result, solo_state(hydro, r)), r.id
