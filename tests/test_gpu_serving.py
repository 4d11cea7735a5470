"""Serving loop: requests of different sizes, microstructures and load paths
admitted into concurrent slots; every result equals the same solve run
alone; memory-budget admission; cancel; timeout; latency statistics."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    return combo


def mix_problems():
    from paper_2204_13624_gb300 import microstructure as ms

    rng = np.random.default_rng(5)
    out = []
    shapes = [(16, 16, 16), (24, 16, 32), (32, 32, 32), (12, 18, 24), (64, 32, 16), (32, 24, 24)]
    for i, n in enumerate(shapes):
        Fb = np.eye(3) + np.diag(rng.uniform(-0.05, 0.05, 3))
        Fb[0, 1] += rng.uniform(-0.05, 0.05)
        if i % 2 == 0:
            p = ms.random_spheres(n, max(3.0, min(n) / 6), 0.08, 100 + i, 10.0, Fb, 1 + i % 3)
        else:
            p = ms.random_boxels(n, seed=200 + i, contrast=10.0, Fbar=Fb, n_steps=1 + i % 3)
        out.append(p)
    return out


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_results_alone_equal_results_in_the_mix(cb, prec):
    probs = mix_problems()
    alone = [cb.solve(p, fields=True, precision=prec, tol=1e-8) for p in probs]
    srv = cb.Server(max_slots=3, keep_fields=True)
    try:
        tickets = [srv.submit(p, precision=prec, tol=1e-8) for p in probs]
        mixed = [srv.wait(t, timeout_ms=120000) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for a, m in zip(alone, mixed):
        assert np.array_equal(a["iters"], m["iters"]) and np.array_equal(a["cg_iters"], m["cg_iters"])
        assert np.max(np.abs(a["Pbar"] - m["Pbar"])) <= 1e-12 * np.max(np.abs(a["Pbar"]))
        assert np.max(np.abs(a["F"] - m["F"])) <= 1e-12 * np.max(np.abs(a["F"]))
    assert st["completed"] == len(probs) and st["failed"] == 0
    assert 1 <= st["peak_running"] <= 3
    assert 0 < st["p50_seconds"] <= st["p99_seconds"]


def test_admission_respects_the_memory_budget(cb):
    probs = mix_problems()
    fps = [cb.footprint(p, precision=1) for p in probs]
    budget = int(max(fps) * 1.5)  # at most one large solve at a time
    srv = cb.Server(max_slots=4, hbm_budget_bytes=budget)
    try:
        tickets = [srv.submit(p, precision=1) for p in probs]
        for t in tickets:
            srv.wait(t, timeout_ms=120000)
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == len(probs)
    assert st["in_use_bytes"] == 0 and st["queued"] == 0 and st["running"] == 0


def test_too_large_for_the_budget_is_rejected(cb):
    p = mix_problems()[2]
    srv = cb.Server(max_slots=1, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(cb.ComboError) as e:
            srv.submit(p)
        assert e.value.code == -2
    finally:
        srv.close()


def test_cancel_and_timeout(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    big = ms.spheres_256(n=128, vf=0.1, n_steps=3)
    small = mix_problems()[0]
    srv = cb.Server(max_slots=1)
    try:
        t1 = srv.submit(big, precision=1)
        t2 = srv.submit(small)
        t3 = srv.submit(small)
        srv.cancel(t3)  # still queued behind t1 and t2
        with pytest.raises(cb.ComboError) as e:
            srv.wait(t3, timeout_ms=60000)
        assert e.value.code == -9
        with pytest.raises(cb.ComboError) as e:
            srv.wait(t2, timeout_ms=0)  # t1 still runs: t2 cannot be done yet
        assert e.value.code == -7
        assert srv.poll(t2) is None  # queued behind the running t1
        srv.cancel(t1)  # running: stops at its next host round trip
        with pytest.raises(cb.ComboError) as e:
            srv.wait(t1, timeout_ms=120000)
        assert e.value.code == -9
        r2 = srv.wait(t2, timeout_ms=120000)
        assert r2["steps_done"] == small["n_steps"]
    finally:
        srv.close()


def test_requests_arriving_while_others_run_are_admitted(cb):
    probs = mix_problems()
    srv = cb.Server(max_slots=2)
    try:
        t0 = [srv.submit(p, precision=1) for p in probs[:2]]
        time.sleep(0.05)
        t1 = [srv.submit(p, precision=1) for p in probs[2:]]
        res = [srv.wait(t, timeout_ms=120000) for t in t0 + t1]
        st = srv.stats()
    finally:
        srv.close()
    assert all(r["steps_done"] == p["n_steps"] for r, p in zip(res, probs))
    assert st["peak_running"] == 2 and st["completed"] == len(probs)


def test_small_compatible_requests_are_batched(cb):
    """Queued requests on the same small grid with the same options are solved
    as one batch; each result equals the same solve run alone."""
    from paper_2204_13624_gb300 import microstructure as ms

    rng = np.random.default_rng(11)
    probs = []
    for i in range(6):
        Fb = np.eye(3) + np.diag(rng.uniform(-0.04, 0.04, 3))
        probs.append(ms.random_spheres((16, 16, 16), 3.0, 0.06 + 0.02 * (i % 3), 500 + i, 5.0 + i, Fb, 1 + i % 2))
    other = mix_problems()[1]  # another grid: never in the same batch
    alone = [cb.solve(p, precision=0, tol=1e-8) for p in probs]
    srv = cb.Server(max_slots=1, batch_max=4)
    try:
        blocker = srv.submit(ms.spheres_256(n=128, vf=0.1, n_steps=1), precision=1)  # keeps the slot busy
        tickets = [srv.submit(p, precision=0, tol=1e-8) for p in probs]
        t_other = srv.submit(other, precision=0, tol=1e-8)
        srv.wait(blocker, timeout_ms=120000)
        res = [srv.wait(t, timeout_ms=120000) for t in tickets]
        r_other = srv.wait(t_other, timeout_ms=120000)
        st = srv.stats()
    finally:
        srv.close()
    assert st["batches"] >= 2 and st["batched_requests"] >= 4
    assert st["completed"] == len(probs) + 2 and st["failed"] == 0
    for a, r in zip(alone, res):
        assert np.array_equal(a["iters"], r["iters"]) and np.array_equal(a["cg_iters"], r["cg_iters"])
        assert np.max(np.abs(a["Pbar"] - r["Pbar"])) <= 1e-12 * np.max(np.abs(a["Pbar"]))
    assert r_other["steps_done"] == other["n_steps"]
