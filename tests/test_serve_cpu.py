"""Scheduler and arena of the serving loop, driven by a simulated executor (no GPU)."""
import numpy as np

from paper_2010_04868_gb300 import inputs, serve


def test_request_mix_follows_the_recipe():
    reqs = serve.request_mix(400)
    assert len(reqs) == 400
    for r in reqs:
        assert r.dim in (1, 2, 3) and 10 <= r.T <= 500
        assert r.cls in serve.CLASSES
        if r.method == 1:
            assert r.shape == 0
        if r.dim == 1:
            assert (1 << 12) - 1 <= r.ext[0] <= (1 << 22) + 1
        elif r.dim == 2:
            assert 255 <= r.ext[0] <= 4097 and r.ext[0] == r.ext[1]
        else:
            assert 63 <= r.ext[0] <= 385 and len(set(r.ext)) == 1
    assert {r.method for r in reqs} == {0, 1} and {r.dim for r in reqs} == {1, 2, 3}
    assert serve.request_mix(50)[7] == serve.request_mix(50)[7]   # deterministic


def test_catalog_weights_are_normalised_and_distinct():
    seen = set()
    for c in serve.CLASSES:
        w = serve.class_weights(c)
        k = 2 * c[1] + 1 if c[2] == 0 else 3 ** c[1]
        assert len(w) == k and (w > 0).all() and abs(w.sum() - 1) < 1e-12
        seen.add(tuple(w))
    assert len(seen) == len(serve.CLASSES)


def test_arena_blocks_never_overlap_and_coalesce():
    """Random allocations and releases against a byte map: aligned, disjoint, inside the cap, and the
    free list returns to one block when everything is released."""
    cap = 1 << 20
    a = serve.ArenaBlocks(cap)
    owner = np.zeros(cap // serve.ALIGN, dtype=np.int64)
    live = {}
    u = inputs.uniform(77, 4000)
    for i in range(2000):
        if live and u[2 * i] < 0.45:
            k = sorted(live)[int(u[2 * i + 1] * len(live))]
            off, n = live.pop(k)
            a.release(off, n)
            owner[off // serve.ALIGN:(off + n + serve.ALIGN - 1) // serve.ALIGN] = 0
        else:
            n = 1 + int(u[2 * i + 1] * 60000)
            off = a.alloc(n)
            if off is None:
                continue
            assert off % serve.ALIGN == 0 and off + n <= cap
            blk = owner[off // serve.ALIGN:(off + n + serve.ALIGN - 1) // serve.ALIGN]
            assert (blk == 0).all(), "overlap"
            blk[:] = i + 1
            live[i] = (off, n)
        assert a.used == sum((n + serve.ALIGN - 1) // serve.ALIGN * serve.ALIGN for _, n in live.values())
        for (o1, l1), (o2, l2) in zip(a.free, a.free[1:]):
            assert o1 + l1 < o2                               # sorted, disjoint, coalesced
    for off, n in live.values():
        a.release(off, n)
    assert a.free == [(0, cap)] and a.used == 0


def test_admission_respects_slots_memory_and_fifo():
    reqs = serve.request_mix(60)
    serve.poisson_arrivals(reqs, rate=2000.0)
    cap = 3 * 10 ** 9
    ex = serve.SimExecutor(slots=4, rate_updates_per_s=5e13)
    st = serve.Server(ex, slots=4, mem_cap=cap).serve(reqs)
    too_big = sum(1 for r in reqs if r.nbytes > cap)
    assert st.completed + st.rejected == len(reqs)
    assert st.rejected == too_big
    assert st.max_mem <= cap
    assert ex.max_inflight <= 4 and ex.slots_seen <= {0, 1, 2, 3}
    assert len(st.latencies_ms) == st.completed
    assert min(st.latencies_ms) >= 0.0


def test_service_model_fit_and_stratified_sample():
    reqs = serve.request_mix(300)
    sample = serve.stratified_sample(reqs, 4)
    assert {r.cls for r in sample} == {r.cls for r in reqs}
    assert all(sum(1 for r in sample if r.cls == c) <= 4 for c in serve.CLASSES)
    secs = [0.01 + 2e-9 * r.updates * (1 + r.method) for r in sample]
    model = serve.fit_service_model(sample, secs)
    for r, s in zip(sample, secs):
        a, b = model[r.cls]
        assert abs(a + b * r.updates - s) < 1e-9 * max(1.0, s) + 1e-12


def test_one_at_a_time_queue_model():
    lat = serve.fifo_one_at_a_time([0.0, 0.0, 5.0], [1.0, 2.0, 1.0])
    assert lat == [1.0, 3.0, 1.0]
