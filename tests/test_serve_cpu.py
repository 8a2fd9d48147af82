"""Scheduler of the serving loop, driven by a simulated executor (no GPU)."""
from paper_2010_04868_gb300 import serve


def test_request_mix_follows_the_recipe():
    reqs = serve.request_mix(400)
    assert len(reqs) == 400
    for r in reqs:
        assert r.dim in (1, 2, 3) and 10 <= r.T <= 500
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
    assert ex.max_inflight <= 4
    assert len(st.latencies_ms) == st.completed
    assert min(st.latencies_ms) >= 0.0


def test_one_at_a_time_queue_model():
    lat = serve.fifo_one_at_a_time([0.0, 0.0, 5.0], [1.0, 2.0, 1.0])
    assert lat == [1.0, 3.0, 1.0]
