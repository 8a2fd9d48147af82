"""Serving: every served request equals the oracle on its seeded input, bit for bit, in the mix."""
import numpy as np
import pytest

import oracle
from paper_2010_04868_gb300 import inputs, serve

pytestmark = pytest.mark.gpu


def _oracle(r):
    return oracle.run(inputs.grid(r.seed, r.ext), r.T, dim=r.dim, shape=r.shape, r=1,
                      weights=serve.class_weights(r.cls), method=r.method)


def _serve(reqs, slots, cap, rate):
    serve.poisson_arrivals(reqs, rate=rate)
    ex = serve.GpuExecutor(slots, cap, keep_results=[r.rid for r in reqs])
    serve.prepare(ex, reqs)
    st = serve.Server(ex, slots=slots, mem_cap=cap).serve(reqs)
    ex.close()
    assert st.completed == len(reqs) and st.rejected == 0
    return ex.results


def test_device_inputs_equal_the_seeded_host_grids():
    import torch
    for ext in [(4099,), (37, 130), (9, 10, 33)]:
        u = torch.empty(ext, dtype=torch.float64, device="cuda")
        inputs.grid_into(u, 12345 + len(ext), chunk=1000)
        assert np.array_equal(u.cpu().numpy(), inputs.grid(12345 + len(ext), ext))


def test_small_requests_in_the_mix_equal_the_oracle():
    """The first 48 requests of the recipe, shrunk so the oracle takes them all in seconds, served
    concurrently on 6 slots: each result against the oracle."""
    reqs = []
    for r in serve.request_mix(48):
        if r.dim == 1:
            ext = (max(64, r.ext[0] // 256),)
        elif r.dim == 2:
            ext = (max(9, r.ext[0] // 32),) * 2
        else:
            ext = (max(8, r.ext[0] // 8),) * 3
        reqs.append(serve.Request(r.rid, r.method, r.dim, r.shape, ext, min(r.T, 40), r.seed))
    results = _serve(reqs, slots=6, cap=2 * 10 ** 9, rate=5000.0)
    for r in reqs:
        ref = _oracle(r)
        assert np.array_equal(results[r.rid].view(np.uint64), ref.view(np.uint64)), r


def test_seeded_one_percent_of_the_mix_at_full_size_equals_the_oracle():
    """A seeded 1 % subset of the first 2000 requests at their drawn extents (up to 384^3 and 4096^2),
    T cut to 8 so that the oracle finishes, served concurrently: each result against the oracle."""
    mix = serve.request_mix(2000)
    pick = inputs.uniform(inputs.SEED_BASE + 41, len(mix)) < 0.01
    reqs = [serve.Request(r.rid, r.method, r.dim, r.shape, r.ext, min(r.T, 8), r.seed)
            for r, p in zip(mix, pick) if p]
    assert len(reqs) >= 10
    results = _serve(reqs, slots=8, cap=16 * 10 ** 9, rate=2000.0)
    for r in reqs:
        ref = _oracle(r)
        assert np.array_equal(results[r.rid].view(np.uint64), ref.view(np.uint64)), r
