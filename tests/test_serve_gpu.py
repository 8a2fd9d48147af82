"""Serving: every request's result is the same alone and in the mix, bit for bit."""
import pytest

pytestmark = pytest.mark.gpu


def test_results_alone_equal_results_in_the_mix():
    import torch
    from paper_2010_04868_gb300 import serve
    from paper_2010_04868_gb300 import stencil as S
    reqs = [r for r in serve.request_mix(200) if r.points <= 300_000][:30]
    for r in reqs:
        r.T = min(r.T, 60)
    serve.poisson_arrivals(reqs, rate=3000.0)
    ex = serve.GpuExecutor(slots=6, keep_results=True)
    st = serve.Server(ex, slots=6, mem_cap=2 * 10 ** 9).serve(reqs)
    assert st.completed == len(reqs)
    torch.cuda.synchronize()
    for r in reqs:
        u = ex.input_grid(r)
        sc = torch.empty_like(u) if r.method == 0 else None
        s = S.Stencil(r.dim, r.shape, 1, list(serve.weights_for(r)), r.method)
        s.run(u, r.T, sc)
        assert s.status() == 0
        assert torch.equal(u, ex.results[r.rid]), r
        s.close()
