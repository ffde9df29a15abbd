"""Serving loop on the GPU: requests arriving while others run are admitted and overlap on the
device; every result is the same, bit for bit, as the request run alone and as the oracle
(MPK requests: every power; Chebyshev requests: the filtered block)."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_12525_gb300 as m
    m.build()
    m.load()
    return m


def test_serving_mix_equals_alone(mpk):
    from paper_2405_12525_gb300.serving import GpuBackend, Request, Server, width_bucket
    host = {"lap": gen.laplacian_3d(14, 13, 12), "xxz": gen.xxz_chain(10, stream=601),
            "band": gen.banded_random(3000, stream=602)}
    mats = {}
    for name, A in host.items():
        lo, hi = gen.gershgorin_bounds(A)
        mats[name] = (mpk.CsrMatrix.from_host(A, is_symmetric=True), (hi - lo) / 2 * 1.01, (hi + lo) / 2)
    names = sorted(host)
    gaps = -np.log(gen.uniform(gen.derive_seed(603), 48, 1e-12, 1.0)) / 400.0  # Poisson, 400 / s
    t = np.cumsum(gaps)
    kinds = gen.uniform(gen.derive_seed(604), 48, 0.0, 1.0)
    reqs = []
    for i in range(48):
        name = names[i % 3]
        n = host[name].n
        nrhs = 1 + i % 5
        if kinds[i] < 0.5:
            r = Request(i, float(t[i]), name, "mpk", 2 + i % 7, nrhs)
        else:
            deg = 8 + (i * 5) % 17
            r = Request(i, float(t[i]), name, "cheb", deg, nrhs)
            r.coeffs = gen.uniform(gen.derive_seed(700 + i), deg + 1, -1.0, 1.0) / (1.0 + np.arange(deg + 1))
        r.x = torch.from_numpy(gen.vector(n, nrhs, stream=800 + i)).cuda()
        reqs.append(r)
    srv = Server(GpuBackend(mats, p_max=8, cheb_block=8, streams=6), hbm_budget=2 ** 30, max_inflight=6)
    done = srv.run(reqs)
    assert len(done) == 48 and not srv.rejected
    assert srv.max_seen_inflight >= 2  # requests overlapped on the device
    st = srv.stats()
    assert st["p50_ms"] <= st["p99_ms"]
    levels = {name: mpk.build_levels(A) for name, (A, _, _) in mats.items()}
    for r in done:
        A, scale, shift = mats[r.matrix]
        m = width_bucket(r.nrhs)
        X = torch.zeros((A.n, m), dtype=torch.float64, device="cuda")
        X[:, :r.nrhs] = r.x
        if r.kind == "mpk":
            P = mpk.plan(A, levels[r.matrix], p_max=r.order, nrhs=m)
            alone = P.apply(X, r.order)[..., :r.nrhs]
            want = oracle.mpk(host[r.matrix], r.x.cpu().numpy(), r.order)
            assert np.array_equal(r.result.cpu().numpy().view(np.uint64), want.view(np.uint64))
        else:
            P = mpk.plan(A, levels[r.matrix], p_max=8, nrhs=m)
            alone = P.cheb_filter(X, r.order, r.coeffs, scale=scale, shift=shift)[..., :r.nrhs]
            want = oracle.cheb(host[r.matrix], r.x.cpu().numpy(), r.order, r.coeffs, scale=scale, shift=shift)
            assert np.array_equal(r.result.cpu().numpy().view(np.uint64), want.view(np.uint64))
        P.sync_status()
        assert torch.equal(r.result.contiguous(), alone.contiguous())
