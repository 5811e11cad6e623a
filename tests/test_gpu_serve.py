"""Serving: continuous batching of distance queries over device-resident
labels.  Each request's answers must be identical whether it is served alone
or mixed with many concurrent requests of other sizes, and equal to the
oracle's landmark query."""
import threading

import numpy as np
import pytest

import oracle as O
from paper_2410_17226_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__ as ge

    ge.build()
    from paper_2410_17226_gb300 import cbfs

    off, adj = I.rmat(12, seed=17)
    clusters, d = I.degree_clusters(off, adj, 12)
    g = cbfs.Graph(off, adj)
    dist, masks = g.run_batched(clusters, d)
    L = cbfs.Labels(g.n, len(clusters), d)
    ks = [len(S) for S in clusters]
    L.append(dist, masks, ks)
    torch.cuda.synchronize()
    return cbfs, g, L, dist.cpu().numpy(), cbfs.as_numpy_u64(masks), ks


def make_requests(n, count, seed, max_pairs):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, n, size=(int(rng.integers(1, max_pairs + 1)), 2)).astype(np.int32) for _ in range(count)]


def test_alone_equals_in_the_mix_and_oracle(setup):
    cbfs, g, L, dist, masks, ks = setup
    from paper_2410_17226_gb300.serve import QueryServer

    reqs = make_requests(g.n, 60, seed=1, max_pairs=3000)
    reqs.append(np.zeros((0, 2), np.int32))
    alone = []
    with QueryServer(L, max_batch=1024, slots=2) as srv:
        for r in reqs:
            alone.append(srv.submit(r).result())  # one request in flight at a time
    mixed = [None] * len(reqs)
    with QueryServer(L, max_batch=1024, slots=4, memory_budget_bytes=3 * 1024 * 10) as srv:
        futs = {}

        def client(lo, hi):
            for i in range(lo, hi):
                futs[i] = srv.submit(reqs[i])

        ts = [threading.Thread(target=client, args=(i, min(i + 16, len(reqs)))) for i in range(0, len(reqs), 16)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        for i, f in futs.items():
            mixed[i] = f.result()
        st = srv.stats()
    assert st["requests"] == len(reqs) - 1 or st["requests"] == len(reqs)
    assert st["batches"] >= 2
    for r, a, m in zip(reqs, alone, mixed):
        assert a.dtype == np.uint16 and a.shape == (r.shape[0],)
        assert (a == m).all()
        if r.shape[0]:
            assert (a == O.query(dist, masks, ks, r)).all()


def test_large_request_split_over_batches(setup):
    cbfs, g, L, dist, masks, ks = setup
    from paper_2410_17226_gb300.serve import QueryServer

    big = np.random.default_rng(3).integers(0, g.n, size=(5000, 2)).astype(np.int32)
    with QueryServer(L, max_batch=512, slots=2) as srv:
        got = srv.submit(big).result()
        assert srv.stats()["batches"] >= 10
    assert (got == O.query(dist, masks, ks, big)).all()


def test_poisson_load_reports_latency(setup):
    cbfs, g, L, dist, masks, ks = setup
    from paper_2410_17226_gb300.serve import QueryServer, poisson_load

    with QueryServer(L, max_batch=4096, slots=3, pause_gc=True, switch_interval_s=1e-4) as srv:
        futs, offered, elapsed = poisson_load(srv, g.n, rate_rps=400.0, duration_s=0.5, max_pairs=2000, seed=5)
        st = srv.stats()
    assert st["requests"] == len(futs)
    assert st["pairs"] == offered
    assert st["p99_ms"] >= st["p50_ms"] >= 0


def test_server_restores_interpreter_settings(setup):
    import gc
    import sys

    cbfs, g, L, dist, masks, ks = setup
    from paper_2410_17226_gb300.serve import QueryServer

    before = (gc.isenabled(), sys.getswitchinterval())
    with QueryServer(L, max_batch=256, slots=1, pause_gc=True, switch_interval_s=2e-4) as srv:
        assert not gc.isenabled() and abs(sys.getswitchinterval() - 2e-4) < 1e-9
        srv.submit(np.zeros((3, 2), np.int32)).result()
    assert (gc.isenabled(), sys.getswitchinterval()) == before


def test_page_locked_requests_and_answer_buffers(setup):
    """Requests and answer buffers in page-locked memory are copied by DMA
    (no host copy in the server); pageable and page-locked requests mixed in
    one server give the oracle's answers."""
    cbfs, g, L, dist, masks, ks = setup
    from paper_2410_17226_gb300.serve import QueryServer, RequestPool

    reqs = make_requests(g.n, 40, seed=9, max_pairs=5000)
    pinned = []
    for r in reqs[::2]:
        p = cbfs.pinned_empty(r.shape, torch.int32).numpy()
        p[:] = r
        pinned.append(p)
    outs = [cbfs.pinned_empty(r.shape[0], torch.int16).numpy().view(np.uint16) for r in reqs[::2]]
    with QueryServer(L, max_batch=4096, slots=3) as srv:
        futs = []
        for i, r in enumerate(reqs):
            if i % 2 == 0:
                futs.append(srv.submit(pinned[i // 2], out=outs[i // 2]))
            else:
                futs.append(srv.submit(r))
        got = [f.result() for f in futs]
    for i, (r, a) in enumerate(zip(reqs, got)):
        assert (a == O.query(dist, masks, ks, r)).all(), i
        if i % 2 == 0:
            assert a is outs[i // 2]
    # the load generator's page-locked pool: answers equal the oracle's
    pool = RequestPool(g.n, 3000, seed=4, pinned=True, ring=8)
    with QueryServer(L, max_batch=2048, slots=2) as srv:
        t = pool.submit(srv, 100, 2500)
        a = t.result().copy()
    assert (a == O.query(dist, masks, ks, pool.pairs[100:2600])).all()
    with QueryServer(L, max_batch=16, slots=1) as srv:
        with pytest.raises(ValueError):
            srv.submit(reqs[1], out=np.empty(3, np.uint16))
