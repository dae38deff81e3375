"""The request server on the GPU: a request gives the same bits alone, in a mixed batch and
through the plain context path; memory-budget admission evicts idle contexts and refuses what
can never fit; requests from several threads all complete."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OBS_KEYS = ["n_prop", "n_acc", "n_meas", "n_meas_q", "clamps", "E", "E2", "m_abs", "m2", "m4", "q", "q_abs",
            "q2", "q4"]


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_06538_gb300 as tn
    tn.build()
    return tn


def _same(a, b):
    for k in OBS_KEYS + ["log_z"]:
        assert a[k] == b[k] or (np.isnan(a[k]) and np.isnan(b[k])), (k, a[k], b[k])
    assert a["build_stats"] == b["build_stats"]


def _context_path(tn, req, precision, n_chains, n_therm, chunk):
    """The same realization through the TNMC context API, sampled in the same steps."""
    seed, L, chi, p, beta, n = req
    J = tn.couplings_pmj(L, [seed], p)
    t = tn.TNMC(L, J, beta, [seed], chi, precision=precision, n_chains=n_chains, n_therm=n_therm)
    lz = t.build_env()
    st = t.build_stats()
    for s0 in range(0, n, chunk):
        t.propose(min(chunk, n - s0), s0, outputs=False)
        t.accept()
    o = t.observables()[0]
    o["log_z"] = float(lz[0])
    o["build_stats"] = [st["max_sweeps"], st["unconverged"], st["total_sweeps"], st["svds"]]
    t.close()
    return o


@pytest.mark.parametrize("precision,L,chi", [("fp64", 10, 4), ("tf32", 16, 16)])
def test_alone_equals_mixed_equals_context_path(tn, precision, L, chi):
    chunk, n_chains, n_therm = 32, 2, 8
    target = (12345, L, chi, 0.109, tn.nishimori_beta(0.109), 75)
    with tn.TNMCServer(precision, n_chains, n_therm, chunk=chunk, max_batch=8, max_inflight=2) as srv:
        alone = srv.wait(srv.submit(*target), timeout=300)
    assert alone["status"] == 0 and alone["batch_size"] == 1
    mix = [(7, L, chi, 0.2, 0.9, 130), target, (99, L, chi, 0.05, 1.3, 20), (5, L, chi, 0.109, 0.6, 75),
           (31, 8, 4, 0.1, 1.0, 40)]
    with tn.TNMCServer(precision, n_chains, n_therm, chunk=chunk, max_batch=8, max_inflight=2,
                       linger_us=200000) as srv:
        ids = [srv.submit(*r) for r in mix]
        res = [srv.wait(i, timeout=300) for i in ids]
        stats = srv.stats()
    assert all(r["status"] == 0 for r in res)
    mixed = res[1]
    assert mixed["batch_size"] == 4          # the four requests of (L, chi) ran together
    _same(alone, mixed)
    ref = _context_path(tn, target, precision, n_chains, n_therm, chunk)
    _same(alone, ref)
    assert alone["n_prop"] == n_chains * 75
    assert stats["completed"] == len(mix) and stats["failed"] == 0 and stats["launches"] > 0
    for r in res:
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]


def test_budget_evicts_idle_contexts_and_refuses_what_cannot_fit(tn):
    import ctypes
    from paper_2409_06538_gb300 import _capi
    lib = _capi.load()
    opts = _capi.Opts(_capi.PRECISIONS["fp64"], 2, 0, None)
    need = lambda L, chi, R: lib.tnmc_estimate_device_bytes(L, R, chi, ctypes.byref(opts), 16)
    budget = max(need(12, 4, 2), need(10, 8, 2)) + 1024   # room for one context at a time
    with tn.TNMCServer("fp64", 2, 0, chunk=16, max_batch=2, max_inflight=2, mem_budget=budget) as srv:
        a = [srv.submit(s, 12, 4, 0.1, 1.0, 20) for s in range(3)]
        b = [srv.submit(s, 10, 8, 0.1, 1.0, 20) for s in range(3)]
        big = srv.submit(1, 64, 32, 0.1, 1.0, 20)           # never fits this budget
        res = {i: srv.wait(i, timeout=300) for i in a + b + [big]}
        st = srv.stats()
    assert all(res[i]["status"] == 0 for i in a + b)
    assert res[big]["status"] == 2 and res[big]["batch_size"] == 0     # TNMC_ERR_OOM
    assert st["contexts_evicted"] >= 1 and st["peak_bytes"] <= budget
    # the eviction did not change results: equal seeds give equal bits across buckets' reruns
    with tn.TNMCServer("fp64", 2, 0, chunk=16, max_batch=2, max_inflight=2) as srv:
        again = srv.wait(srv.submit(0, 12, 4, 0.1, 1.0, 20), timeout=300)
    _same(res[a[0]], again)


def test_many_threads_submit_and_wait(tn):
    out, errs = {}, []
    with tn.TNMCServer("fp32", 2, 0, chunk=64, max_batch=16, max_inflight=3) as srv:
        def client(t):
            try:
                ids = [(srv.submit(1000 * t + k, 8, 4, 0.109, 0.8, 50 + 10 * k), 50 + 10 * k) for k in range(6)]
                for i, n in ids:
                    out[i] = (n, srv.wait(i, timeout=300))
            except Exception as e:  # pragma: no cover - reported below
                errs.append(e)
        th = [threading.Thread(target=client, args=(t,)) for t in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        srv.drain(timeout=60)
        assert srv.poll() == []          # every result was collected by its waiter
        st = srv.stats()
    assert not errs
    assert len(out) == 24 and all(r["status"] == 0 for _, r in out.values())
    assert st["completed"] == 24 and st["batches"] >= 2
    for n, r in out.values():
        assert r["n_prop"] == 2 * n and 0 < r["n_acc"] <= r["n_prop"] and r["n_meas"] == 2 * n


def test_invalid_request_is_refused(tn):
    with tn.TNMCServer("fp64", 1, 0, chunk=8, max_batch=2, max_inflight=1) as srv:
        with pytest.raises(tn._capi.TnmcError):
            srv.submit(1, 8, 64, 0.1, 1.0, 10)       # chi above the compiled maximum
        with pytest.raises(tn._capi.TnmcError):
            srv.submit(1, 8, 4, 1.5, 1.0, 10)        # p outside [0, 1]
        with pytest.raises(tn._capi.TnmcError):
            srv.wait(12345, timeout=0.1)             # unknown id

