"""GPU checks of the tools around the method: the pilot-based bond-dimension choice, the bounded-wait
failure detection and the caller-supplied device allocator."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_06538_gb300 as tn
    tn.build()
    return tn


def test_chi_autotuning_prefers_the_cheapest_accepted_proposal(tn):
    """The pilot-based chi choice returns a candidate, every pilot reports p_a in [0, 1], and
    the chosen chi has the least time per accepted proposal among the pilots that completed."""
    from paper_2409_06538_gb300 import acceptance_sweep as sw
    best, table = sw.tune_chi(32, 0.10926, chis=(4, 16), R=4, n=40)
    assert best in (4, 16) and len(table) == 2
    for r in table:
        assert r["failed_realizations"] > 0 or 0.0 <= r["p_a"] <= 1.0
    costs = {r["chi"]: r["s_per_accepted"] for r in table}
    assert costs[best] == min(costs.values())


def test_bounded_wait_times_out_and_the_context_survives(tn):
    """Failure detection without a fault: the sampler's bounded mbarrier wait, run on a barrier
    that nothing arrives on, gives up, the kernel records TNMC_ERR_TIMEOUT and returns; with one
    arrival it succeeds; afterwards the same CUDA context still runs a full build."""
    import ctypes
    import numpy as np
    from paper_2409_06538_gb300 import _capi
    lib = _capi.load()
    us = ctypes.c_int64(-1)
    assert lib.tnmc_selftest_bounded_wait(1, ctypes.byref(us)) == 0
    assert lib.tnmc_selftest_bounded_wait(0, ctypes.byref(us)) == 5      # TNMC_ERR_TIMEOUT
    assert 0 <= us.value < 1_000_000                                     # gave up within a second
    J = tn.couplings_pmj(6, [1, 2], 0.1)
    t = tn.TNMC(6, J, 1.0, [1, 2], 4, precision="fp64")
    assert np.isfinite(t.build_env()).all()
    t.propose(8, 0, outputs=False)
    t.accept()
    assert all(o["n_prop"] == 16 for o in t.observables())
    t.close()


def test_device_memory_comes_from_the_callers_allocator():
    """With the Python binding's default allocator every device buffer of a context comes from
    PyTorch's caching allocator through tnmc_opts.alloc/free (PyTorch's count grows by at least
    the context's bytes and falls back when it is destroyed); with allocator="library" the
    library allocates on its own and PyTorch's count does not move."""
    import paper_2409_06538_gb300 as tn
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tn.build()
    L, chi, p = 16, 8, 0.109
    beta = tn.nishimori_beta(p)
    seeds = [3, 4]
    J = tn.couplings_pmj(L, seeds, p)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    ctx = tn.TNMC(L, J, [beta] * 2, seeds, chi, precision="fp32")
    held = ctx.device_bytes()
    assert torch.cuda.memory_allocated() - base >= held > 0
    ctx.build_env()
    ctx.propose(4, 0)
    ctx.accept()
    assert all(o["status"] == 0 for o in ctx.observables())
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    ctx = tn.TNMC(L, J, [beta] * 2, seeds, chi, precision="fp32", allocator="library")
    assert torch.cuda.memory_allocated() == base
    ctx.close()
