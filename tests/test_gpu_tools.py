"""GPU checks of the measurement tools: the pilot-based bond-dimension choice."""
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
