"""Host logic of the C ABI that needs no device: the disorder averages of Sec. III.C
(tnmc_disorder_average) against the oracle's on per-realization thermal means the oracle
produced, with a flagged realization left out; and the Nishimori temperature against the
paper's printed MNP."""
import os

import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import lattice, metropolis, sampler

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nishimori_mnp.txt")


@pytest.fixture(scope="module")
def tn():
    import paper_2409_06538_gb300 as pkg
    pkg.build()
    return pkg


def oracle_realizations(L, p, chi, seeds, n, n_therm):
    """Thermal means of each seeded realization from the oracle's own TNMC run."""
    beta = lattice.nishimori_beta(p)
    per = []
    for s in seeds:
        Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(s, L, p), L)
        env = bm.build_envs(Jh, Jv, beta, chi)
        cs, ce, nacc = [], [], 0
        for ch in range(2):
            pr = sampler.propose(env, s, ch, np.arange(n))
            acc, cur, _ = metropolis.metropolis_chain(pr["energy"], pr["logq"], beta, s, ch, np.arange(n))
            nacc += int(acc[1:].sum())
            cs.append(pr["spins"][cur])
            ce.append(pr["energy"][cur])
        tm = metropolis.thermal_means(metropolis.chain_observables(np.stack(cs), np.stack(ce)), n_therm)
        tm.update(n_prop=2 * n, n_tests=2 * (n - 1), n_acc=nacc, clamps=0, status=0)
        per.append(tm)
    return per


def test_disorder_average_matches_oracle(tn):
    L, p, chi = 4, 0.109, 2
    beta = lattice.nishimori_beta(p)
    per = oracle_realizations(L, p, chi, range(9), 40, 5)
    bad = dict(per[0], E=1e9, m2=7.0, q2=-3.0, status=4)        # a flagged realization: skipped
    got = tn.disorder_average(per + [bad], L, beta)
    ref = metropolis.disorder_average([{k: v for k, v in d.items() if k not in
                                        ("n_prop", "n_tests", "n_acc", "clamps", "status")} for d in per], L, beta)
    assert got["n_used"] == 9 and got["n_dropped"] == 1
    for k in ("E", "E2", "m_abs", "m2", "m4", "q", "q_abs", "q2", "q4", "m_edge", "m_edge_abs", "m_edge2"):
        assert abs(got[k][0] - ref[k][0]) <= 1e-13 * max(1.0, abs(ref[k][0])), k
        assert abs(got[k][1] - ref[k][1]) <= 1e-12 * max(1.0, abs(ref[k][1])), k
    for k in ("U_m", "Q_q", "q2_sq", "chi_q", "chi_edge"):
        assert abs(got[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    assert got["acceptance"] == sum(d["n_acc"] for d in per) / sum(d["n_tests"] for d in per)


def test_disorder_average_no_usable_realization(tn):
    per = oracle_realizations(3, 0.109, 2, [1], 10, 0)
    out = tn.disorder_average([dict(per[0], status=4)], 3, 1.0)
    assert out["n_used"] == 0 and np.isnan(out["U_m"])


def test_nishimori_beta_against_the_printed_mnp(tn):
    """Sec. III.B prints the MNP as (T = 0.9531, p = 0.10926) on exp(-2/T) = p/(1-p)."""
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    assert round(1.0 / tn.nishimori_beta(vals["p"]), 4) == vals["T"]
    for p in (0.05, 0.109, 0.2):
        assert abs(np.tanh(tn.nishimori_beta(p)) - (1 - 2 * p)) < 1e-15
    from paper_2409_06538_gb300 import _capi
    with pytest.raises(_capi.TnmcError):
        tn.nishimori_beta(0.5)
