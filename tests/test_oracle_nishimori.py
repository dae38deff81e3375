"""Pins from the gauge symmetry of the Nishimori line (Sec. III.A): exact disorder
averages by enumerating every bond configuration, the paper's printed MNP temperature,
and the full oracle TNMC (truncated proposals + Metropolis) against those identities."""
import os

import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import brute, lattice, metropolis, sampler

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nishimori_mnp.txt")


def test_paper_mnp_temperature():
    """Sec. III.B quotes the MNP as (T = 0.9531, p = 0.10926); exp(-2/T) = p/(1-p)."""
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    assert round(lattice.nishimori_T(vals["p"]), 4) == vals["T"]
    # the line used by the workloads: tanh(beta) = 1 - 2p
    for p in (0.1, 0.109, 0.13):
        assert abs(np.tanh(lattice.nishimori_beta(p)) - (1 - 2 * p)) < 1e-15


def test_nishimori_identities_by_enumeration():
    """L = 3, all 2^12 bond configurations: [<H>] = -N_B (1 - 2p), [<m^2>] = [<q^2>],
    [<m^4>] = [<q^4>] on the line; off the line the correlation identity fails."""
    L, p = 3, 0.1
    res = brute.nishimori_disorder_average(L, p, lattice.nishimori_beta(p))
    nb = 2 * L * (L - 1)
    assert abs(res["H"] + nb * (1 - 2 * p)) < 1e-10
    assert abs(res["m2"] - res["q2"]) < 1e-12
    assert abs(res["m4"] - res["q4"]) < 1e-12
    off = brute.nishimori_disorder_average(L, p, 0.5 * lattice.nishimori_beta(p))
    assert abs(off["m2"] - off["q2"]) > 1e-3


@pytest.mark.slow
def test_tnmc_oracle_on_nishimori_line():
    """The full oracle (chi = 2 < exact, Metropolis-corrected) on 4x4 at p = 0.109:
    [<H>] = -N_B (1-2p) and [<m^2>] = [<q^2>] within 3 standard errors."""
    L, p, chi, R, n = 4, 0.109, 2, 120, 300
    beta = lattice.nishimori_beta(p)
    per = []
    acc = []
    for seed in range(R):
        J = lattice.couplings_pmj(seed, L, p)
        Jh, Jv = lattice.split_couplings(J, L)
        env = bm.build_envs(Jh, Jv, beta, chi)
        cur_sp, cur_E = [], []
        for chain in range(2):
            pr = sampler.propose(env, seed, chain, np.arange(n))
            a, cur, _ = metropolis.metropolis_chain(pr["energy"], pr["logq"], beta, seed, chain, np.arange(n))
            acc.append(a[1:].mean())
            cur_sp.append(pr["spins"][cur])
            cur_E.append(pr["energy"][cur])
        obs = metropolis.chain_observables(np.stack(cur_sp), np.stack(cur_E))
        per.append(metropolis.thermal_means(obs, 20))
    avg = metropolis.disorder_average(per)
    nb = 2 * L * (L - 1)
    E, seE = avg["E"]
    assert abs(E + nb * (1 - 2 * p)) < 3 * seE
    d = np.array([x["m2"] - x["q2"] for x in per])
    assert abs(d.mean()) < 3 * d.std(ddof=1) / np.sqrt(R)
    assert np.mean(acc) < 1.0
