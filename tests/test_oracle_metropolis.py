"""Pins of the oracle's Metropolis step: the 1D periodic-ring example of App. A, the exact
stationary acceptance of an independence sampler, and stationarity of the chain."""
import numpy as np

from oracle import boundary_mps as bm
from oracle import brute, lattice, metropolis, philox, sampler


def _ring_setup(L, beta, n, seed):
    env = bm.build_envs(np.ones((1, L - 1), int), np.zeros((0, L), int), beta, 2)
    pr = sampler.propose(env, seed=seed, chain=0, steps=np.arange(n))
    s = pr["spins"][:, 0, :]
    E_ring = pr["energy"] - s[:, 0] * s[:, -1]      # E_P - E = -s_1 s_L  (App. A)
    return s, E_ring, pr["logq"]


def test_ring_acceptance_closed_form():
    """Sampling the periodic ring with the open-chain sampler: p_a = min{1,
    exp(beta s'_1 s'_L) / exp(beta s_1 s_L)} (Eq. eq:accptanceoned)."""
    L, beta, n, seed = 10, 0.8, 3000, 9
    s, E_ring, logq = _ring_setup(L, beta, n, seed)
    acc, cur, _ = metropolis.metropolis_chain(E_ring, logq, beta, seed, 0, np.arange(n))
    u = philox.uniform(seed, 0, np.arange(n, dtype=np.uint64), 0, philox.PURPOSE_ACCEPT)
    c = 0
    want = [True]
    for t in range(1, n):
        ratio = np.exp(beta * s[t, 0] * s[t, -1]) / np.exp(beta * s[c, 0] * s[c, -1])
        ok = ratio >= 1.0 or u[t] < ratio
        want.append(ok)
        if ok:
            c = t
    assert np.array_equal(acc, np.array(want))
    assert 0.3 < acc.mean() < 1.0


def test_ring_stationary_distribution():
    """The corrected chain samples the ring's Boltzmann distribution (chi^2 over E_P)."""
    L, beta, n, seed = 6, 0.9, 60000, 2
    s, E_ring, logq = _ring_setup(L, beta, n, seed)
    acc, cur, _ = metropolis.metropolis_chain(E_ring, logq, beta, seed, 0, np.arange(n))
    Ecur = E_ring[cur]
    # exact ring distribution of E_P over the 2^L states
    X = brute.row_configs(L)
    Eall = -(X[:, :-1] * X[:, 1:]).sum(axis=1) - X[:, 0] * X[:, -1]
    vals = np.unique(Eall)
    w = np.array([np.exp(-beta * Eall[Eall == v]).sum() for v in vals])
    P = w / w.sum()
    counts = np.array([(Ecur == v).sum() for v in vals])
    chi2 = ((counts - P * n) ** 2 / (P * n)).sum()
    assert chi2 < 30


def test_independence_sampler_exact_acceptance_rate():
    """3x3 lattice, chi = 1 (truncated): the chain's acceptance rate matches the exact
    stationary rate sum_{s,s'} P(s) q(s') min(1, w(s')/w(s)), w = P/q."""
    rng = np.random.default_rng(5)
    Jh = np.where(rng.random((3, 2)) < 0.15, -1, 1)
    Jv = np.where(rng.random((2, 3)) < 0.15, -1, 1)
    beta = 1.0
    env = bm.build_envs(Jh, Jv, beta, 1)
    S, E, logZ, P = brute.exact(Jh, Jv, beta)
    q = np.exp(sampler.evaluate(env, S)["logq"])
    w = P / q
    rate = (P[:, None] * q[None, :] * np.minimum(1.0, w[None, :] / w[:, None])).sum()
    assert rate < 0.99                       # truncation makes it a real test
    n, seed = 30000, 17
    pr = sampler.propose(env, seed=seed, chain=0, steps=np.arange(n))
    acc, cur, _ = metropolis.metropolis_chain(pr["energy"], pr["logq"], beta, seed, 0, np.arange(n))
    assert abs(acc[1:].mean() - rate) < 0.015
    # stationarity: the current state's energy histogram follows P(E)
    Ecur = pr["energy"][cur]
    vals = np.unique(E)
    PE = np.array([P[E == v].sum() for v in vals])
    counts = np.array([(Ecur == v).sum() for v in vals])
    keep = PE * n > 20
    chi2 = ((counts[keep] - PE[keep] * n) ** 2 / (PE[keep] * n)).sum()
    assert chi2 < 3 * keep.sum() + 30


def test_exact_proposals_always_accepted():
    """q = P (untruncated): every proposal is accepted (Delta = 0 up to rounding)."""
    rng = np.random.default_rng(8)
    Jh = np.where(rng.random((4, 3)) < 0.1, -1, 1)
    Jv = np.where(rng.random((3, 4)) < 0.1, -1, 1)
    beta = lattice.nishimori_beta(0.1)
    env = bm.build_envs(Jh, Jv, beta, 4)
    pr = sampler.propose(env, seed=0, chain=0, steps=np.arange(500))
    w = -beta * pr["energy"] - pr["logq"]
    assert np.ptp(w) < 1e-10
    acc, _, _ = metropolis.metropolis_chain(pr["energy"], pr["logq"], beta, 0, 0, np.arange(500))
    # Delta may round to -1e-15; u < exp(Delta) ~ 1 - 1e-15 then fails only if u is that close to 1
    assert acc.mean() == 1.0


def test_carried_state_continues_chain():
    """Splitting a chain into two calls with the carried state gives the same decisions."""
    rng = np.random.default_rng(3)
    Jh = np.where(rng.random((3, 2)) < 0.2, -1, 1)
    Jv = np.where(rng.random((2, 3)) < 0.2, -1, 1)
    env = bm.build_envs(Jh, Jv, 1.0, 1)
    pr = sampler.propose(env, seed=1, chain=1, steps=np.arange(400))
    a_all, _, _ = metropolis.metropolis_chain(pr["energy"], pr["logq"], 1.0, 1, 1, np.arange(400))
    a1, _, st = metropolis.metropolis_chain(pr["energy"][:150], pr["logq"][:150], 1.0, 1, 1, np.arange(150))
    a2, _, _ = metropolis.metropolis_chain(pr["energy"][150:], pr["logq"][150:], 1.0, 1, 1,
                                           np.arange(150, 400), state=st)
    assert np.array_equal(a_all, np.concatenate([a1, a2]))
