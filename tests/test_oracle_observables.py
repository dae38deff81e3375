"""Pins of the oracle's edge magnetisation and susceptibilities (Sec. III.C): closed forms on
hand-made configurations, lattice symmetries, and a chain with exact proposals against exact
enumeration of one realization."""
import numpy as np

from oracle import boundary_mps as bm
from oracle import brute, lattice, metropolis, sampler


def test_edge_segment_read_literally():
    """i = L/4 ... 3L/4 (1-based, inclusive): L/2 + 1 sites when 4 divides L."""
    assert list(lattice.edge_segment(8)) == [1, 2, 3, 4, 5]
    assert list(lattice.edge_segment(4)) == [0, 1, 2]
    assert list(lattice.edge_segment(6)) == [1, 2, 3]          # 1.5 <= i <= 4.5
    assert len(lattice.edge_segment(256)) == 129


def test_edge_magnetisation_closed_forms():
    L = 8
    up = np.ones((L, L), dtype=np.int64)
    full = 4 * 5 / (2 * L)                                      # four segments of 5 sites
    assert lattice.edge_magnetisation(up) == full
    assert lattice.edge_magnetisation(-up) == -full
    for (r, c), change in (((0, 3), -2), ((0, 0), 0), ((3, 3), 0), ((5, 7), -2), ((7, 1), -2),
                           ((6, 0), 0), ((2, 0), -2)):
        s = up.copy()
        s[r, c] = -1
        assert abs(lattice.edge_magnetisation(s) - (full + change / (2 * L))) < 1e-15, (r, c)
    rng = np.random.default_rng(3)
    for L in (4, 6, 8, 12):
        s = np.where(rng.random((5, L, L)) < 0.5, 1, -1)
        me = lattice.edge_magnetisation(s)
        # transposition swaps the top and left (bottom and right) segments, which share their
        # index set; the literal segment is not centred, so rotations are not symmetries
        assert np.allclose(lattice.edge_magnetisation(np.swapaxes(s, 1, 2)), me)
        assert np.allclose(lattice.edge_magnetisation(-s), -me)
        assert np.allclose(me, [lattice.edge_magnetisation(x) for x in s])


def test_edge_moments_of_an_exact_chain_match_enumeration():
    """L = 4, chi = 4 (untruncated, so q = P and every proposal is an independent exact
    draw): the chain's <m_edge^2> and <|m_edge|> agree with the enumerated Boltzmann
    averages within 4 standard errors."""
    L, p, chi, n = 4, 0.109, 4, 3000
    beta = lattice.nishimori_beta(p)
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(11, L, p), L)
    env = bm.build_envs(Jh, Jv, beta, chi)
    S = brute.all_states(L, L)
    a = -beta * lattice.energy(S, Jh, Jv)
    P = np.exp(a - a.max())
    P /= P.sum()
    me = lattice.edge_magnetisation(S)
    exact2, exact_abs = float((P * me ** 2).sum()), float((P * np.abs(me)).sum())
    cur_sp, cur_E = [], []
    for chain in range(2):
        pr = sampler.propose(env, 11, chain, np.arange(n))
        acc, cur, _ = metropolis.metropolis_chain(pr["energy"], pr["logq"], beta, 11, chain, np.arange(n))
        assert acc.all()
        cur_sp.append(pr["spins"][cur])
        cur_E.append(pr["energy"][cur])
    obs = metropolis.chain_observables(np.stack(cur_sp), np.stack(cur_E))
    tm = metropolis.thermal_means(obs, 0)
    x2 = obs["m_edge"].ravel() ** 2
    xa = np.abs(obs["m_edge"].ravel())
    assert abs(tm["m_edge2"] - exact2) < 4 * x2.std() / np.sqrt(x2.size)
    assert abs(tm["m_edge_abs"] - exact_abs) < 4 * xa.std() / np.sqrt(xa.size)


def test_susceptibility_invariants():
    """chi_q = (L^2/T)([<q^2>] - [<q>]^2) vanishes when every realization has <q^2> = <q>^2
    = c^2, equals (L^2/T)[<q^2>] when [<q>] = 0, and chi_edge = L [<m_edge^2>]."""
    base = dict(E=0.0, E2=0.0, m_abs=0.5, m2=0.3, m4=0.2, m_edge=0.0, m_edge_abs=0.1, m_edge2=0.04)
    L, beta = 16, 0.9
    same = [dict(base, q=0.4, q_abs=0.4, q2=0.16, q4=0.0256) for _ in range(5)]
    assert abs(metropolis.disorder_average(same, L, beta)["chi_q"]) < 1e-12
    sym = [dict(base, q=s * 0.2, q_abs=0.2, q2=0.05 + 0.01 * k, q4=0.01) for k, s in enumerate((1, -1, 1, -1))]
    out = metropolis.disorder_average(sym, L, beta)
    assert abs(out["chi_q"] - L * L * beta * np.mean([d["q2"] for d in sym])) < 1e-12
    assert abs(out["chi_edge"] - L * 0.04) < 1e-15


def _enumerated_realization(L, same_states):
    """Per-step observables over every ordered pair (s, s') of an L x L lattice's states, each
    pair once: chain 0 takes s, chain 1 takes s' (independent uniform replicas, i.e. infinite
    temperature) -- or, with same_states, chain 1 repeats chain 0 (overlap q = 1 at every step)."""
    S = brute.all_states(L, L)
    n = len(S)
    i0 = np.repeat(np.arange(n), n)
    i1 = np.tile(np.arange(n), n)
    if same_states:
        i0 = i1 = np.arange(n)
    cur = np.stack([S[i0], S[i1]])
    return metropolis.thermal_means(metropolis.chain_observables(cur, np.zeros(cur.shape[:2])), 0)


def test_binder_ratios_closed_forms():
    """Eq. eq:binderEA as ratios of disorder means, pinned by closed forms.  N independent
    uniform spins have <m^2> = 1/N and <m^4> = (3N^2 - 2N)/N^4 (the fourth moment of a sum of
    N independent +-1 variables), and the overlap of two independent such replicas has the same
    law.  Realization A is exactly that (every pair of states of a 2 x 2 lattice, N = 4);
    realization B has chain 1 equal to chain 0, so q = 1 at every step while m keeps the
    independent-spin moments; realization C is the fully ordered state (m = q = 1).  The
    ratios of the disorder means differ from the means of per-realization ratios and from the
    other replica's moments, so a per-realization ratio, a swapped q2/q4 or an m/q mix-up fails."""
    L = 2
    N = L * L
    m2, m4 = 1.0 / N, (3.0 * N * N - 2.0 * N) / N ** 4
    A = _enumerated_realization(L, same_states=False)
    B = _enumerated_realization(L, same_states=True)
    for key, want in (("m2", m2), ("m4", m4), ("q2", m2), ("q4", m4)):
        assert abs(A[key] - want) < 1e-15, key
    assert abs(B["m2"] - m2) < 1e-15 and abs(B["m4"] - m4) < 1e-15
    assert abs(B["q2"] - 1.0) < 1e-15 and abs(B["q4"] - 1.0) < 1e-15
    C = dict(A, m_abs=1.0, m2=1.0, m4=1.0, q=1.0, q_abs=1.0, q2=1.0, q4=1.0)
    out = metropolis.disorder_average([A, B])
    assert abs(out["U_m"] - m4 / m2 ** 2) < 1e-13                      # 3 - 2/N = 2.5
    assert abs(out["U_m"] - (3.0 - 2.0 / N)) < 1e-13
    Qq = ((m4 + 1.0) / 2) / ((m2 + 1.0) / 2) ** 2                      # 1.48
    assert abs(out["Q_q"] - Qq) < 1e-13
    assert abs(out["q2_sq"] - (m2 ** 2 + 1.0) / 2) < 1e-15
    out = metropolis.disorder_average([A, C])
    assert abs(out["U_m"] - ((m4 + 1.0) / 2) / ((m2 + 1.0) / 2) ** 2) < 1e-13
    per_real = ((3.0 - 2.0 / N) + 1.0) / 2                              # the wrong reading: 1.75
    assert abs(out["U_m"] - per_real) > 0.2
