"""Pins of the periodic-boundary oracle (Sec. IV: a pinned pair of lines per step): torus energy
closed forms, the region's couplings and fields against the torus energy, exactness when nothing
is truncated, and the exact transition matrix of a truncated step leaving the torus Boltzmann
distribution invariant."""
import itertools

import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import brute, lattice, periodic, sampler


def _torus(L, p, seed):
    return periodic.split_torus(periodic.torus_couplings_pmj(seed, L, p), L)


def _all_torus_states(L):
    return brute.all_states(L, L)


def test_torus_energy_closed_forms():
    for L in (3, 4, 6):
        Jh = np.ones((L, L), dtype=np.int64)
        Jv = np.ones((L, L), dtype=np.int64)
        up = np.ones((L, L), dtype=np.int64)
        assert periodic.torus_energy(up, Jh, Jv) == -2 * L * L          # every bond satisfied
        if L % 2 == 0:
            chk = np.where((np.add.outer(np.arange(L), np.arange(L)) % 2) == 0, 1, -1)
            assert periodic.torus_energy(chk, Jh, Jv) == 2 * L * L     # every bond frustrated
        s = up.copy()
        s[1, 2] = -1                                                     # one flip: four broken bonds
        assert periodic.torus_energy(s, Jh, Jv) == -2 * L * L + 8
    Jh, Jv = _torus(4, 0.3, 5)
    s = np.where(np.random.default_rng(1).random((4, 4)) < 0.5, 1, -1)
    # translation invariance of the torus: shifting spins and couplings together
    assert periodic.torus_energy(np.roll(s, (1, 2), (0, 1)), np.roll(Jh, (1, 2), (0, 1)),
                                 np.roll(Jv, (1, 2), (0, 1))) == periodic.torus_energy(s, Jh, Jv)


@pytest.mark.parametrize("L,i0,j0", [(3, 0, 0), (3, 2, 1), (4, 1, 3), (4, 3, 0)])
def test_region_weight_is_the_torus_weight_up_to_the_fixed_lines(L, i0, j0):
    """For fixed lines, -beta E_torus(s) - [-beta E_reg(x) + H.x] does not depend on the region's
    configuration x: the region's couplings and the fields of the fixed spins account for every
    bond that touches the region."""
    beta = 0.7
    Jh, Jv = _torus(L, 0.3, 11)
    rng = np.random.default_rng(L * 10 + i0 + j0)
    s = np.where(rng.random((L, L)) < 0.5, 1, -1)
    Jh_reg, Jv_reg, H, R, C = periodic.region(Jh, Jv, beta, s, i0, j0)
    diffs = []
    for bits in itertools.product((1, -1), repeat=(L - 1) ** 2):
        x = np.array(bits).reshape(L - 1, L - 1)
        t = s.copy()
        t[np.ix_(R, C)] = x
        diffs.append(-beta * periodic.torus_energy(t, Jh, Jv) - periodic.region_log_weight(x, Jh_reg, Jv_reg, H, beta))
    assert np.ptp(diffs) < 1e-12


def test_untruncated_region_proposals_are_the_exact_conditional():
    """L = 3 (a 2 x 2 region, chi = 2: nothing truncated): q(x | lines) equals the torus Boltzmann
    distribution conditioned on the fixed lines, and every step is accepted."""
    L, beta, chi = 3, 0.8, 2
    Jh, Jv = _torus(L, 0.25, 3)
    S = _all_torus_states(L)
    a = -beta * periodic.torus_energy(S, Jh, Jv)
    rng = np.random.default_rng(7)
    s = np.where(rng.random((L, L)) < 0.5, 1, -1)
    for i0, j0 in ((0, 0), (1, 2), (2, 1)):
        Jh_reg, Jv_reg, H, R, C = periodic.region(Jh, Jv, beta, s, i0, j0)
        env = bm.build_envs(Jh_reg, Jv_reg, beta, chi, H)
        X = brute.all_states(L - 1, L - 1)
        lq = sampler.evaluate(env, X)["logq"]
        # the same conditional from the torus enumeration
        fixed = np.ones(len(S), dtype=bool)
        for r in range(L):
            for c in range(L):
                if r == i0 or c == j0:
                    fixed &= S[:, r, c] == s[r, c]
        sub = S[fixed]
        w = np.exp(a[fixed] - a[fixed].max())
        w /= w.sum()
        idx = {tuple(t[np.ix_(R, C)].ravel()): k for k, t in enumerate(sub)}
        ref = np.array([w[idx[tuple(x.ravel())]] for x in X])
        assert np.abs(np.exp(lq) - ref).max() < 1e-12
    states, acc = periodic.chain(s, Jh, Jv, beta, chi, seed=9, chain_id=0, steps=range(40))
    assert acc.all()


def test_truncated_step_leaves_the_torus_distribution_invariant():
    """L = 3 with chi = 1 (the region's 2 x 2 environments truncated, acceptance below 1): the
    exact transition matrix of one periodic step -- lines uniform over the 3 x 3 choices, proposal
    q(x' | lines) from the truncated environments, Metropolis on the region's conditional weight --
    has the torus Boltzmann distribution as its stationary distribution."""
    L, beta, chi = 3, 0.9, 1
    Jh, Jv = _torus(L, 0.3, 21)
    S = _all_torus_states(L)
    n = len(S)
    a = -beta * periodic.torus_energy(S, Jh, Jv)
    pi = np.exp(a - a.max())
    pi /= pi.sum()
    code = {tuple(t.ravel()): k for k, t in enumerate(S)}
    X = brute.all_states(L - 1, L - 1)
    T = np.zeros((n, n))
    rejected_any = False
    for k in range(n):
        s = S[k]
        for i0 in range(L):
            for j0 in range(L):
                Jh_reg, Jv_reg, H, R, C = periodic.region(Jh, Jv, beta, s, i0, j0)
                env = bm.build_envs(Jh_reg, Jv_reg, beta, chi, H)
                lq = sampler.evaluate(env, X)["logq"]
                lw = periodic.region_log_weight(X, Jh_reg, Jv_reg, H, beta) - lq
                xc = tuple(s[np.ix_(R, C)].ravel())
                cur = [m for m, x in enumerate(X) if tuple(x.ravel()) == xc][0]
                for m, x in enumerate(X):
                    acc = min(1.0, float(np.exp(lw[m] - lw[cur])))
                    rejected_any |= acc < 1.0
                    t = s.copy()
                    t[np.ix_(R, C)] = x
                    pm = np.exp(lq[m]) / (L * L)
                    T[k, code[tuple(t.ravel())]] += pm * acc
                    T[k, k] += pm * (1.0 - acc)
    assert rejected_any
    assert np.abs(T.sum(axis=1) - 1.0).max() < 1e-12
    assert np.abs(pi @ T - pi).max() < 1e-14
