"""Pins of the oracle where TNMC is exact: brute-force enumeration (Eq. P, Z, Bayes)
and the closed forms of App. A (1D chain)."""
import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import brute, lattice, sampler

RNG = np.random.default_rng(20240906)


def _random_bonds(Ly, Lx, p, rng=RNG):
    Jh = np.where(rng.random((Ly, Lx - 1)) < p, -1, 1)
    Jv = np.where(rng.random((Ly - 1, Lx)) < p, -1, 1)
    return Jh, Jv


@pytest.mark.parametrize("Ly,Lx,p", [(3, 3, 0.2), (4, 4, 0.109), (4, 4, 0.0), (2, 5, 0.3), (3, 4, 0.5)])
def test_untruncated_q_equals_boltzmann(Ly, Lx, p):
    """chi >= 2^{floor(Lx/2)}: nothing is truncated, so q(s) = P(s) exactly (Sec. II.A:
    exact conditionals give unbiased samples with acceptance 1)."""
    beta = 0.8 if p == 0.0 else lattice.nishimori_beta(max(p, 0.05))
    Jh, Jv = _random_bonds(Ly, Lx, p)
    chi = 2 ** (Lx // 2)
    env = bm.build_envs(Jh, Jv, beta, chi)
    S, E, logZ, _ = brute.exact(Jh, Jv, beta)
    assert abs(env.log_z - logZ) < 1e-11 * max(1.0, abs(logZ))
    ev = sampler.evaluate(env, S)
    assert np.abs(ev["logq"] + beta * E + logZ).max() < 1e-10
    assert abs(np.exp(ev["logq"]).sum() - 1.0) < 1e-12
    assert ev["clamps"].sum() == 0


def test_sampled_proposals_exact():
    """Proposals drawn from the untruncated sampler satisfy log q = -beta E - log Z."""
    Jh, Jv = _random_bonds(4, 4, 0.15)
    beta = 0.9
    env = bm.build_envs(Jh, Jv, beta, 16)
    _, _, logZ, _ = brute.exact(Jh, Jv, beta)
    pr = sampler.propose(env, seed=11, chain=0, steps=np.arange(64))
    assert np.abs(pr["logq"] + beta * pr["energy"] + logZ).max() < 1e-10
    # the sampler's log q agrees with teacher forcing on its own spins
    ev = sampler.evaluate(env, pr["spins"])
    assert np.abs(ev["logq"] - pr["logq"]).max() < 1e-13
    assert np.abs(ev["qplus"] - pr["qplus"]).max() < 1e-15


def test_sampled_frequencies_match_boltzmann():
    """Empirical frequencies of 40000 exact proposals on a 2x3 lattice follow P (chi^2)."""
    Jh, Jv = _random_bonds(2, 3, 0.3)
    beta = 0.7
    env = bm.build_envs(Jh, Jv, beta, 4)
    S, E, logZ, P = brute.exact(Jh, Jv, beta)
    pr = sampler.propose(env, seed=3, chain=1, steps=np.arange(40000))
    bits = ((1 - pr["spins"].reshape(len(pr["spins"]), -1)) // 2)
    idx = (bits * (1 << np.arange(5, -1, -1))).sum(axis=1)
    counts = np.bincount(idx, minlength=64)
    expct = P * len(idx)
    chi2 = ((counts - expct) ** 2 / expct).sum()
    assert chi2 < 130     # 63 dof, p ~ 1e-6


def test_one_dimensional_closed_forms():
    """App. A: z_i = (2 cosh beta)^{L-i}, Z = 2 (2 cosh beta)^{L-1}, and the conditional
    P(s_{i+1}|s_<i+1) = exp(beta h_i s_{i+1}) z_{i+1}(s_{i+1}) / z_i(h_i) (Eq. onedprob)."""
    L, beta = 9, 0.65
    Jh = np.ones((1, L - 1), dtype=int)
    Jv = np.zeros((0, L), dtype=int)
    env = bm.build_envs(Jh, Jv, beta, 2)
    assert abs(env.log_z - (np.log(2) + (L - 1) * np.log(2 * np.cosh(beta)))) < 1e-12
    s = np.where(RNG.random((5, 1, L)) < 0.5, 1, -1)
    ev = sampler.evaluate(env, s)
    for k in range(5):
        assert abs(ev["qplus"][k, 0, 0] - 0.5) < 1e-15           # z_1(+) = z_1(-)
        for i in range(L - 1):
            h = s[k, 0, i]
            want = np.exp(beta * h) / (2 * np.cosh(beta))     # z_{i+1} constant in s
            assert abs(ev["qplus"][k, 0, i + 1] - want) < 1e-14


def test_random_bond_chain_partition_function():
    """A random-bond open chain: Z = 2 prod_i 2 cosh(beta J_i) (same recursion as App. A)."""
    L, beta = 12, 1.1
    J = np.where(RNG.random(L - 1) < 0.4, -1, 1)
    env = bm.build_envs(J[None, :], np.zeros((0, L), dtype=int), beta, 2)
    want = np.log(2) + np.log(2 * np.cosh(beta * J)).sum()
    assert abs(env.log_z - want) < 1e-12


def test_pure_ising_2x2_closed_form():
    """p = 0 on the 2x2 open lattice (a 4-cycle): Z = 2 e^{4 beta} + 12 + 2 e^{-4 beta}."""
    beta = 0.37
    env = bm.build_envs(np.ones((2, 1), int), np.ones((1, 2), int), beta, 4)
    want = np.log(2 * np.exp(4 * beta) + 12 + 2 * np.exp(-4 * beta))
    assert abs(env.log_z - want) < 1e-13


def test_energy_definition():
    """Eq. (E) on a hand-checked 2x2 configuration."""
    Jh = np.array([[1], [-1]])
    Jv = np.array([[1, -1]])
    s = np.array([[1, -1], [1, 1]])
    # -(Jh00 s00 s01 + Jh10 s10 s11 + Jv00 s00 s10 + Jv01 s01 s11) = -(-1 - 1 + 1 + 1) = 0
    assert lattice.energy(s, Jh, Jv) == 0
    s2 = np.ones((2, 2), int)
    assert lattice.energy(s2, Jh, Jv) == -(1 - 1 + 1 - 1)


def test_coupling_generator_layout_and_rate():
    L, p = 64, 0.109
    J = lattice.couplings_pmj(0, L, p)
    assert J.dtype == np.int8 and J.shape == (2 * L * (L - 1),)
    frac = (J == -1).mean()
    assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / len(J))
    # bond b is decided by Philox counter (b, 0, 0, 0) alone: a prefix is stable in L
    J2 = lattice.couplings_pmj(0, 8, p)
    from oracle import philox
    u = philox.uniform(0, np.arange(len(J2), dtype=np.uint64), 0, 0, philox.PURPOSE_BOND)
    assert np.array_equal(J2, np.where(u < p, -1, 1).astype(np.int8))
    Jh, Jv = lattice.split_couplings(J2, 8)
    assert Jh.shape == (8, 7) and Jv.shape == (7, 8)


@pytest.mark.parametrize("Ly,Lx", [(3, 3), (4, 4), (2, 5)])
def test_untruncated_with_external_fields(Ly, Lx):
    """External fields H (weight exp(-beta E + sum H s)): untruncated environments give
    log Z and q(s) = P(s) of the enumerated distribution with fields, and the fields matter
    (the distribution differs from the field-free one)."""
    rng = np.random.default_rng(Ly * 7 + Lx)
    Jh, Jv = _random_bonds(Ly, Lx, 0.2, rng)
    H = rng.normal(0.0, 0.7, (Ly, Lx))
    beta = 0.85
    env = bm.build_envs(Jh, Jv, beta, 2 ** (Lx // 2), H)
    S, E, logZ, P = brute.exact(Jh, Jv, beta, H)
    assert abs(env.log_z - logZ) < 1e-11 * max(1.0, abs(logZ))
    ev = sampler.evaluate(env, S)
    assert np.abs(np.exp(ev["logq"]) - P).max() < 1e-12
    _, _, _, P0 = brute.exact(Jh, Jv, beta)
    assert np.abs(P - P0).max() > 1e-3
