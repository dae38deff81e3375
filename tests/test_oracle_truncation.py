"""Pins of the truncated (chi < exact) oracle against definitions with no MPS machinery:
full 2^Lx row vectors, the row transfer as a dense matrix and the sequential SVD cut
applied cut by cut to the full vector (Sec. II.B)."""
import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import brute, lattice, sampler

RNG = np.random.default_rng(7)


def _bonds(Ly, Lx, p):
    Jh = np.where(RNG.random((Ly, Lx - 1)) < p, -1, 1)
    Jv = np.where(RNG.random((Ly - 1, Lx)) < p, -1, 1)
    return Jh, Jv


CASES = [(4, 4, 1), (4, 4, 2), (5, 5, 2), (5, 5, 3), (3, 6, 2), (6, 4, 2), (4, 6, 3)]


@pytest.mark.parametrize("Ly,Lx,chi", CASES)
def test_environments_match_full_vector_truncation(Ly, Lx, chi):
    Jh, Jv = _bonds(Ly, Lx, 0.2)
    beta = lattice.nishimori_beta(0.2)
    env = bm.build_envs(Jh, Jv, beta, chi)
    G, lam = brute.envs_full(Jh, Jv, beta, chi)
    for r in range(Ly):
        assert np.abs(bm.contract_row(env.B[r]) - G[r]).max() < 1e-12
    assert np.abs(env.lam - lam).max() < 1e-11
    for r in range(Ly - 1):              # the last row is the exact all-ones environment
        dims = env.bond_dims(r)
        assert max(dims) <= chi
        for c in range(Lx):            # right-canonical sites c >= 1
            if c > 0:
                B = env.B[r][c].reshape(env.B[r][c].shape[0], -1)
                assert np.abs(B @ B.T - np.eye(B.shape[0])).max() < 1e-12


@pytest.mark.parametrize("Ly,Lx,chi", CASES)
def test_conditionals_match_brute_force(Ly, Lx, chi):
    """Site conditionals (with the clamp reading) equal row weights summed over the
    unsampled spins of the row."""
    Jh, Jv = _bonds(Ly, Lx, 0.25)
    beta = lattice.nishimori_beta(0.25)
    env = bm.build_envs(Jh, Jv, beta, chi)
    G, _ = brute.envs_full(Jh, Jv, beta, chi)
    pr = sampler.propose(env, seed=1, chain=0, steps=np.arange(12))
    for k in range(12):
        qp, lq = brute.conditionals_full(G, Jh, Jv, beta, pr["spins"][k])
        assert np.abs(qp - pr["qplus"][k]).max() < 1e-12
        if pr["clamps"][k] == 0:
            assert abs(lq - pr["logq"][k]) < 1e-10


@pytest.mark.parametrize("chi", [1, 2])
def test_q_normalised_over_all_states(chi):
    """Sum_s q(s) = 1 over all 2^16 states of a 4x4 lattice, for a truncated chi."""
    Jh, Jv = _bonds(4, 4, 0.109)
    beta = lattice.nishimori_beta(0.109)
    env = bm.build_envs(Jh, Jv, beta, chi)
    S = brute.all_states(4, 4)
    ev = sampler.evaluate(env, S)
    assert abs(np.exp(ev["logq"]).sum() - 1.0) < 1e-11
    # truncation really changed q: it is not the Boltzmann distribution
    _, E, logZ, _ = brute.exact(Jh, Jv, beta)
    assert np.abs(ev["logq"] + beta * E + logZ).max() > 1e-3


def test_row_marginal_formula():
    """With no clamps, log q(s) = sum_r [log(phi_r(s_{r-1}, s_r) Gt_r(s_r))
    - log sum_x phi_r(s_{r-1}, x) Gt_r(x)]: the site sweep samples each row's marginal."""
    Ly = Lx = 5
    Jh, Jv = _bonds(Ly, Lx, 0.1)
    beta = lattice.nishimori_beta(0.1)
    env = bm.build_envs(Jh, Jv, beta, 2)
    pr = sampler.propose(env, seed=4, chain=1, steps=np.arange(20))
    X = brute.row_configs(Lx)
    for k in range(20):
        if pr["clamps"][k]:
            continue
        s = pr["spins"][k]
        tot = 0.0
        for r in range(Ly):
            Gr = bm.contract_row(env.B[r])
            h = np.zeros(Lx) if r == 0 else beta * Jv[r - 1] * s[r - 1]
            phi = brute.row_weight(X, Jh[r].astype(float), beta) * np.exp(X @ h)
            xi = int(((1 - s[r]) // 2) @ (1 << np.arange(Lx - 1, -1, -1)))
            tot += np.log(phi[xi] * Gr[xi]) - np.log((phi * Gr).sum())
        assert abs(tot - pr["logq"][k]) < 1e-11


def test_log_z_of_truncated_network_is_finite_and_close():
    """log Z from the truncated contraction approximates the exact one (not a pin of
    equality; a sanity bound that catches a dropped log-norm)."""
    Jh, Jv = _bonds(4, 4, 0.109)
    beta = lattice.nishimori_beta(0.109)
    _, _, logZ, _ = brute.exact(Jh, Jv, beta)
    for chi in (2, 3):
        env = bm.build_envs(Jh, Jv, beta, chi)
        assert abs(env.log_z - logZ) < 0.5


def test_doubly_clamped_site_is_an_error():
    """The clamp reading: a negative truncated weight is clamped to zero and counted, and a
    site whose two weights are both clamped (or not finite) is an error, not a draw."""
    beta = 0.7
    B0 = np.array([-1.0, -2.0]).reshape(1, 2, 1)          # both weights of site 0 negative
    B1 = np.array([0.3, 1.1]).reshape(1, 2, 1)
    jh = np.array([1.0, 0.0])
    with pytest.raises(sampler.NumericError):
        sampler.sweep_row([B0, B1], jh, np.zeros((1, 2)), beta, uniforms=np.array([[0.3, 0.5]]))
    with pytest.raises(sampler.NumericError):
        sampler.sweep_row([np.full((1, 2, 1), np.inf), B1], jh, np.zeros((1, 2)), beta,
                          uniforms=np.array([[0.3, 0.5]]))
    # one negative weight is clamped: the other branch is taken with q = 1, two clamps per row
    # here (site 0 has w- < 0; site 1's left vector then carries B0's + entry)
    B0m = np.array([1.0, -2.0]).reshape(1, 2, 1)
    s, lq, qp, cl = sampler.sweep_row([B0m, B1], jh, np.zeros((1, 2)), beta, uniforms=np.array([[0.99, 0.5]]))
    assert s[0, 0] == 1 and qp[0, 0] == 1.0 and cl[0] >= 1
