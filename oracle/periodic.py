"""Periodic boundaries by a pinned pair of lines (Sec. IV).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

On an L x L torus every step picks a horizontal line (row i0) and a vertical line (column j0),
keeps their spins fixed, and treats the rest -- an (L-1) x (L-1) region with open boundaries --
as in the open-boundary method: the fixed spins act on their neighbours in the region as
external fields, the region's environments are built with those fields, a new region
configuration x' is proposed from them, and it replaces the current one x with the Metropolis
probability of the region's conditional distribution P(x | fixed lines):

    Delta = [-beta E_reg(x') + H.x' - log q(x')] - [-beta E_reg(x) + H.x - log q(x)],
    accept iff Delta >= 0 or u < exp(Delta),

where E_reg is the energy of the bonds inside the region and H the fields of the fixed lines.
The fixed lines are part of the state and do not change during the step, so each step
leaves P(s) on the torus invariant; the choice of lines changes from step to step.

Torus couplings: Jh[r][c] couples (r, c)-(r, c+1 mod L), Jv[r][c] couples (r, c)-(r+1 mod L, c);
the flat array holds Jh row-major then Jv row-major (2 L^2 bonds), drawn like the open
lattice's (J_b = -1 iff u_b < p, counter (b, 0, 0, PURPOSE_BOND)).

Readings where the paper is silent: the lines of step t of chain k are i0 = floor(u L) and
j0 = floor(u' L) with u, u' the uniforms of counters (0, t, k, PURPOSE_LINES) and
(1, t, k, PURPOSE_LINES); region site (r, c) is torus site (i0 + 1 + r, j0 + 1 + c) mod L and its
spin draw uses the region's own site index r (L-1) + c; the accept uniform is the one of the open
method, counter (0, t, k, PURPOSE_ACCEPT).
"""
import numpy as np

from . import boundary_mps as bm
from . import lattice, philox, sampler

PURPOSE_LINES = 3


def torus_couplings_pmj(seed, L, p):
    """Flat int8 couplings of one torus realization: 2 L^2 bonds, J_b = -1 with probability p."""
    b = np.arange(2 * L * L, dtype=np.uint64)
    u = philox.uniform(seed, b, 0, 0, philox.PURPOSE_BOND)
    return np.where(u < p, -1, 1).astype(np.int8)


def split_torus(J, L):
    J = np.asarray(J).astype(np.int64)
    return J[:L * L].reshape(L, L), J[L * L:].reshape(L, L)


def torus_energy(s, Jh, Jv):
    """E(s) = -sum J s s' over the 2 L^2 bonds of the torus (Eq. E with periodic bonds)."""
    s = np.asarray(s).astype(np.int64)
    return -((Jh * s * np.roll(s, -1, axis=-1)).sum(axis=(-2, -1)) +
             (Jv * s * np.roll(s, -1, axis=-2)).sum(axis=(-2, -1)))


def lines(seed, chain, t, L):
    """The pinned row and column of step t of a chain."""
    u0 = float(philox.uniform(seed, 0, t, chain, PURPOSE_LINES))
    u1 = float(philox.uniform(seed, 1, t, chain, PURPOSE_LINES))
    return min(int(u0 * L), L - 1), min(int(u1 * L), L - 1)


def region(Jh, Jv, beta, s, i0, j0):
    """Open-lattice problem of the region left by the lines (i0, j0): its couplings
    (Jh_reg (L-1, L-2), Jv_reg (L-2, L-1)), the fields H (L-1, L-1) of the fixed spins of s on
    their neighbours, and the torus rows and columns of the region."""
    L = Jh.shape[0]
    R = (i0 + 1 + np.arange(L - 1)) % L
    C = (j0 + 1 + np.arange(L - 1)) % L
    Jh_reg = Jh[np.ix_(R, C[:-1])]
    Jv_reg = Jv[np.ix_(R[:-1], C)]
    H = np.zeros((L - 1, L - 1))
    H[0, :] += beta * Jv[i0, C] * s[i0, C]                    # row i0 above the region's first row
    H[-1, :] += beta * Jv[(i0 - 1) % L, C] * s[i0, C]         # row i0 below the region's last row
    H[:, 0] += beta * Jh[R, j0] * s[R, j0]                    # column j0 left of the first column
    H[:, -1] += beta * Jh[R, (j0 - 1) % L] * s[R, j0]         # column j0 right of the last column
    return Jh_reg, Jv_reg, H, R, C


def region_log_weight(x, Jh_reg, Jv_reg, H, beta):
    """log of the region's conditional weight: -beta E_reg(x) + sum H x."""
    return -beta * lattice.energy(x, Jh_reg, Jv_reg) + (np.asarray(x) * H).sum(axis=(-2, -1))


def step(s, Jh, Jv, beta, chi, seed, chain, t):
    """One periodic TNMC step of one chain on state s (L x L, +-1): returns (new state, accepted,
    log q of the proposal, clamps)."""
    L = s.shape[0]
    i0, j0 = lines(seed, chain, t, L)
    Jh_reg, Jv_reg, H, R, C = region(Jh, Jv, beta, s, i0, j0)
    env = bm.build_envs(Jh_reg, Jv_reg, beta, chi, H)
    pr = sampler.propose(env, seed, chain, [t])
    xn = pr["spins"][0]
    xc = s[np.ix_(R, C)]
    lq_cur = sampler.evaluate(env, xc[None])["logq"][0]
    delta = (region_log_weight(xn, Jh_reg, Jv_reg, H, beta) - pr["logq"][0]) - \
            (region_log_weight(xc, Jh_reg, Jv_reg, H, beta) - lq_cur)
    u = float(philox.uniform(seed, 0, t, chain, philox.PURPOSE_ACCEPT))
    ok = bool(delta >= 0.0 or u < np.exp(delta))
    out = s.copy()
    if ok:
        out[np.ix_(R, C)] = xn
    return out, ok, float(pr["logq"][0]), int(pr["clamps"][0])


def chain(s0, Jh, Jv, beta, chi, seed, chain_id, steps):
    """Run steps (global step indices) from state s0; returns the states after every step and
    the accept flags."""
    s = np.asarray(s0).astype(np.int64).copy()
    states, acc = [], []
    for t in steps:
        s, ok, _, _ = step(s, Jh, Jv, beta, chi, seed, chain_id, int(t))
        states.append(s.copy())
        acc.append(ok)
    return np.array(states), np.array(acc)
