"""Metropolis correction of the tensor-network proposals and the sampled observables.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Proposals are independent draws from q (Sec. II.B: each proposal is sampled afresh from the
environments, with no dependence on the current state), so g(s'|s) = q(s') and
Eq. (accptanceratio) becomes
    p_a(s'|s) = min{1, q(s) P(s') / (q(s') P(s))}
              = min{1, exp([-beta E(s') - log q(s')] - [-beta E(s) - log q(s)])},
the form App. A works through for the 1D ring.  Readings where the paper is silent:
the first proposal of a chain is taken as its initial state; a proposal is accepted iff
Delta >= 0 or u < exp(Delta), u the Philox uniform of counter
(0, step, chain, PURPOSE_ACCEPT); observables are measured after every step from step
``n_therm`` on.

Observables (Sec. III.C): energy E, magnetisation m = (1/N) sum s, the two-replica
overlap q = (1/N) sum s^(1) s^(2) between chains 0 and 1 at the same step, the edge
magnetisation m_edge (``lattice.edge_magnetisation``), the Binder ratios
U_m = [<m^4>]/[<m^2>]^2 and Q_q = [<q^4>]/[<q^2>]^2 (Eq. eq:binderEA with the denominator
read as [<q^2>]^2; [<q^2>^2] is also returned), the overlap susceptibility
chi_q = (L^2/T) ([<q^2>] - [<q>]^2) (Eq. eq:susEA, with 1/T and the square of the disorder
mean taken as printed) and the edge susceptibility chi_edge = L [<m_edge^2>].
"""
import numpy as np

from . import lattice, philox


def metropolis_chain(energy, logq, beta, seed, chain, steps, state=None):
    """Run the accept/reject over one chain's proposals in step order.

    energy, logq: (n,) of the proposals; state: (E, logq) of the carried-in current state,
    or None (then proposal 0 is taken unconditionally).
    Returns accepted (n,) bool, current (n,) index of the current state after each step
    (-1 = the carried-in state), and the final (E, logq).
    """
    steps = np.asarray(steps, dtype=np.uint64)
    n = len(steps)
    u = philox.uniform(seed, 0, steps, chain, philox.PURPOSE_ACCEPT)
    accepted = np.zeros(n, dtype=bool)
    current = np.zeros(n, dtype=np.int64)
    cur_idx = -1
    cur = state
    for t in range(n):
        if cur is None:
            ok = True
        else:
            delta = (-beta * energy[t] - logq[t]) - (-beta * cur[0] - cur[1])
            ok = bool(delta >= 0.0 or u[t] < np.exp(delta))
        if ok:
            cur = (float(energy[t]), float(logq[t]))
            cur_idx = t
        accepted[t] = ok
        current[t] = cur_idx
    return accepted, current, cur


def chain_observables(spins_cur, energy_cur):
    """Per-step observables of the current states.

    spins_cur: (n_chains, n, Ly, Lx) +-1 current configuration after each step,
    energy_cur: (n_chains, n).  Returns a dict of per-step arrays.
    """
    N = spins_cur.shape[-1] * spins_cur.shape[-2]
    m = spins_cur.reshape(spins_cur.shape[0], spins_cur.shape[1], -1).sum(axis=-1) / N
    out = dict(E=energy_cur.astype(np.float64), m=m, m_edge=lattice.edge_magnetisation(spins_cur))
    if spins_cur.shape[0] >= 2:
        a = spins_cur[0].reshape(spins_cur.shape[1], -1)
        b = spins_cur[1].reshape(spins_cur.shape[1], -1)
        out['q'] = (a * b).sum(axis=-1) / N
    return out


def thermal_means(obs, n_therm):
    """Thermal means of one realization over steps >= n_therm (chains pooled for E, m)."""
    E = obs['E'][:, n_therm:]
    m = obs['m'][:, n_therm:]
    me = obs['m_edge'][:, n_therm:]
    res = dict(E=E.mean(), E2=(E ** 2).mean(), m_abs=np.abs(m).mean(),
               m2=(m ** 2).mean(), m4=(m ** 4).mean(),
               m_edge=me.mean(), m_edge_abs=np.abs(me).mean(), m_edge2=(me ** 2).mean())
    if 'q' in obs:
        q = obs['q'][n_therm:]
        res.update(q=q.mean(), q_abs=np.abs(q).mean(), q2=(q ** 2).mean(), q4=(q ** 4).mean())
    return res


def disorder_average(per_real, L=None, beta=None):
    """Disorder means [.] and standard errors over realizations, plus Binder ratios and,
    given L (and beta for chi_q), the susceptibilities chi_q and chi_edge."""
    keys = per_real[0].keys()
    R = len(per_real)
    out = {}
    for k in keys:
        x = np.array([d[k] for d in per_real])
        out[k] = (x.mean(), x.std(ddof=1) / np.sqrt(R) if R > 1 else 0.0)
    out['U_m'] = out['m4'][0] / out['m2'][0] ** 2
    if 'q2' in out:
        out['Q_q'] = out['q4'][0] / out['q2'][0] ** 2
        out['q2_sq'] = float(np.mean([d['q2'] ** 2 for d in per_real]))
        if L is not None and beta is not None:
            out['chi_q'] = L * L * beta * (out['q2'][0] - out['q'][0] ** 2)
    if L is not None and 'm_edge2' in out:
        out['chi_edge'] = L * out['m_edge2'][0]
    return out
