"""Exhaustive enumeration on small lattices: the definitions the rest of the oracle is
pinned against.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Eq. (P), (Z), (E): Boltzmann weights by summing over all 2**N configurations.
* Eq. (Bayes)/(cond): exact conditionals as ratios of conditional partition functions.
* The environments without the MPS machinery: full 2**Lx row vectors, the row transfer as
  a dense matrix, and the sequential SVD truncation applied to the full vector cut by cut
  from the right (keeping, at the cut before site c, the top-k right singular subspace of
  the current state, k = min(chi, 2**c, 2**(Lx-c))).
* The row-by-row conditionals with clamping, by summing the unnormalised row weight over
  the not-yet-sampled spins of the row.

Configuration index convention: big-endian over sites, bit value 1 <-> spin -1.
"""
import itertools

import numpy as np

from . import lattice


def all_states(Ly, Lx):
    N = Ly * Lx
    idx = np.arange(2 ** N)
    bits = (idx[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1
    return (1 - 2 * bits).reshape(-1, Ly, Lx)


def row_configs(Lx):
    idx = np.arange(2 ** Lx)
    bits = (idx[:, None] >> (Lx - 1 - np.arange(Lx))[None, :]) & 1
    return 1 - 2 * bits                     # (2**Lx, Lx)


def exact(Jh, Jv, beta, H=None):
    """(states, energies, log Z, probabilities) by enumeration; with fields H (Ly, Lx) the
    weight is exp(-beta E(s) + sum H s)."""
    Jh = np.asarray(Jh).astype(np.int64)
    Jv = np.asarray(Jv).astype(np.int64)
    Ly, Lx = Jh.shape[0], Jh.shape[1] + 1
    S = all_states(Ly, Lx)
    E = lattice.energy(S, Jh, Jv)
    a = -beta * E
    if H is not None:
        a = a + (S * np.asarray(H, dtype=np.float64)[None]).sum(axis=(1, 2))
    amax = a.max()
    logZ = amax + np.log(np.exp(a - amax).sum())
    return S, E, logZ, np.exp(a - logZ)


def row_weight(x, jh_row, beta):
    """prod_c exp(beta Jh[r,c] x_c x_{c+1}) for rows x (M, Lx)."""
    return np.exp(beta * (jh_row[None, :] * x[:, :-1] * x[:, 1:]).sum(axis=1))


def transfer(beta, jv_row, jh_below):
    """T[x, y] = prod_c exp(beta Jv[r,c] x_c y_c) * prod_c exp(beta Jh[r+1,c] y_c y_{c+1})."""
    X = row_configs(len(jv_row))
    vert = np.exp(beta * np.einsum('xc,yc,c->xy', X, X, jv_row))
    return vert * row_weight(X, jh_below, beta)[None, :]


def truncate_full(psi, Lx, chi):
    """Sequential SVD truncation of a full row vector, cut by cut from the right."""
    psi = psi.copy()
    for c in range(Lx - 1, 0, -1):
        M = psi.reshape(2 ** c, 2 ** (Lx - c))
        _, _, Vh = np.linalg.svd(M, full_matrices=False)
        k = min(chi, 2 ** c, 2 ** (Lx - c))
        P = Vh[:k].T @ Vh[:k]
        psi = (M @ P).reshape(-1)
    return psi


def envs_full(Jh, Jv, beta, chi):
    """Normalised truncated environments as full vectors Gt_r (2**Lx,) and lam_r, with the
    same normalisation as the MPS oracle (G_r ~ exp(sum_{r'>=r} lam) Gt_r)."""
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    Ly, Lx = Jh.shape[0], Jh.shape[1] + 1
    G = [None] * Ly
    lam = np.zeros(Ly)
    G[Ly - 1] = np.ones(2 ** Lx)
    for r in range(Ly - 2, -1, -1):
        psi = transfer(beta, Jv[r], Jh[r + 1]) @ G[r + 1]
        psi = truncate_full(psi, Lx, chi)
        nrm = np.linalg.norm(psi)
        G[r] = psi / nrm
        lam[r] = np.log(nrm)
    return G, lam


def row_conditionals(G_row, jh_row, h, beta, x):
    """Site-by-site q(+) for one row given the full environment vector, fields h (Lx,) and
    the row's spins x (Lx,): w(y) sums the unnormalised row weight over the spins to the
    right of the site with the spins to the left fixed; negative w is clamped to 0."""
    Lx = len(x)
    X = row_configs(Lx)
    p = G_row * row_weight(X, jh_row, beta) * np.exp(X @ h)
    qp = np.zeros(Lx)
    P = p.reshape((2,) * Lx)
    for c in range(Lx):
        prefix = tuple(int((1 - v) // 2) for v in x[:c])
        sub = P[prefix]                       # axes: site c, then sites > c
        w = sub.reshape(2, -1).sum(axis=1)
        w = np.maximum(w, 0.0)
        qp[c] = w[0] / w.sum()
    return qp


def conditionals_full(G, Jh, Jv, beta, s):
    """q(+) at every site of configuration s (Ly, Lx) and log q(s), from full vectors."""
    Ly, Lx = s.shape
    qp = np.zeros((Ly, Lx))
    for r in range(Ly):
        h = np.zeros(Lx) if r == 0 else beta * np.asarray(Jv[r - 1], dtype=np.float64) * s[r - 1]
        qp[r] = row_conditionals(G[r], np.asarray(Jh[r], dtype=np.float64), h, beta, s[r])
    q_s = np.where(s == 1, qp, 1.0 - qp)
    return qp, np.log(q_s).sum()


def nishimori_disorder_average(L, p, beta):
    """Exact disorder averages [<H>], [<m^2>], [<q^2>], [<m^4>], [<q^4>] on an L x L lattice
    by enumerating every bond configuration with weight p^{n-} (1-p)^{n+}."""
    nb = 2 * L * (L - 1)
    S = all_states(L, L)
    N = L * L
    m = S.reshape(len(S), -1).sum(axis=1) / N
    flat = S.reshape(len(S), -1).astype(np.float64)
    res = dict(H=0.0, m2=0.0, q2=0.0, m4=0.0, q4=0.0)
    for bonds in itertools.product((1, -1), repeat=nb):
        J = np.array(bonds, dtype=np.int64)
        Jh, Jv = lattice.split_couplings(J, L)
        nneg = int((J < 0).sum())
        wdis = p ** nneg * (1 - p) ** (nb - nneg)
        E = lattice.energy(S, Jh, Jv)
        a = -beta * E
        P = np.exp(a - a.max())
        P /= P.sum()
        res['H'] += wdis * (P * E).sum()
        res['m2'] += wdis * (P * m ** 2).sum()
        res['m4'] += wdis * (P * m ** 4).sum()
        C = flat.T @ (P[:, None] * flat)      # <s_i s_j>
        res['q2'] += wdis * (C ** 2).sum() / N ** 2
        # <q^4> for two independent replicas: (1/N^4) sum <s_i s_j s_k s_l>^2
        F = np.einsum('n,ni,nj->nij', np.sqrt(P), flat, flat).reshape(len(S), -1)
        G4 = F.T @ F                         # <s_i s_j s_k s_l> over pairs (ij),(kl)
        res['q4'] += wdis * (G4 ** 2).sum() / N ** 4
    return res
