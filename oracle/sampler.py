"""Autoregressive proposals q(s) = prod_i q(s_i | s_<i) from the cached environments
(Sec. II.A Eq. approximate_bayes; Sec. II.B sampling in reverse contraction order).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Spins are drawn row by row, top to bottom, each row left to right (sites numbered from
the top left to the bottom right, Sec. II.B).  For row r the fixed spins of row r-1 act
through the vertical Boltzmann matrices as external fields h_c = beta Jv[r-1,c] s_{r-1,c}
(Fig. fig:Z4); external fields of the network (the fixed lines of a periodic step) add to
them.  The process tensors of row r are contracted from the right to the left
with those fields (the right sweep), then each spin's conditional partition function is
the left part with fixed spins, the site tensor and the right part, times the bond
factor to the spin on its left (Fig. fig:ZS4):

    w(y) = exp(h_c s_y + beta Jh[r,c-1] s_{c-1} s_y) * (l_{c-1} B[c]^y) . R_{c+1}(y),

    R_c(y') = sum_y exp(beta Jh[r,c-1] s_{y'} s_y + h_c s_y) B[c]^y R_{c+1}(y),  R_Lx = 1.

Readings where the paper is silent: a negative truncated weight is clamped to zero and
counted; q(+) = w+/(w+ + w-), q(-) = w-/(w+ + w-); the spin is +1 iff u < q(+), u the
Philox uniform of counter (site, step, chain, PURPOSE_SPIN); log q is summed in FP64.
"""
import numpy as np

from . import lattice, philox

SV = np.array([1.0, -1.0])


class NumericError(RuntimeError):
    pass


def sweep_row(Brow, jh_row, h, beta, uniforms=None, forced=None):
    """One row for K proposals at once.

    Brow: list of Lx site tensors (k_c, 2, k_{c+1}); jh_row: Jh[r, :]; h: (K, Lx) fields.
    Exactly one of ``uniforms`` (K, Lx) and ``forced`` (K, Lx) +-1 spins is given.
    Returns spins (K, Lx) +-1, log q of the row (K,), q(+) per site (K, Lx), clamp counts (K,).
    """
    K, Lx = h.shape
    v = [None] * Lx
    R = np.ones((K, 2, 1))                   # R_{Lx}(y) for both y
    for c in range(Lx - 1, -1, -1):
        Bc = Brow[c]
        vc = np.einsum('ayb,Kyb->Kya', Bc, R)     # v_y = B[c]^y R_{c+1}(y)
        v[c] = vc
        if c > 0:
            Rn = np.zeros((K, 2, Bc.shape[0]))
            for yp in range(2):
                for y in range(2):
                    fac = np.exp(beta * jh_row[c - 1] * SV[yp] * SV[y] + h[:, c] * SV[y])
                    Rn[:, yp, :] += fac[:, None] * vc[:, y, :]
            m = np.abs(Rn).max(axis=(1, 2), keepdims=True)
            R = Rn / np.where(m > 0, m, 1.0)
    ell = np.ones((K, 1))
    spins = np.zeros((K, Lx), dtype=np.int64)
    qplus = np.zeros((K, Lx))
    logq = np.zeros(K)
    clamps = np.zeros(K, dtype=np.int64)
    prev = None
    for c in range(Lx):
        expo = h[:, c, None] * SV[None, :]
        if c > 0:
            expo = expo + beta * jh_row[c - 1] * prev[:, None] * SV[None, :]
        w = np.exp(expo) * np.einsum('Ka,Kya->Ky', ell, v[c])
        clamps += (w < 0).sum(axis=1)
        w = np.maximum(w, 0.0)
        tot = w.sum(axis=1)
        if not np.all(np.isfinite(tot) & (tot > 0)):
            raise NumericError(f"conditional weights vanish or are not finite at site {c}")
        qp = w[:, 0] / tot
        qm = w[:, 1] / tot
        qplus[:, c] = qp
        if forced is not None:
            s = np.asarray(forced[:, c]).astype(np.int64)
        else:
            s = np.where(uniforms[:, c] < qp, 1, -1)
        spins[:, c] = s
        with np.errstate(divide='ignore'):
            logq += np.where(s == 1, np.log(qp), np.log(qm))
        idx = (1 - s) // 2
        ell = np.einsum('Ka,aKb->Kb', ell, Brow[c][:, idx, :])
        m = np.abs(ell).max(axis=1, keepdims=True)
        ell = ell / np.where(m > 0, m, 1.0)
        prev = s.astype(np.float64)
    return spins, logq, qplus, clamps


def propose(envs, seed, chain, steps):
    """Draw len(steps) proposals of one chain.  Returns dict with spins (K, Ly, Lx),
    logq (K,), energy (K,), qplus (K, Ly, Lx), clamps (K,)."""
    steps = np.asarray(steps, dtype=np.uint64)
    K = steps.shape[0]
    Ly, Lx = envs.Ly, envs.Lx
    spins = np.zeros((K, Ly, Lx), dtype=np.int64)
    qplus = np.zeros((K, Ly, Lx))
    logq = np.zeros(K)
    clamps = np.zeros(K, dtype=np.int64)
    cols = np.arange(Lx, dtype=np.uint64)
    for r in range(Ly):
        h = np.zeros((K, Lx)) if r == 0 else envs.beta * envs.Jv[r - 1][None, :] * spins[:, r - 1, :]
        if envs.H is not None:
            h = h + envs.H[r][None, :]
        site = np.uint64(r * Lx) + cols
        u = philox.uniform(seed, site[None, :], steps[:, None], chain, philox.PURPOSE_SPIN)
        s, lq, qp, cl = sweep_row(envs.B[r], envs.Jh[r], h, envs.beta, uniforms=u)
        spins[:, r, :] = s
        qplus[:, r, :] = qp
        logq += lq
        clamps += cl
    E = lattice.energy(spins, envs.Jh.astype(np.int64), envs.Jv.astype(np.int64))
    return dict(spins=spins, logq=logq, energy=E, qplus=qplus, clamps=clamps)


def evaluate(envs, spins):
    """Teacher-forced q: per-site q(+) (K, Ly, Lx), log q (K,), clamps, for given spins."""
    spins = np.asarray(spins).astype(np.int64)
    K, Ly, Lx = spins.shape
    qplus = np.zeros((K, Ly, Lx))
    logq = np.zeros(K)
    clamps = np.zeros(K, dtype=np.int64)
    for r in range(Ly):
        h = np.zeros((K, Lx)) if r == 0 else envs.beta * envs.Jv[r - 1][None, :] * spins[:, r - 1, :]
        if envs.H is not None:
            h = h + envs.H[r][None, :]
        _, lq, qp, cl = sweep_row(envs.B[r], envs.Jh[r], h, envs.beta, forced=spins[:, r, :])
        qplus[:, r, :] = qp
        logq += lq
        clamps += cl
    return dict(logq=logq, qplus=qplus, clamps=clamps)


def spin_uniforms(seed, chain, steps, Ly, Lx):
    """The Philox uniforms a proposal consumes, (K, Ly*Lx)."""
    steps = np.asarray(steps, dtype=np.uint64)
    site = np.arange(Ly * Lx, dtype=np.uint64)
    return philox.uniform(seed, site[None, :], steps[:, None], chain, philox.PURPOSE_SPIN)
