"""The +-J random-bond Ising model on an open Ly x Lx square lattice (Sec. III.A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions shared (by specification, not by code) with the CUDA library:
* spin s in {+1, -1}; tensor index 0 <-> +1 and 1 <-> -1 (Sec. II.B, copy tensor).
* Jh[r, c] couples (r, c)-(r, c+1), shape (Ly, Lx-1); Jv[r, c] couples (r, c)-(r+1, c),
  shape (Ly-1, Lx).
* Flat bond index on the square L x L lattice: horizontal b = r*(L-1) + c, vertical
  b = L*(L-1) + r*L + c; the flat coupling array is Jh row-major then Jv row-major.
"""
import numpy as np

from . import philox


def nishimori_beta(p):
    """Inverse temperature on the Nishimori line exp(-2/T) = p/(1-p) with |J| = 1 (Sec. III.A)."""
    return 0.5 * np.log((1.0 - p) / p)


def nishimori_T(p):
    return 1.0 / nishimori_beta(p)


def couplings_pmj(seed, L, p):
    """Flat int8 couplings of one realization: J_b = -1 with probability p, else +1
    (the P(J) of Sec. III.A), bond b drawn from Philox counter (b, 0, 0, PURPOSE_BOND)."""
    nb = 2 * L * (L - 1)
    b = np.arange(nb, dtype=np.uint64)
    u = philox.uniform(seed, b, 0, 0, philox.PURPOSE_BOND)
    return np.where(u < p, -1, 1).astype(np.int8)


def split_couplings(J, L):
    """Flat couplings -> (Jh (L, L-1), Jv (L-1, L)) as int arrays."""
    J = np.asarray(J).astype(np.int64)
    nh = L * (L - 1)
    return J[:nh].reshape(L, L - 1), J[nh:].reshape(L - 1, L)


def energy(s, Jh, Jv):
    """Eq. (E): E(s) = -sum_<ij> J_ij s_i s_j over nearest neighbours, open boundaries.
    s: (..., Ly, Lx) array of +-1; returns an exact integer array."""
    s = np.asarray(s).astype(np.int64)
    eh = (Jh * s[..., :, :-1] * s[..., :, 1:]).sum(axis=(-2, -1))
    ev = (Jv * s[..., :-1, :] * s[..., 1:, :]).sum(axis=(-2, -1))
    return -(eh + ev)


def n_bonds(Ly, Lx):
    return Ly * (Lx - 1) + (Ly - 1) * Lx


def edge_segment(L):
    """0-based positions along one edge that the edge magnetisation sums: the paper's 1-based
    i = L/4 ... 3L/4 inclusive (Sec. III.C, the m_edge equation), i.e. every integer i with
    L/4 <= i <= 3L/4, shifted by one.  Read literally: L/2 + 1 sites when 4 divides L."""
    i = np.arange(1, L + 1)
    return i[(4 * i >= L) & (4 * i <= 3 * L)] - 1


def edge_magnetisation(s):
    """m_edge = (1/(2L)) sum_i (s_{i,1} + s_{1,i} + s_{L,i} + s_{i,L}) over the edge segment,
    for spins s (..., L, L); the 1/(2L) normalisation is the paper's, read literally
    (Sec. III.C)."""
    s = np.asarray(s)
    L = s.shape[-1]
    seg = edge_segment(L)
    tot = (s[..., seg, 0].sum(axis=-1) + s[..., 0, seg].sum(axis=-1) +
           s[..., L - 1, seg].sum(axis=-1) + s[..., seg, L - 1].sum(axis=-1))
    return tot / (2.0 * L)

