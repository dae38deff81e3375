"""Row environments of the partition-function network by boundary MPS (Sec. II.B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The network of Fig. fig:2d_tn is contracted from the last row upward.  The environment
of row r is the sum over every spin below row r,

    G_{Ly-1}(x) = 1,
    G_r(x) = sum_y  prod_c exp(beta Jv[r,c] s(x_c) s(y_c))
                  * prod_c exp(beta Jh[r+1,c] s(y_c) s(y_{c+1}))  * G_{r+1}(y),

which is the row-transfer MPO (bond 2: the T tensors of Sec. II.B with the copy tensor
delta and the Boltzmann matrices W absorbed) applied to the MPS of G_{r+1}.  The bond
dimension doubles and is cut back to D = chi by singular value decomposition (Sec. II.B): a
left-to-right Householder-QR sweep brings the MPS to left-canonical form, then a
right-to-left SVD sweep keeps at every bond the min(chi, rows, cols) largest singular
values (no tolerance cut).  The result is stored normalised, G_r ~ exp(Lambda_r) Gt_r
with Lambda_r = sum_{r' >= r} lam[r'], and every row is kept for the sampler, which reuses
the cached process tensors (Sec. II.B).

Site tensors are arrays B[c] of shape (k_c, 2, k_{c+1}); physical index 0 <-> s=+1.
"""
import numpy as np

SV = np.array([1.0, -1.0])   # spin value of tensor index 0 / 1


def row_mpo(beta, jv_row, jh_below, h_below=None):
    """MPO of one row transfer: O[c][a, x, y, b] for the upper spin x (row r), the lower
    spin y (row r+1), left MPO bond a = y_{c-1} and right MPO bond b = y_c.

    jv_row: Jv[r, :] (Lx,), jh_below: Jh[r+1, :] (Lx-1,); h_below: optional external fields
    on the spins of row r+1 (Lx,), entering as the site weight exp(h s(y)).
    """
    Lx = len(jv_row)
    ops = []
    for c in range(Lx):
        Da = 1 if c == 0 else 2
        Db = 1 if c == Lx - 1 else 2
        O = np.zeros((Da, 2, 2, Db))
        for a in range(Da):
            for x in range(2):
                for y in range(2):
                    val = np.exp(beta * jv_row[c] * SV[x] * SV[y])
                    if c > 0:
                        val *= np.exp(beta * jh_below[c - 1] * SV[a] * SV[y])
                    if h_below is not None:
                        val *= np.exp(h_below[c] * SV[y])
                    if c < Lx - 1:
                        O[a, x, y, y] = val          # delta_{b, y}: pass y_c to the right
                    else:
                        O[a, x, y, 0] = val
        ops.append(O)
    return ops


def apply_mpo(ops, mps):
    """MPO x MPS; merged bond index (mpo, mps) -> mpo * D_mps + mps."""
    out = []
    for O, B in zip(ops, mps):
        Da, _, _, Db = O.shape
        Dl, _, Dr = B.shape
        A = np.einsum('axyb,lyr->alxbr', O, B).reshape(Da * Dl, 2, Db * Dr)
        out.append(A)
    return out


def compress(A, chi):
    """QR sweep (left-canonical) then truncating SVD sweep; returns (normalised right-
    canonical MPS, log of the removed scale)."""
    A = [a.copy() for a in A]
    Lx = len(A)
    logs = 0.0
    for c in range(Lx - 1):
        Dl, _, Dr = A[c].shape
        Q, R = np.linalg.qr(A[c].reshape(Dl * 2, Dr))
        nrm = np.linalg.norm(R)
        R = R / nrm
        logs += np.log(nrm)
        A[c] = Q.reshape(Dl, 2, Q.shape[1])
        A[c + 1] = np.einsum('kd,dxe->kxe', R, A[c + 1])
    for c in range(Lx - 1, 0, -1):
        Dl, _, Dr = A[c].shape
        U, S, Vh = np.linalg.svd(A[c].reshape(Dl, 2 * Dr), full_matrices=False)
        k = min(chi, S.shape[0])
        A[c] = Vh[:k].reshape(k, 2, Dr)
        A[c - 1] = np.einsum('lxd,dk->lxk', A[c - 1], U[:, :k] * S[:k])
        nrm = np.linalg.norm(A[c - 1])
        A[c - 1] = A[c - 1] / nrm
        logs += np.log(nrm)
    return A, logs


def compress_zipup(A, chi):
    """Zip-up compression of the MPO x MPS product A, right to left: one truncating SVD sweep
    and no canonicalising QR sweep.  At site c the truncated right part already found is
    contracted into A[c] and the min(chi, rows, cols) largest singular values of the result are
    kept; the sweep relies on the input MPS being left-canonical, so that the part it has not
    reached is close to an isometry (the MPO spoils that a little, which is the approximation).
    Returns (normalised right-canonical MPS, log of the removed scale)."""
    Lx = len(A)
    out = [None] * Lx
    logs = 0.0
    C = np.ones((1, 1))
    for c in range(Lx - 1, 0, -1):
        T = np.einsum('lxd,dk->lxk', A[c], C)                 # (D_left, 2, k_right)
        Dl, _, kr = T.shape
        U, S, Vh = np.linalg.svd(T.reshape(Dl, 2 * kr), full_matrices=False)
        k = min(chi, S.shape[0])
        out[c] = Vh[:k].reshape(k, 2, kr)
        C = U[:, :k] * S[:k]
        nrm = np.linalg.norm(C)
        C = C / nrm
        logs += np.log(nrm)
    T = np.einsum('lxd,dk->lxk', A[0], C)
    nrm = np.linalg.norm(T)
    out[0] = T / nrm
    return out, logs + np.log(nrm)


def mirror(mps):
    """The same row vector with the sites in reverse order: site c becomes site Lx-1-c and its
    bonds swap."""
    return [b.transpose(2, 1, 0) for b in reversed(mps)]


class Envs:
    """Cached row environments: B[r][c] (k_c, 2, k_{c+1}), lam[r], log_z, and the external
    fields H (Ly, Lx) the network was built with (None: no fields)."""

    def __init__(self, B, lam, log_z, Jh, Jv, beta, chi, H=None):
        self.B, self.lam, self.log_z = B, lam, log_z
        self.Jh, self.Jv, self.beta, self.chi, self.H = Jh, Jv, beta, chi, H

    @property
    def Ly(self):
        return len(self.B)

    @property
    def Lx(self):
        return len(self.B[0])

    def bond_dims(self, r):
        return [b.shape[0] for b in self.B[r]] + [1]


def build_envs(Jh, Jv, beta, chi, H=None, method="canonical"):
    """All row environments of the Ly x Lx lattice (Jh (Ly, Lx-1), Jv (Ly-1, Lx)), optionally
    with external fields H (Ly, Lx): the weight of a configuration gains exp(sum H s).

    method "canonical": the QR sweep + truncating SVD sweep of Sec. II.B (compress).
    method "zipup": compress_zipup, alternating the sweep direction from row to row so that
    every row's input is canonical on the side the sweep reaches last: the row built from the
    exact bond-1 last row sweeps left to right (its result is left-canonical), the next one
    right to left, and so on.  A left-to-right row is the right-to-left sweep of the mirrored
    row: reversed couplings (so each horizontal bond factor sits at the bond's right site
    instead of its left one), the mirrored input, and the result mirrored back.
    method "sitewise": the contraction order of Fig. fig:contraction read literally -- the T
    tensors of every row absorbed one at a time from the right, the bond truncated by SVD at
    each absorption, no canonical form -- i.e. compress_zipup right to left on every row."""
    if method not in ("canonical", "zipup", "sitewise"):
        raise ValueError(method)
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    H = None if H is None else np.asarray(H, dtype=np.float64)
    Ly, Lx = Jh.shape[0], Jh.shape[1] + 1
    B = [None] * Ly
    lam = np.zeros(Ly)
    B[Ly - 1] = [np.ones((1, 2, 1)) for _ in range(Lx)]
    for r in range(Ly - 2, -1, -1):
        h = None if H is None else H[r + 1]
        if method == "canonical":
            B[r], lam[r] = compress(apply_mpo(row_mpo(beta, Jv[r], Jh[r + 1], h), B[r + 1]), chi)
        elif method == "sitewise" or (Ly - 2 - r) % 2 == 1:
            B[r], lam[r] = compress_zipup(apply_mpo(row_mpo(beta, Jv[r], Jh[r + 1], h), B[r + 1]), chi)
        else:
            A = apply_mpo(row_mpo(beta, Jv[r][::-1], Jh[r + 1][::-1], None if h is None else h[::-1]),
                          mirror(B[r + 1]))
            Bm, lam[r] = compress_zipup(A, chi)
            B[r] = mirror(Bm)
    log_z = float(lam.sum()) + log_row_sum(B[0], Jh[0], beta, None if H is None else H[0])
    return Envs(B, lam, log_z, Jh, Jv, beta, chi, H)


def log_row_sum(mps, jh_row, beta, h_row=None):
    """log sum_x prod_c exp(beta Jh[0,c] s(x_c) s(x_{c+1}) + h[c] s(x_c)) Gt_0(x): closes the
    network on the top row (Eq. Z), with the top row's own fields when given."""
    f = (lambda c: np.ones(2)) if h_row is None else (lambda c: np.exp(h_row[c] * SV))
    ell = mps[0][0] * f(0)[:, None]          # (2, k1): left vector for each x_0
    logs = 0.0
    for c in range(1, len(mps)):
        W = np.exp(beta * jh_row[c - 1] * np.outer(SV, SV))     # W[x', x]
        ell = np.einsum('pa,px,axb->xb', ell, W, mps[c]) * f(c)[:, None]
        m = np.abs(ell).max()
        ell = ell / m
        logs += np.log(m)
    return logs + np.log(ell.sum())


def contract_row(mps):
    """Full 2**Lx vector Gt(x) of an MPS (big-endian: site 0 is the slowest index)."""
    v = mps[0][0]                            # (2, k1)
    for B in mps[1:]:
        v = np.einsum('...a,axb->...xb', v, B)
    return v.reshape(-1)
