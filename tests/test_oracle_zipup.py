"""Pins of the zip-up compression of the oracle (a compression variant of the boundary MPS of
Sec. II.B): exact when nothing is truncated, exact at chi = 1 when beta = 0, equal to a
brute-force TT-SVD of the full vector when its input is canonical from the side the sweep has not
reached, and alternating left- and right-canonical rows."""
import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import brute, lattice


def _random_mps(rng, L, D):
    dims = [1] + [min(D, 2 ** min(c, L - c)) for c in range(1, L)] + [1]
    return [rng.standard_normal((dims[c], 2, dims[c + 1])) for c in range(L)]


def _right_canonical(mps):
    A = [a.copy() for a in mps]
    for c in range(len(A) - 1, 0, -1):
        Dl, _, Dr = A[c].shape
        Q, R = np.linalg.qr(A[c].reshape(Dl, 2 * Dr).T)          # M = R^T Q^T
        A[c] = Q.T.reshape(Q.shape[1], 2, Dr)
        A[c - 1] = np.einsum('lxd,dk->lxk', A[c - 1], R.T)
    return A


def _left_canonical(mps):
    A = [a.copy() for a in mps]
    for c in range(len(A) - 1):
        Dl, _, Dr = A[c].shape
        Q, R = np.linalg.qr(A[c].reshape(Dl * 2, Dr))
        A[c] = Q.reshape(Dl, 2, Q.shape[1])
        A[c + 1] = np.einsum('kd,dxe->kxe', R, A[c + 1])
    return A


def _tt_svd(v, L, chi, left_to_right):
    """Truncated TT-SVD of a full 2**L vector: sequential truncated SVDs of its unfoldings,
    from the left or from the right, returned as the full truncated vector."""
    if not left_to_right:
        return _tt_svd(v.reshape((2,) * L).transpose(range(L - 1, -1, -1)).reshape(-1), L, chi,
                       True).reshape((2,) * L).transpose(range(L - 1, -1, -1)).reshape(-1)
    cores, rest, k = [], v.reshape(1, -1), 1
    for _ in range(L - 1):
        U, S, Vh = np.linalg.svd(rest.reshape(k * 2, -1), full_matrices=False)
        kk = min(chi, S.shape[0])
        cores.append(U[:, :kk].reshape(k, 2, kk))
        rest, k = S[:kk, None] * Vh[:kk], kk
    cores.append(rest.reshape(k, 2, 1))
    return bm.contract_row(cores)


@pytest.mark.parametrize("left_to_right", [True, False])
@pytest.mark.parametrize("L,D,chi", [(6, 8, 3), (8, 16, 5), (8, 16, 2)])
def test_zipup_equals_tt_svd_on_canonical_input(left_to_right, L, D, chi):
    """With no MPO and an input that is left-canonical (right-to-left sweep) or right-canonical
    (left-to-right sweep, the mirrored right-to-left one), every zip-up truncation sees an
    orthonormal remainder, so the result is the TT-SVD of the full vector from the same side."""
    rng = np.random.default_rng(L * 100 + chi)
    mps = _random_mps(rng, L, D)
    mps = _right_canonical(mps) if left_to_right else _left_canonical(mps)
    full = bm.contract_row(mps)
    if left_to_right:                       # the mirrored right-to-left sweep
        out, logs = bm.compress_zipup(bm.mirror(mps), chi)
        out = bm.mirror(out)
    else:
        out, logs = bm.compress_zipup(mps, chi)
    ours = bm.contract_row(out) * np.exp(logs)
    ref = _tt_svd(full, L, chi, left_to_right)
    assert np.abs(ours - ref).max() < 1e-12 * np.abs(ref).max()
    # and the truncation is real: the result differs from the input
    assert np.abs(ref - full).max() > 1e-6 * np.abs(full).max()


@pytest.mark.parametrize("L,seed", [(4, 3), (4, 11), (5, 8)])
def test_zipup_untruncated_is_exact(L, seed):
    """chi >= 2^(L/2): nothing is truncated; log Z equals enumeration and every row
    environment equals the canonical method's as a full vector."""
    beta = 0.7
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(seed, L, 0.25), L)
    _, _, logZ, _ = brute.exact(Jh, Jv, beta)
    ez = bm.build_envs(Jh, Jv, beta, 2 ** L, method="zipup")
    ec = bm.build_envs(Jh, Jv, beta, 2 ** L)
    assert abs(ez.log_z - logZ) < 1e-12 * abs(logZ)
    for r in range(L):
        gz = bm.contract_row(ez.B[r]) * np.exp(ez.lam[r:].sum())
        gc = bm.contract_row(ec.B[r]) * np.exp(ec.lam[r:].sum())
        assert np.abs(gz - gc).max() < 1e-10 * np.abs(gc).max()


def test_zipup_beta_zero_exact_at_chi_one():
    """beta = 0: every row environment is the constant 2^(rows below) (a product state), so a
    bond dimension of one is exact: log Z = L^2 log 2."""
    L = 7
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(1, L, 0.3), L)
    e = bm.build_envs(Jh, Jv, 0.0, 1, method="zipup")
    assert abs(e.log_z - L * L * np.log(2.0)) < 1e-12


def test_zipup_rows_alternate_canonical_forms():
    """The row built from the bond-1 last row is left-canonical (left-to-right sweep), the next
    right-canonical, and so on; the site the sweep ends on carries the norm.  Mirroring a row
    twice is the identity."""
    L, chi = 8, 4
    beta = lattice.nishimori_beta(0.109)
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(4, L, 0.109), L)
    e = bm.build_envs(Jh, Jv, beta, chi, method="zipup")
    for r in range(L - 1):
        B = e.B[r]
        if (L - 2 - r) % 2 == 0:
            for c in range(L - 1):
                M = B[c].reshape(-1, B[c].shape[2])
                assert np.abs(M.T @ M - np.eye(M.shape[1])).max() < 1e-12
            assert abs(np.linalg.norm(B[L - 1]) - 1.0) < 1e-12
        else:
            for c in range(1, L):
                M = B[c].reshape(B[c].shape[0], -1)
                assert np.abs(M @ M.T - np.eye(M.shape[0])).max() < 1e-12
            assert abs(np.linalg.norm(B[0]) - 1.0) < 1e-12
        assert all(np.array_equal(a, b) for a, b in zip(bm.mirror(bm.mirror(B)), B))


def test_zipup_truncated_close_to_canonical():
    """Truncated: zip-up's log Z is within a small tolerance of the untruncated value at the
    same chi as the canonical method's (on this lattice also further from it; that order is not
    general, the truncation errors of log Z can cancel); an unknown method is refused."""
    L, p = 12, 0.109
    beta = lattice.nishimori_beta(p)
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(5, L, p), L)
    ref = bm.build_envs(Jh, Jv, beta, 64).log_z
    for chi in (4, 8):
        dz = abs(bm.build_envs(Jh, Jv, beta, chi, method="zipup").log_z - ref)
        dc = abs(bm.build_envs(Jh, Jv, beta, chi).log_z - ref)
        assert dz < 1e-2 * abs(ref) and dc <= dz
    with pytest.raises(ValueError):
        bm.build_envs(Jh, Jv, beta, 4, method="variational")


@pytest.mark.parametrize("L,seed", [(4, 3), (4, 11)])
def test_sitewise_untruncated_is_exact(L, seed):
    """The literal site-by-site reading (right to left on every row, no canonical form) is exact
    when nothing is truncated: log Z equals enumeration."""
    beta = 0.7
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(seed, L, 0.25), L)
    _, _, logZ, _ = brute.exact(Jh, Jv, beta)
    assert abs(bm.build_envs(Jh, Jv, beta, 2 ** L, method="sitewise").log_z - logZ) < 1e-12 * abs(logZ)


def test_sitewise_rows_right_canonical():
    """Every row of the literal site-by-site reading is swept right to left: right-canonical,
    the norm at site 0; rows after the first equal no zip-up row (the input's canonical side is
    the wrong one)."""
    L, chi = 8, 4
    beta = lattice.nishimori_beta(0.109)
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(4, L, 0.109), L)
    e = bm.build_envs(Jh, Jv, beta, chi, method="sitewise")
    for r in range(L - 1):
        B = e.B[r]
        for c in range(1, L):
            M = B[c].reshape(B[c].shape[0], -1)
            assert np.abs(M @ M.T - np.eye(M.shape[0])).max() < 1e-12
        assert abs(np.linalg.norm(B[0]) - 1.0) < 1e-12
    z = bm.build_envs(Jh, Jv, beta, chi, method="zipup")
    assert abs(z.log_z - e.log_z) > 1e-9 * abs(z.log_z)
