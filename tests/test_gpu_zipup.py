"""GPU parity of the zip-up compression (tnmc_compression TNMC_COMPRESS_ZIPUP) against the
oracle's zip-up (`oracle.boundary_mps.build_envs(method="zipup")`) on the same seeded inputs:
log Z, per-site conditionals teacher-forced on the GPU's own proposals, log q, spins, energies.
Covers rows swept in both directions (mirrored rows), ragged bond dimensions, external fields,
the chi = 64 build and the reduced-precision paths."""
import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import lattice, sampler
from tests.gpu_helpers import (ABS_REDUCED, REL_FP64, assert_logq_within_site_tolerance, assert_qplus_close,
                               check_spins_match)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tn():
    import paper_2409_06538_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    return pkg


def _zip_envs(seed, L, p, chi, H=None):
    beta = lattice.nishimori_beta(p)
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(seed, L, p), L)
    return bm.build_envs(Jh, Jv, beta, chi, H, method="zipup")


# Cases are chosen with a gap at the cut: at L = 13, chi = 5 (seed 3) a near-degenerate pair of
# singular values is split, and the oracle itself moves by 4e-5 in q(+) between two LAPACK SVD
# drivers, so no FP64 tolerance applies there; chi = 7 on the same lattice agrees to 5e-13.
@pytest.mark.parametrize("precision,L,chi,fields", [
    ("fp64", 8, 16, False),          # nothing truncated
    ("fp64", 12, 8, False), ("fp64", 13, 7, False), ("fp64", 16, 16, False), ("fp64", 12, 8, True),
    ("fp32", 16, 8, False), ("tf32", 24, 16, False), ("tf32", 20, 32, False),
    ("fp32", 16, 64, False),         # the chi = 64 build (M in global scratch)
])
def test_zipup_parity(tn, precision, L, chi, fields):
    p = 0.109
    beta = lattice.nishimori_beta(p)
    seeds = [3, 11]
    n = 4
    J = tn.couplings_pmj(L, seeds, p)
    ctx = tn.TNMC(L, J, [beta] * len(seeds), seeds, chi, precision=precision, n_chains=2,
                  compression="zipup")
    k = None
    if fields:
        k = np.random.default_rng(L).integers(-2, 3, size=(len(seeds), L, L)).astype(np.int8)
        ctx.set_fields(k)
    lz = ctx.build_env()
    out = ctx.propose(n, 2)
    spins = ctx.spins().cpu().numpy()
    lq = out["logq"].cpu().numpy()
    E = out["energy"].cpu().numpy()
    lq_tf, qp_tf = ctx.eval_conditionals(torch.from_numpy(spins.reshape(len(seeds), 2 * n, L, L)).cuda())
    lq_tf = lq_tf.cpu().numpy().reshape(len(seeds), 2, n)
    qp_tf = qp_tf.cpu().numpy().reshape(len(seeds), 2, n, L, L)
    tol = REL_FP64 if precision == "fp64" else ABS_REDUCED
    for r, s in enumerate(seeds):
        env = _zip_envs(s, L, p, chi, None if k is None else beta * k[r].astype(np.float64))
        assert abs(lz[r] - env.log_z) < (1e-11 if precision == "fp64" else 1e-4) * abs(env.log_z)
        if L == 8:       # untruncated: the canonical compression gives the same log Z
            canon = bm.build_envs(env.Jh, env.Jv, beta, chi)
            assert abs(lz[r] - canon.log_z) < 1e-11 * abs(canon.log_z)
        for ch in range(2):
            ev = sampler.evaluate(env, spins[r, ch])
            assert_qplus_close(qp_tf[r, ch], ev["qplus"], precision)
            assert np.abs(lq[r, ch] - lq_tf[r, ch]).max() <= 1e-9 * np.abs(lq_tf[r, ch]).max() + 1e-12
            if precision == "fp64":
                assert np.abs(lq[r, ch] - ev["logq"]).max() <= REL_FP64 * np.abs(ev["logq"]).max() + 1e-10
            else:
                assert_logq_within_site_tolerance(lq[r, ch], ev["logq"], ev["qplus"], spins[r, ch], qp_tf[r, ch])
            assert np.array_equal(E[r, ch], lattice.energy(spins[r, ch], env.Jh.astype(np.int64),
                                                           env.Jv.astype(np.int64)))
            check_spins_match(env, s, ch, np.arange(2, 2 + n), spins[r, ch], ev["qplus"], max(tol, 1e-12))
    assert np.all(ctx.realization_status() == 0)
    ctx.close()


def test_zipup_differs_from_canonical_and_rejects_unknown(tn):
    """When truncating, the two compressions give different environments, both close to the
    untruncated log Z (the sign and size of the truncation error of log Z is not ordered between
    them: it is a sum of errors that can cancel); an unknown compression is an argument error."""
    from paper_2409_06538_gb300 import _capi
    L, p, chi, seeds = 16, 0.109, 4, [5]
    beta = lattice.nishimori_beta(p)
    J = tn.couplings_pmj(L, seeds, p)
    lz = {}
    for comp in ("canonical", "zipup"):
        ctx = tn.TNMC(L, J, [beta], seeds, chi, precision="fp64", compression=comp)
        lz[comp] = float(ctx.build_env()[0])
        ctx.close()
    ctx = tn.TNMC(L, J, [beta], seeds, 32, precision="fp64")
    ref = float(ctx.build_env()[0])
    ctx.close()
    assert abs(lz["zipup"] - lz["canonical"]) > 1e-9 * abs(ref)
    assert max(abs(lz["zipup"] - ref), abs(lz["canonical"] - ref)) < 1e-4 * abs(ref)
    lib = _capi.load()
    opts = _capi.Opts(_capi.PRECISIONS["fp64"], 2, 0, None)
    opts.compression = 7
    Jn = np.ascontiguousarray(J.cpu().numpy())
    b = np.array([beta])
    s = np.array(seeds, dtype=np.uint64)
    ctx = _capi.ctypes.c_void_p()
    code = lib.tnmc_create(L, 1, _capi.ctypes.c_void_p(Jn.ctypes.data), b.ctypes.data_as(_capi.c_double_p),
                           s.ctypes.data_as(_capi.c_uint64_p), chi, _capi.ctypes.byref(opts),
                           _capi.ctypes.byref(ctx))
    assert code == 1 and not ctx.value
