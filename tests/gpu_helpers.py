"""Shared helpers of the GPU parity tests: build the same seeded workload on both sides."""
import numpy as np

from oracle import boundary_mps as bm
from oracle import lattice, philox, sampler

# tolerances on per-site conditionals q(+) (teacher forced on the GPU's own spins)
REL_FP64 = 1e-9       # relative, on q(+) and q(-) = 1 - q(+)
ABS_REDUCED = 1e-3    # absolute, FP32 / BF16 / TF32 paths


def oracle_envs(seed, L, p, chi, beta=None):
    beta = lattice.nishimori_beta(p) if beta is None else beta
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(seed, L, p), L)
    return bm.build_envs(Jh, Jv, beta, chi)


def assert_qplus_close(q_gpu, q_ref, precision):
    q_gpu = np.asarray(q_gpu)
    q_ref = np.asarray(q_ref)
    d = np.abs(q_gpu - q_ref)
    if precision == "fp64":
        lim = REL_FP64 * np.minimum(q_ref, 1.0 - q_ref) + 4e-16
        bad = d > lim
        assert not bad.any(), f"max rel err {(d / np.maximum(np.minimum(q_ref, 1 - q_ref), 1e-300)).max():.3e}"
    else:
        assert d.max() <= ABS_REDUCED, f"max abs err {d.max():.3e}"
    return float(d.max())


def assert_logq_within_site_tolerance(lq_gpu, lq_ref, qplus_ref, spins, qplus_gpu):
    """|log q_gpu - log q_ref| per proposal within the bound that the per-site tolerance implies:
    a conditional within ABS_REDUCED of the oracle's changes log q(s_i) by at most
    ABS_REDUCED / (q_ref(s_i) - ABS_REDUCED); at the rare sampled branches with
    q_ref(s_i) <= 2 ABS_REDUCED that bound is useless, and the site's own measured error
    |log q_gpu(s_i) - log q_ref(s_i)| (from the GPU's teacher-forced q(+), itself within the
    tolerance) stands in for it.  A 1e-6-per-site slack covers the FP32 logarithms."""
    sp = np.asarray(spins).reshape(len(spins), -1)
    q_s = np.where(sp == 1, np.asarray(qplus_ref).reshape(sp.shape), 1.0 - np.asarray(qplus_ref).reshape(sp.shape))
    g_s = np.where(sp == 1, np.asarray(qplus_gpu).reshape(sp.shape), 1.0 - np.asarray(qplus_gpu).reshape(sp.shape))
    big = q_s > 2 * ABS_REDUCED
    per_site = np.where(big, ABS_REDUCED / np.where(big, q_s - ABS_REDUCED, 1.0),
                        np.abs(np.log(np.maximum(g_s, 1e-300)) - np.log(np.maximum(q_s, 1e-300))))
    bound = per_site.sum(axis=1) + 1e-6 * sp.shape[1]
    d = np.abs(np.asarray(lq_gpu) - np.asarray(lq_ref))
    assert (d <= bound).all(), f"log q error {d.max():.3e} above the per-site bound {bound.min():.3e}"
    return float(d.max())


def check_spins_match(env, seed, chain, steps, spins_gpu, qplus_ref, tol):
    """The GPU's spins equal the oracle's own draws with the same Philox uniforms, except
    after a site where |u - q(+)| < tol (then the oracle's decision is not robust)."""
    L = env.Lx
    pr = sampler.propose(env, seed, chain, steps)
    u = sampler.spin_uniforms(seed, chain, steps, L, L)
    n_diff = 0
    for k in range(len(steps)):
        a = pr["spins"][k].reshape(-1)
        b = np.asarray(spins_gpu[k]).reshape(-1)
        diff = np.nonzero(a != b)[0]
        if len(diff):
            i = diff[0]
            n_diff += 1
            assert abs(u[k, i] - qplus_ref[k].reshape(-1)[i]) < tol, \
                f"proposal {k}: first differing site {i} has |u-q| = {abs(u[k, i] - qplus_ref[k].reshape(-1)[i]):.3e}"
    return n_diff
