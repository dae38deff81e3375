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
