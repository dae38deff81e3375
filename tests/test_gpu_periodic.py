"""GPU parity of external fields and of periodic boundaries by a pinned pair of lines (Sec. IV),
through the C ABI, against the oracle on the same seeded inputs."""
import numpy as np
import pytest

from oracle import boundary_mps as bm
from oracle import brute, lattice, periodic, sampler
from tests.gpu_helpers import assert_qplus_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tn():
    import paper_2409_06538_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    return pkg


@pytest.mark.parametrize("precision,L,chi", [("fp64", 4, 4), ("fp64", 12, 8), ("tf32", 12, 16), ("fp32", 10, 8)])
def test_fields_parity_open_lattice(tn, precision, L, chi):
    """Integer fields k (units of beta) on an open lattice: log Z (against enumeration when
    untruncated at L = 4) and the teacher-forced conditionals of the GPU's own proposals equal
    the oracle's with H = beta k."""
    p = 0.15
    beta = lattice.nishimori_beta(p)
    seeds = [5, 6]
    rng = np.random.default_rng(L + chi)
    k = rng.integers(-2, 3, size=(len(seeds), L, L)).astype(np.int8)
    J = tn.couplings_pmj(L, seeds, p)
    ctx = tn.TNMC(L, J, [beta] * 2, seeds, chi, precision=precision, n_chains=2)
    ctx.set_fields(k)
    lz = ctx.build_env()
    ctx.propose(3, 0)
    sp = ctx.spins().cpu().numpy().reshape(2, 6, L, L)
    _, qp = ctx.eval_conditionals(torch.from_numpy(sp).cuda())
    qp = qp.cpu().numpy().reshape(2, 6, L, L)
    for r, s in enumerate(seeds):
        Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(s, L, p), L)
        H = beta * k[r].astype(np.float64)
        env = bm.build_envs(Jh, Jv, beta, chi, H)
        tol = 1e-11 if precision == "fp64" else 1e-4
        assert abs(lz[r] - env.log_z) < tol * abs(env.log_z)
        if L == 4:
            _, _, logZ, _ = brute.exact(Jh, Jv, beta, H)
            assert abs(lz[r] - logZ) < tol * abs(logZ)
        ev = sampler.evaluate(env, sp[r])
        assert_qplus_close(qp[r], ev["qplus"], precision)
    ctx.set_fields(None)
    lz0 = ctx.build_env()
    for r, s in enumerate(seeds):
        Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(s, L, p), L)
        assert abs(lz0[r] - bm.build_envs(Jh, Jv, beta, chi).log_z) < 1e-4 * abs(lz0[r])
    ctx.close()


def test_torus_couplings_bit_exact(tn):
    seeds = [0, 9, 123456789]
    for L in (3, 8, 33):
        J = tn.torus_couplings_pmj(L, seeds, 0.2).cpu().numpy()
        for r, s in enumerate(seeds):
            assert np.array_equal(J[r], periodic.torus_couplings_pmj(s, L, 0.2))


@pytest.mark.parametrize("L,chi", [(5, 4), (7, 4), (9, 8)])
def test_periodic_chain_parity_fp64(tn, L, chi):
    """Step by step, the GPU's torus states equal the oracle's periodic chain on the same seeds
    (lines, region proposals and accept decisions from the same Philox counters), for an
    untruncated region (L = 5, chi = 4) and truncated ones; the thermal means of E, m^2 and the
    overlap equal the oracle's means over the same states."""
    p = 0.12
    beta = lattice.nishimori_beta(p)
    seeds = [3, 8]
    n = 8
    J = tn.torus_couplings_pmj(L, seeds, p)
    ctx = tn.TNMCPeriodic(L, J, [beta] * 2, seeds, chi, precision="fp64", n_chains=2)
    gpu = []
    for t in range(n):
        ctx.step(1, t)
        gpu.append(ctx.spins().cpu().numpy())
    gpu = np.stack(gpu, axis=2)                       # [real, chain, step, L, L]
    obs = ctx.observables()
    ctx.close()
    accepted_all = True
    for r, s in enumerate(seeds):
        Jh, Jv = periodic.split_torus(periodic.torus_couplings_pmj(s, L, p), L)
        sts = []
        for ch in range(2):
            st, acc = periodic.chain(np.ones((L, L), dtype=np.int64), Jh, Jv, beta, chi, s, ch, range(n))
            assert np.array_equal(gpu[r, ch], st), f"seed {s} chain {ch}"
            accepted_all &= bool(acc.all())
            sts.append(st)
        E = np.array([periodic.torus_energy(x, Jh, Jv) for x in sts]).astype(np.float64)
        m = np.array([x.reshape(n, -1).mean(axis=1) for x in sts])
        q = (sts[0] * sts[1]).reshape(n, -1).mean(axis=1)
        assert abs(obs[r]["E"] - E.mean()) < 1e-9 * max(1.0, abs(E.mean()))
        assert abs(obs[r]["m2"] - (m ** 2).mean()) < 1e-12
        assert abs(obs[r]["q2"] - (q ** 2).mean()) < 1e-12
        assert obs[r]["n_tests"] == 2 * n and obs[r]["status"] == 0
    if L == 5:
        assert accepted_all                          # untruncated region: exact conditional


def test_periodic_tf32_runs_and_stays_consistent(tn):
    """The mixed path on the torus: acceptance in (0, 1], every state +-1, no failure, and the
    overlap and magnetisation moments within their bounds."""
    L, chi, p = 16, 16, 0.109
    beta = lattice.nishimori_beta(p)
    seeds = [1, 2, 3, 4]
    J = tn.torus_couplings_pmj(L, seeds, p)
    ctx = tn.TNMCPeriodic(L, J, [beta] * 4, seeds, chi, precision="tf32", n_chains=2, n_therm=5)
    ctx.step(30, 0)
    sp = ctx.spins().cpu().numpy()
    obs = ctx.observables()
    assert set(np.unique(sp)) <= {-1, 1}
    for o in obs:
        assert o["status"] == 0 and 0 < o["n_acc"] <= o["n_tests"] == 60
        assert 0.0 <= o["m2"] <= 1.0 and 0.0 <= o["q2"] <= 1.0 and o["n_meas"] == 2 * 25
    ctx.close()
