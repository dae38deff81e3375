"""GPU parity: the CUDA path through the C ABI against the oracle, element by element on the
same seeded inputs (spin draws, conditionals, log q, energies, accept decisions,
observables) for the FP64, FP32 and mixed TF32 (tensor-core) paths, and the measured
error of BF16-stored environments."""
import numpy as np
import pytest

from oracle import brute, lattice, metropolis, sampler
from tests.gpu_helpers import (ABS_REDUCED, REL_FP64, assert_logq_within_site_tolerance, assert_qplus_close,
                               check_spins_match, oracle_envs)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tn():
    import paper_2409_06538_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    return pkg


def _ctx(tn, L, p, chi, seeds, precision, n_chains=2, n_therm=0, beta=None):
    beta = lattice.nishimori_beta(p) if beta is None else beta
    J = tn.couplings_pmj(L, seeds, p)
    return tn.TNMC(L, J, [beta] * len(seeds), seeds, chi, precision=precision, n_chains=n_chains, n_therm=n_therm)


def test_couplings_bit_exact(tn):
    seeds = [0, 1, 7, 123456789012345]
    for L in (2, 5, 32):
        J = tn.couplings_pmj(L, seeds, 0.109).cpu().numpy()
        for k, s in enumerate(seeds):
            assert np.array_equal(J[k], lattice.couplings_pmj(s, L, 0.109))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32"])
def test_exact_when_untruncated(tn, precision):
    """chi >= 2^{L/2}: log Z equals enumeration (L=4), every proposal has
    log q = -beta E - log Z, and every proposal is accepted (config: L=8, chi=16, p=0.10)."""
    p = 0.10
    beta = lattice.nishimori_beta(p)
    seeds = list(range(6))
    ctx = _ctx(tn, 4, p, 16, seeds, precision)
    lz = ctx.build_env()
    for k, s in enumerate(seeds):
        Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(s, 4, p), 4)
        _, _, logZ, _ = brute.exact(Jh, Jv, beta)
        assert abs(lz[k] - logZ) < (1e-11 if precision == "fp64" else 1e-4) * abs(logZ)
    ctx.close()
    ctx = _ctx(tn, 8, p, 16, seeds, precision)
    lz = ctx.build_env()
    out = ctx.propose(50, 0)
    acc = ctx.accept(flags=True, count=True)
    lq = out["logq"].cpu().numpy()
    E = out["energy"].cpu().numpy()
    for k, s in enumerate(seeds):
        env = oracle_envs(s, 8, p, 16)
        assert abs(lz[k] - env.log_z) < (1e-11 if precision == "fp64" else 1e-4) * abs(env.log_z)
        resid = lq[k] + beta * E[k] + env.log_z
        assert np.abs(resid).max() < (1e-9 if precision == "fp64" else 2e-3)
    if precision == "fp64":
        assert acc["flags"].cpu().numpy().all()
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
def test_exact_when_untruncated_chi64(tn, precision):
    """chi = 64 = 2^{L/2} at L = 12: nothing is truncated, so the GPU log Z equals the oracle's
    and every proposal has log q = -beta E - log Z (the chi = 64 build keeps M in global
    scratch and reads R and the tiles from global memory; the sampler holds two bond indices
    per lane)."""
    p, L, chi = 0.10, 12, 64
    beta = lattice.nishimori_beta(p)
    seeds = [1, 5]
    ctx = _ctx(tn, L, p, chi, seeds, precision)
    lz = ctx.build_env()
    out = ctx.propose(20, 0)
    ctx.accept()
    lq = out["logq"].cpu().numpy()
    E = out["energy"].cpu().numpy()
    for k, s in enumerate(seeds):
        env = oracle_envs(s, L, p, chi)
        assert abs(lz[k] - env.log_z) < 1e-4 * abs(env.log_z)
        resid = lq[k] + beta * E[k] + env.log_z
        assert np.abs(resid).max() < 5e-3
    assert np.all(ctx.realization_status() == 0)
    ctx.close()


@pytest.mark.parametrize("precision,L,chi,p", [
    ("fp64", 16, 8, 0.109), ("fp64", 24, 16, 0.109), ("fp64", 13, 5, 0.2),
    ("fp32", 16, 8, 0.109), ("fp32", 24, 16, 0.109),
    ("tf32", 24, 16, 0.109), ("tf32", 20, 32, 0.109), ("tf32", 40, 32, 0.109),
    ("fp32", 16, 64, 0.109), ("tf32", 20, 64, 0.109),
])
def test_conditionals_and_spins(tn, precision, L, chi, p):
    """Per-site q(+) teacher-forced on the GPU's spins; log q; the spins themselves equal the
    oracle's draws wherever |u - q(+)| exceeds the tolerance; integer energies exact."""
    seeds = [3, 11, 2024]
    n = 6
    ctx = _ctx(tn, L, p, chi, seeds, precision)
    ctx.build_env(return_logz=False)
    out = ctx.propose(n, 5)
    spins = ctx.spins().cpu().numpy()                 # [R, chains, n, L, L]
    lq = out["logq"].cpu().numpy()
    E = out["energy"].cpu().numpy()
    M = out["magnet"].cpu().numpy()
    flat = torch.from_numpy(spins.reshape(len(seeds), 2 * n, L, L)).cuda()
    lq_tf, qp_tf = ctx.eval_conditionals(flat)
    lq_tf = lq_tf.cpu().numpy().reshape(len(seeds), 2, n)
    qp_tf = qp_tf.cpu().numpy().reshape(len(seeds), 2, n, L, L)
    tol = REL_FP64 if precision == "fp64" else ABS_REDUCED
    for k, s in enumerate(seeds):
        env = oracle_envs(s, L, p, chi)
        for ch in range(2):
            ev = sampler.evaluate(env, spins[k, ch])
            assert_qplus_close(qp_tf[k, ch], ev["qplus"], precision)
            # the chain uses exactly the q it sampled from: a proposal's log q equals the same
            # kernel's teacher-forced log q of its own spins on every path
            assert np.abs(lq[k, ch] - lq_tf[k, ch]).max() <= 1e-9 * np.abs(lq_tf[k, ch]).max() + 1e-12
            if precision == "fp64":
                assert np.abs(lq[k, ch] - ev["logq"]).max() <= REL_FP64 * np.abs(ev["logq"]).max() + 1e-10
            else:
                assert_logq_within_site_tolerance(lq[k, ch], ev["logq"], ev["qplus"], spins[k, ch], qp_tf[k, ch])
            Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(s, L, p), L)
            assert np.array_equal(E[k, ch], lattice.energy(spins[k, ch], Jh, Jv))
            assert np.array_equal(M[k, ch], spins[k, ch].reshape(n, -1).sum(axis=1))
            check_spins_match(env, s, ch, np.arange(5, 5 + n), spins[k, ch], ev["qplus"], max(tol, 1e-12))
    ctx.close()


def test_bf16_environments_characterised(tn):
    """BF16-rounded cached environments do NOT meet the 1e-3 conditional tolerance: the
    contraction of a sign-indefinite MPS amplifies element rounding (about 100 x 2^-8 at
    L = 16, growing with L).  The path stays self-consistent -- the log q a proposal carries
    equals the teacher-forced log q of the same environments -- so Metropolis still corrects
    it exactly; the error is measured and bounded here, not hidden."""
    L, p, chi = 16, 0.109, 8
    seeds = [3, 11]
    ctx = _ctx(tn, L, p, chi, seeds, "bf16")
    ctx.build_env(return_logz=False)
    out = ctx.propose(4, 0)
    spins = ctx.spins()
    lq_tf, qp_tf = ctx.eval_conditionals(spins.reshape(len(seeds), 8, L, L))
    lq = out["logq"].cpu().numpy().reshape(len(seeds), 8)
    assert np.abs(lq - lq_tf.cpu().numpy()).max() < 1e-9 * np.abs(lq).max()
    err = 0.0
    sp = spins.cpu().numpy().reshape(len(seeds), 8, L, L)
    for k, s in enumerate(seeds):
        env = oracle_envs(s, L, p, chi)
        ev = sampler.evaluate(env, sp[k])
        err = max(err, float(np.abs(qp_tf.cpu().numpy()[k] - ev["qplus"]).max()))
    print(f"bf16 environments: max |dq(+)| = {err:.3e} at L={L}, chi={chi}")
    assert err < 0.1
    ctx.close()


def test_environment_vectors_fp64(tn):
    """The cached environments as full 2^L vectors equal the oracle's (gauge invariant)."""
    from oracle import boundary_mps as bm
    L, p, chi = 7, 0.2, 3
    seeds = [5, 6]
    ctx = _ctx(tn, L, p, chi, seeds, "fp64")
    ctx.build_env()
    for k, s in enumerate(seeds):
        env = oracle_envs(s, L, p, chi)
        for r in range(L):
            tiles, dims, lam = ctx.copy_env(k, r)
            mps = [np.transpose(tiles[c][:, :dims[c], :dims[c + 1]], (1, 0, 2)) for c in range(L)]
            assert list(dims) == env.bond_dims(r)
            v_gpu = bm.contract_row(mps)
            v_ref = bm.contract_row(env.B[r])
            assert np.abs(v_gpu - v_ref).max() < 1e-12 * max(1.0, np.abs(v_ref).max())
            assert abs(lam - env.lam[r]) < 1e-11 * max(1.0, abs(env.lam[r]))
    ctx.close()


def test_metropolis_and_observables_parity(tn):
    """Accept decisions equal the oracle's on the GPU's own (E, log q) stream, across two
    calls (carried state), and the per-realization observables equal the oracle's means of
    the current states (E, |m|, m^2, m^4, overlap q between the two chains)."""
    L, p, chi = 8, 0.109, 2
    beta = lattice.nishimori_beta(p)
    seeds = [0, 1, 2, 3]
    n, n_therm = 40, 10
    ctx = _ctx(tn, L, p, chi, seeds, "fp64", n_therm=n_therm)
    ctx.build_env(return_logz=False)
    E_all, lq_all, sp_all, fl_all = [], [], [], []
    for call in range(2):
        out = ctx.propose(n, call * n)
        sp_all.append(ctx.spins().cpu().numpy())
        fl_all.append(ctx.accept(flags=True)["flags"].cpu().numpy())
        E_all.append(out["energy"].cpu().numpy())
        lq_all.append(out["logq"].cpu().numpy())
    obs = ctx.observables()
    E = np.concatenate(E_all, axis=2)
    lq = np.concatenate(lq_all, axis=2)
    sp = np.concatenate(sp_all, axis=2)
    fl = np.concatenate(fl_all, axis=2)
    per = []
    for k, s in enumerate(seeds):
        cur_sp, cur_E = [], []
        for ch in range(2):
            acc, cur, _ = metropolis.metropolis_chain(E[k, ch], lq[k, ch], beta, s, ch, np.arange(2 * n))
            assert np.array_equal(acc, fl[k, ch].astype(bool))
            cur_sp.append(sp[k, ch][cur])
            cur_E.append(E[k, ch][cur])
        o = metropolis.chain_observables(np.stack(cur_sp), np.stack(cur_E))
        ref = metropolis.thermal_means(o, n_therm)
        for key in ("E", "E2", "m_abs", "m2", "m4", "q", "q_abs", "q2", "q4", "m_edge", "m_edge_abs", "m_edge2"):
            assert abs(obs[k][key] - ref[key]) <= 1e-12 * max(1.0, abs(ref[key])), key
        assert obs[k]["n_prop"] == 2 * 2 * n
        assert obs[k]["n_tests"] == 2 * 2 * n - 2          # each chain's initial state is no test
        assert obs[k]["n_acc"] == int(fl[k].sum()) - 2
        assert obs[k]["status"] == 0
        per.append(ref)
    assert 0.0 < np.mean([o["n_acc"] for o in obs]) < 2 * 2 * n
    assert np.all(ctx.realization_status() == 0)


def test_observables_match_independent_oracle_run(tn):
    """Disorder-averaged E, m^2 and Binder ratio within two combined standard errors of a
    fully independent oracle run on the same seeds (p = 0.109, Nishimori beta, chi = 4)."""
    import paper_2409_06538_gb300 as pkg
    L, p, chi = 8, 0.109, 4
    beta = lattice.nishimori_beta(p)
    seeds = list(range(24))
    n, n_therm = 60, 5
    ctx = _ctx(tn, L, p, chi, seeds, "fp64", n_therm=n_therm)
    ctx.build_env(return_logz=False)
    ctx.propose(n, 0)
    ctx.accept()
    gobs = ctx.observables()
    g = pkg.disorder_average(gobs, L, beta)
    per = []
    for s in seeds:
        env = oracle_envs(s, L, p, chi)
        cs, ce = [], []
        for ch in range(2):
            pr = sampler.propose(env, s, ch, np.arange(n))
            acc, cur, _ = metropolis.metropolis_chain(pr["energy"], pr["logq"], beta, s, ch, np.arange(n))
            cs.append(pr["spins"][cur]); ce.append(pr["energy"][cur])
        per.append(metropolis.thermal_means(metropolis.chain_observables(np.stack(cs), np.stack(ce)), n_therm))
    o = metropolis.disorder_average(per)
    for key in ("E", "m2", "q2", "m_edge2"):
        se = np.hypot(g[key][1], o[key][1])
        assert abs(g[key][0] - o[key][0]) <= 2 * se + 1e-12, key

    def jackknife_se(m4, m2):
        # standard error of the ratio of means [m4]/[m2]^2 by leave-one-out over realizations
        m4, m2 = np.asarray(m4), np.asarray(m2)
        R = len(m4)
        loo = np.array([np.delete(m4, i).mean() / np.delete(m2, i).mean() ** 2 for i in range(R)])
        return np.sqrt((R - 1) / R * ((loo - loo.mean()) ** 2).sum())

    se_g = jackknife_se([x["m4"] for x in gobs], [x["m2"] for x in gobs])
    se_o = jackknife_se([x["m4"] for x in per], [x["m2"] for x in per])
    assert abs(g["U_m"] - o["U_m"]) <= 2 * np.hypot(se_g, se_o), (g["U_m"], o["U_m"], se_g, se_o)


def test_set_realizations_reuses_a_context(tn):
    """New seeds on an existing context (couplings generated on the device, asynchronously)
    give the same environments as a fresh context and as the oracle, twice in a row."""
    L, p, chi = 12, 0.109, 8
    beta = lattice.nishimori_beta(p)
    ctx = _ctx(tn, L, p, chi, [1, 2, 3], "fp64")
    ctx.build_env()
    for seeds in ([10, 11, 12], [7, 8, 9]):
        ctx.set_realizations(seeds, [beta] * 3, p)
        lz = ctx.build_env()
        fresh = _ctx(tn, L, p, chi, seeds, "fp64")
        lz_fresh = fresh.build_env()
        fresh.close()
        assert np.abs(lz - lz_fresh).max() == 0.0
        for k, s in enumerate(seeds):
            assert abs(lz[k] - oracle_envs(s, L, p, chi).log_z) < 1e-11 * abs(lz[k])
        out = ctx.propose(3, 0)
        ctx.accept()
        assert np.isfinite(out["logq"].cpu().numpy()).all()
    ctx.close()


def test_argument_errors(tn):
    from paper_2409_06538_gb300 import _capi
    L = 4
    J = np.ones((1, 2 * L * (L - 1)), dtype=np.int8)
    with pytest.raises(_capi.TnmcError) as e:
        tn.TNMC(L, J, [1.0], [0], 64)
    assert e.value.code == 7
    bad = J.copy(); bad[0, 3] = 0
    with pytest.raises(_capi.TnmcError) as e:
        tn.TNMC(L, bad, [1.0], [0], 4)
    assert e.value.code == 1
    with pytest.raises(_capi.TnmcError) as e:
        tn.TNMC(L, J, [-1.0], [0], 4)
    assert e.value.code == 1
    ctx = tn.TNMC(L, J, [1.0], [0], 4)
    with pytest.raises(_capi.TnmcError) as e:
        ctx.propose(3)
    assert e.value.code == 6
    with pytest.raises(_capi.TnmcError) as e:
        ctx.accept()
    assert e.value.code == 6
    ctx.close()


@pytest.mark.parametrize("L,seed", [(128, 77), (256, 1_000_003), (256, 18_000_068)])
def test_large_lattice_parity_tf32(tn, L, seed):
    """The configuration the throughput is quoted on (chi = 32, p = 0.109, mixed TF32) at L = 128
    and 256: teacher-forced q(+) at every site of the GPU's own proposals within 1e-3 of the FP64
    oracle, log q within the bound that per-site tolerance implies, proposal log q equal to the
    teacher-forced one, and the spins equal to the oracle's own draws wherever |u - q(+)| exceeds
    the tolerance.  One realization, two chains x two proposals (the oracle needs about a minute
    per L = 256 realization on the host)."""
    p, chi, n = 0.109, 32, 2
    ctx = _ctx(tn, L, p, chi, [seed], "tf32")
    ctx.build_env(return_logz=False)
    out = ctx.propose(n, 3)
    spins = ctx.spins().cpu().numpy()
    lq = out["logq"].cpu().numpy()
    E = out["energy"].cpu().numpy()
    lq_tf, qp_tf = ctx.eval_conditionals(torch.from_numpy(spins.reshape(1, 2 * n, L, L)).cuda())
    lq_tf = lq_tf.cpu().numpy().reshape(2, n)
    qp_tf = qp_tf.cpu().numpy().reshape(2, n, L, L)
    assert np.all(ctx.realization_status() == 0)
    env = oracle_envs(seed, L, p, chi)
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(seed, L, p), L)
    for ch in range(2):
        ev = sampler.evaluate(env, spins[0, ch])
        err = assert_qplus_close(qp_tf[ch], ev["qplus"], "tf32")
        print(f"L={L}: chain {ch} max |dq(+)| = {err:.3e}")
        assert np.abs(lq[0, ch] - lq_tf[ch]).max() <= 1e-9 * np.abs(lq_tf[ch]).max()
        assert_logq_within_site_tolerance(lq[0, ch], ev["logq"], ev["qplus"], spins[0, ch], qp_tf[ch])
        assert np.array_equal(E[0, ch], lattice.energy(spins[0, ch], Jh, Jv))
        check_spins_match(env, seed, ch, np.arange(3, 3 + n), spins[0, ch], ev["qplus"], ABS_REDUCED)
    ctx.close()
