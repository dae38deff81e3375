"""Benchmark of the TNMC hot path on GB300: one step = one full pass over a batch of
disorder realizations -- seeded +-J couplings, boundary-MPS environments (all rows cached),
proposals with log q, Metropolis and observables.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Default workload (one GPU): L = 256, chi = 32, p = 0.109 on the Nishimori line,
64 realizations x 2 chains x 250 proposals (500 proposals per realization) per step, mixed
precision (FP32 environment build and cache, 3xTF32 tensor-core sampling, FP64 log-norms,
log q and Metropolis).  Up to --inflight steps run concurrently, one context and CUDA
stream each (continuous batching: a batch's environment build leaves most SMs free); by default
as many batches as the SMs hold environment-build CTAs (seven here, 448 of 456 slots), and as
many timed steps.
Under torchrun every rank runs its own batches (weak scaling, no data-path collective).
Prints one JSON line on rank 0.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes per unit of work from one ncu capture of the current kernels (dram__bytes_read.sum +
# dram__bytes_write.sum at L = 128, chi = 32, 16 realizations x 500 proposals, mixed TF32;
# profiles/dram_traffic_L128_chi32_R16_tf32.md), scaled by the units of a launch in roofline()
ENV_DRAM_BYTES_PER_SITE_STEP = (304292096 + 6117933568) / (16 * 127 * 128)              # 24.7 KB
SAMPLE_TC_DRAM_BYTES_PER_PROPOSAL_SITE = (29919938048 + 34385152512) / (16 * 500 * 128 * 128)   # 491 B

METRIC = "spins proposed/s at L=256 χ=32, BF16/TF32 vs FP64 GPU path; p50/p99 latency"
UNIT = "spins/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed batches (default: as many as run at once, at least 4)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32", choices=["bf16", "tf32", "fp32", "fp64"])
    ap.add_argument("--compression", default="canonical", choices=["canonical", "zipup"],
                    help="boundary-MPS compression of the environment build (tnmc_compression)")
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--chi", type=int, default=32)
    ap.add_argument("--R", type=int, default=64, help="realizations per GPU")
    ap.add_argument("--n", type=int, default=250, help="proposals per chain per step")
    ap.add_argument("--chains", type=int, default=2)
    ap.add_argument("--p", type=float, default=0.109)
    ap.add_argument("--inflight", type=int, default=0,
                    help="batches in flight (contexts on streams); 0 = as many as the SMs hold at once")
    ap.add_argument("--obs-out", default=None,
                    help="write the per-realization thermal means of the last batch of every context (JSON)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle sample")
    ap.add_argument("--periodic", action="store_true",
                    help="periodic boundaries (pinned pair of lines per step) on L x L tori: one JSON line")
    ap.add_argument("--serve", action="store_true",
                    help="serving measurement: a Poisson request stream through the request server")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--serve-Ls", default="16,32,64,128,256,512")
    ap.add_argument("--serve-chi-max", type=int, default=64)
    ap.add_argument("--serve-inflight", type=int, default=32)
    ap.add_argument("--serve-linger-ms", type=float, default=20.0)
    return ap.parse_args()


# ----------------------------------------------------------------------------- oracle legs
def _oracle_sample_worker(args):
    """Time the oracle on a bounded sample of one realization: `rows` environment rows
    (after the bond dimension has saturated) and the sampling sweep of those rows."""
    L, chi, p, seed, rows = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    from oracle import boundary_mps as bm, lattice, sampler
    beta = lattice.nishimori_beta(p)
    Jh, Jv = lattice.split_couplings(lattice.couplings_pmj(seed, L, p), L)
    Jh = Jh.astype(float); Jv = Jv.astype(float)
    mps = [np.ones((1, 2, 1)) for _ in range(L)]
    warm = int(math.ceil(math.log2(max(chi, 2)))) + 1
    t_build = 0.0
    built = []
    for i, r in enumerate(range(L - 2, L - 2 - warm - rows, -1)):
        t0 = time.perf_counter()
        mps, _ = bm.compress(bm.apply_mpo(bm.row_mpo(beta, Jv[r], Jh[r + 1]), mps), chi)
        dt = time.perf_counter() - t0
        if i >= warm:
            t_build += dt
            built.append((r, mps))
    t_samp = 0.0
    K = 2
    rng = np.random.default_rng(seed)
    for r, m in built:
        h = beta * Jv[r - 1][None, :] * np.where(rng.random((K, L)) < 0.5, 1.0, -1.0)
        u = rng.random((K, L))
        t0 = time.perf_counter()
        sampler.sweep_row(m, Jh[r], h, beta, uniforms=u)
        t_samp += time.perf_counter() - t0
    return t_build / len(built), t_samp / (len(built) * K)


def oracle_rate(L, chi, p, n_props_per_real, cores, budget_s):
    """Spins proposed/s of the oracle on `cores` host processes, extrapolated from a bounded
    sample: per-row environment cost and per-row-per-proposal sampling cost."""
    import multiprocessing as mp
    # size the sample: ~budget_s seconds per worker
    rows = max(2, min(24, int(budget_s / max(1e-3, 0.6e-5 * L * chi ** 2))))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_sample_worker, [(L, chi, p, 1000 + i, rows) for i in range(cores)])
    wall = time.perf_counter() - t0
    t_row = statistics.mean(r[0] for r in res)
    t_srow = statistics.mean(r[1] for r in res)
    t_real = (L - 1) * t_row + n_props_per_real * L * t_srow
    rate = cores * n_props_per_real * L * L / t_real
    sample = (f"{cores} processes x 1 realization each: {rows} environment rows (after bond saturation) and "
              f"{rows} rows x 2 proposals of sampling, L={L} chi={chi}; extrapolated to {L - 1} rows + "
              f"{n_props_per_real} proposals per realization (t_row={t_row:.3f}s, t_row_sample={t_srow * 1e3:.2f}ms)")
    return rate, sample, wall


def run_reference(a, rank, world):
    if a.steps is None:
        a.steps = 4
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    vals = []
    sample = ""
    for i in range(a.warmup + a.steps):
        budget = max(3.0, a.cpu_seconds / 3)
        rate, sample, _ = oracle_rate(a.L, a.chi, a.p, a.chains * a.n, cores, budget)
        if i >= a.warmup:
            vals.append(rate)
    v = statistics.mean(vals)
    spins_per_step = a.R * a.chains * a.n * a.L * a.L
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=a.gpus, steps=a.steps, warmup=a.warmup,
                ms_per_step=1e3 * spins_per_step / v, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic: Philox +-J disorder on the Nishimori line", impl="reference",
                config=_config(a),
                cpu_baseline=dict(value=v, unit=UNIT, cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def _config(a):
    return dict(workload=f"TNMC L={a.L} chi={a.chi} p={a.p} Nishimori beta, {a.R} realizations x "
                         f"{a.chains} chains x {a.n} proposals per GPU per step",
                L=a.L, chi=a.chi, p=a.p, realizations_per_gpu=a.R, chains=a.chains,
                proposals_per_chain=a.n, precision=("fp64" if a.impl == "reference" else a.precision),
                compression=("canonical" if a.impl == "reference" else a.compression),
                l2="inputs larger than L2: the environment cache read by the sampler is rebuilt every step")


# ----------------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        fd, self.path = tempfile.mkstemp(prefix="tnmc_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            try:
                os.remove(self.path)
            except OSError:
                pass
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        load = [x for x in sm if x > 0.5 * mx] or sm
        try:
            os.remove(self.path)
        except OSError:
            pass
        return dict(sm_mhz=statistics.median(load), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


# ----------------------------------------------------------------------------- our arm
def run_waves(steps, S, streams, make_event, inputs, work, marks=None):
    """Queue the batches `steps` (global step indices) on S contexts and streams, in waves of
    S.  A wave first queues every batch's new inputs (small kernels) on its stream, then every
    stream of the wave waits for all of them before its environment build: the builds of a wave
    are dispatched together onto SMs that no small kernel of another stream occupies.  (With
    the build filling 448 of 456 CTA slots, a couplings kernel resident on an SM when the builds
    are dispatched can keep a build CTA waiting for a whole build to finish elsewhere.)
    inputs(k, i) queues batch k's inputs on context i; work(i, marks) queues the rest;
    marks[j] (optional) are four timing events of the j-th batch, the first recorded here."""
    steps = list(steps)
    for w0 in range(0, len(steps), S):
        wave = steps[w0:w0 + S]
        ready = []
        for j, k in enumerate(wave):
            i = (w0 + j) % S
            if marks is not None:
                marks[w0 + j][0].record(streams[i])
            inputs(k, i)
            e = make_event()
            e.record(streams[i])
            ready.append(e)
        for j, k in enumerate(wave):
            i = (w0 + j) % S
            for e in ready:
                streams[i].wait_event(e)
            work(i, marks[w0 + j] if marks is not None else None)


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if a.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    if a.impl == "reference":
        run_reference(a, rank, world)
        return _finish(world)
    if a.periodic:
        if rank == 0:
            return run_periodic(a)
        return _finish(world)
    if a.serve:
        if rank == 0:
            rc = run_serve(a)
            if world == 1:
                return rc
        return _finish(world)

    import threading
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06538_gb300 as tn
    from paper_2409_06538_gb300 import _capi
    import ctypes

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    beta = tn.nishimori_beta(a.p)
    R, L = a.R, a.L
    per_sm, n_sms = tn.env_build_occupancy(L, a.chi, a.precision)
    slots = per_sm * n_sms                         # environment-build CTAs the GPU holds at once
    if a.inflight <= 0:
        a.inflight = max(1, slots // R)
    if a.steps is None:
        a.steps = max(4, a.inflight)
    S = max(1, min(a.inflight, a.steps))          # batches in flight (one context + stream each)

    def seeds_for(step):
        base = 1_000_003 * (step + 1) + rank * R
        return np.arange(base, base + R, dtype=np.uint64)

    streams = [torch.cuda.Stream(device=dev) for _ in range(S)]
    J0 = tn.couplings_pmj(L, seeds_for(0), a.p)
    ctxs = [tn.TNMC(L, J0, [beta] * R, seeds_for(0), a.chi, precision=a.precision, n_chains=a.chains,
                    n_therm=0, stream=streams[i], compression=a.compression) for i in range(S)]
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # per timed batch, the realizations' failure flags (copied on the device after the
    # Metropolis step, read once at the end)
    flags = torch.zeros((a.warmup + a.steps, R), dtype=torch.int32, device=dev)
    step_of = {}

    def inputs(step, i):
        """New realizations on context i: couplings generated on the device, queued on stream i."""
        ctxs[i].set_realizations(seeds_for(step), [beta] * R, a.p)
        step_of[i] = step

    def work(i, marks=None):
        """Environments, proposals, Metropolis on context i -- queued on stream i, no host sync."""
        ctx, st = ctxs[i], streams[i]
        ctx.build_env(return_logz=False)
        if marks: marks[1].record(st)
        ctx.propose(a.n, 0, outputs=False)
        if marks: marks[2].record(st)
        ctx.accept()
        ctx.realization_status_async(flags[step_of[i]])
        if marks: marks[3].record(st)

    sync_ev = lambda: torch.cuda.Event()  # noqa: E731
    run_waves(range(a.warmup), S, streams, sync_ev, inputs, work)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = sum(c.launch_count() for c in ctxs)
    main_st = torch.cuda.current_stream()
    t_start, t_end = ev(), ev()
    torch.cuda.synchronize()
    t_start.record(main_st)
    for st in streams:
        st.wait_event(t_start)
    marks = [[ev() for _ in range(4)] for _ in range(a.steps)]
    run_waves(range(a.warmup, a.warmup + a.steps), S, streams, sync_ev, inputs, work, marks)
    for st in streams:
        e = ev(); e.record(st); main_st.wait_event(e)
    t_end.record(main_st)
    torch.cuda.synchronize()
    gpu_launches = sum(c.launch_count() for c in ctxs) - launches0
    elapsed = t_start.elapsed_time(t_end) / 1e3
    if world > 1:
        t = torch.tensor([elapsed], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
    clk = clocks.stop()
    per_step = [m[0].elapsed_time(m[3]) for m in marks]
    build_ms = statistics.mean(m[0].elapsed_time(m[1]) for m in marks)
    samp_ms = statistics.mean(m[1].elapsed_time(m[2]) for m in marks)
    acc_ms = statistics.mean(m[2].elapsed_time(m[3]) for m in marks)
    # union of the device intervals in which an environment build / a sampling sweep ran
    def union(pairs):
        iv = sorted((t_start.elapsed_time(x), t_start.elapsed_time(y)) for x, y in pairs)
        tot, cur = 0.0, None
        for s0, s1 in iv:
            if cur is None or s0 > cur[1]:
                if cur: tot += cur[1] - cur[0]
                cur = [s0, s1]
            else:
                cur[1] = max(cur[1], s1)
        if cur: tot += cur[1] - cur[0]
        return tot
    build_union_ms = union([(m[0], m[1]) for m in marks])
    samp_union_ms = union([(m[1], m[2]) for m in marks])
    stats = [c.build_stats() for c in ctxs]
    mean_sweeps = sum(s_["total_sweeps"] for s_ in stats) / max(1, sum(s_["svds"] for s_ in stats))
    # realizations that met a doubly clamped site (TNMC_ERR_NUMERIC under the clamp reading):
    # reported with their seeds, left out of the averages and of the throughput
    fl = flags.cpu().numpy()
    failed_seeds = [int(seeds_for(k)[r]) for k in range(a.warmup + a.steps) for r in range(R) if fl[k, r] != 0]
    n_failed_timed = int((fl[a.warmup:] != 0).sum())
    obs = []        # the last batch of every context (observables of the realizations it holds)
    obs_seeds = []
    for i, c in enumerate(ctxs):
        obs += c.observables(allow_numeric=True)
        obs_seeds += [int(x) for x in seeds_for(step_of[i])]
    if a.obs_out and rank == 0:
        with open(a.obs_out, "w") as f:
            json.dump([dict(o, seed=sd) for o, sd in zip(obs, obs_seeds)], f)
    if world > 1:       # the one cross-rank exchange: per-realization means for [.] averages
        from paper_2409_06538_gb300 import shard
        dav, _ = shard.gather_disorder_average(obs, L, beta)
    else:
        dav = tn.disorder_average(obs, L, beta)
    spins_per_step = R * a.chains * a.n * L * L
    spins_ok = (R * a.steps - n_failed_timed) * a.chains * a.n * L * L
    if world > 1:
        t = torch.tensor([spins_ok], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t)
        spins_ok = float(t.item())
    value = spins_ok / elapsed

    # ---- end to end through the public API with host buffers: one host thread per context,
    # each step copies its couplings from pinned host memory and reads its observables back
    e2e = None
    if not a.no_e2e:
        Jhost = [torch.empty((R, 2 * L * (L - 1)), dtype=torch.int8).pin_memory() for _ in range(S)]
        for jh in Jhost:
            jh.copy_(J0.cpu())
        k_e2e = max(1, a.steps)
        torch.cuda.synchronize()

        def worker(i):
            torch.cuda.set_device(local)
            for k in range(i, k_e2e, S):
                ctxs[i].set_couplings(Jhost[i], [beta] * R, seeds_for(k))
                ctxs[i].build_env(return_logz=False)
                ctxs[i].propose(a.n, 0, outputs=False)
                ctxs[i].accept()
                # device-to-host read of the step's result, per-realization status included
                ctxs[i].observables(allow_numeric=True)
        t0 = time.perf_counter()
        ths = [threading.Thread(target=worker, args=(i,)) for i in range(S)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        e_el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e_el], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e_el = float(t.item())
        e2e = dict(value=world * spins_per_step * k_e2e / e_el, unit=UNIT,
                   h2d_bytes_per_step=int(R * 2 * L * (L - 1) + 16 * R),
                   d2h_bytes_per_step=int(R * (ctypes.sizeof(_capi.Obs) + 8)),
                   note="every realization's spins counted (the couplings of step 0 are reused)")

    roof = roofline(a, marks, build_union_ms, samp_union_ms, mean_sweeps)

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, sample, _ = oracle_rate(L, a.chi, a.p, a.chains * a.n, cores, a.cpu_seconds)
        cpu = dict(value=rate, unit=UNIT, cores=cores, kind="oracle", sample=sample)

    if rank == 0:
        cfg = _config(a)
        cfg["inflight_batches"] = S
        cfg["env_build_ctas_per_sm"] = per_sm
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=a.steps, warmup=a.warmup,
                    ms_per_step=1e3 * elapsed / a.steps, higher_is_better=True, scaling="weak",
                    vs_baseline=None, dtype=a.precision,
                    data="synthetic: Philox +-J disorder on the Nishimori line (seeded, no dataset)",
                    config=cfg, e2e=e2e, gpu_launches=int(gpu_launches),
                    roofline=roof, cpu_baseline=cpu, clocks=clk,
                    latency_ms=dict(p50=float(np.percentile(per_step, 50)), p99=float(np.percentile(per_step, 99)),
                                    unit="per batch of realizations, queue to Metropolis done"),
                    phases_ms=dict(env_build=build_ms, propose=samp_ms, accept=acc_ms,
                                   env_build_busy=build_union_ms, propose_busy=samp_union_ms),
                    jacobi_mean_sweeps=mean_sweeps,
                    accepted_proposals_per_s=value / (L * L) * dav["acceptance"],
                    acceptance=dav["acceptance"], clamps=dav["clamps"],
                    failed_realizations=dict(
                        timed=n_failed_timed, of=R * a.steps * world, seeds_rank0=failed_seeds,
                        rule="realizations whose proposals met a site with w+ + w- <= 0 after clamping; "
                             "their spins are not counted in value and their means not in the averages"),
                    observables=dict({k: dav[k] for k in ("E", "m2", "q2", "U_m", "Q_q", "m_edge2", "chi_q",
                                                          "chi_edge")},
                                     realizations=dav["n_used"], dropped=dav["n_dropped"],
                                     nishimori_E=-2 * L * (L - 1) * (1 - 2 * a.p)))
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    return _finish(world)


def roofline(a, marks, build_union_ms, samp_union_ms, mean_sweeps):
    """Roofline of the dominant kernel from live CUDA-event timings.  Algorithmic work of the
    environment build per site step (the boundary-MPS compression count of the method, not of this
    implementation's iterations): Householder QR of the 4chi x 2chi matrix ~27 chi^3, the MPO
    product R A ~32 chi^3, the truncating SVD of the 2chi x 2chi matrix ~100 chi^3 and the
    product carrying the truncated state on ~16 chi^3, i.e. 175 chi^3 flops, times (L-1) L site
    steps per realization (the zip-up compression has no QR: 148 chi^3).  It runs on the FP32 (FP64) CUDA cores, so the peak is the ALU peak
    derived from 152 SMs x 128 FP32 lanes x 2 flops x the SM clock (a 64th of it for FP64).
    Sampling sweep: bytes of the environment tiles read twice per row per 128-proposal tile plus
    the per-site workspace written and read back, against the measured HBM copy bandwidth."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    L, chi = a.L, a.chi
    CHI = 4 if chi <= 4 else 8 if chi <= 8 else 16 if chi <= 16 else 32 if chi <= 32 else 64
    site_flops = (148.0 if getattr(a, "compression", "canonical") == "zipup" else 175.0) * chi ** 3
    build_flops = a.R * (L - 1) * L * site_flops                  # per launch (one batch)
    K = len(marks)
    sm_clock = peaks.get("sm_max_mhz", 2070.0) * 1e6
    alu_peak = 152 * 128 * 2 * sm_clock / 1e12                    # FP32 lanes x FMA x clock
    if a.precision == "fp64":
        alu_peak = alu_peak / 64.0
    per_launch_ms = statistics.mean(m[0].elapsed_time(m[1]) for m in marks)
    build_tf = K * build_flops / (build_union_ms / 1e3) / 1e12
    te = {"fp64": 8, "fp32": 4, "tf32": 4, "bf16": 2}[a.precision]
    items = a.chains * a.n
    M = 128 if a.precision == "tf32" and CHI in (16, 32) else 8
    tiles = math.ceil(items / M) * a.R
    samp_bytes = tiles * 2 * L * L * (2 * CHI * CHI) * te + a.R * items * L * L * (2 * CHI) * 4 * 2
    samp_gbs = K * samp_bytes / (samp_union_ms / 1e3) / 1e9
    env_traffic = samp_traffic = None
    if a.precision == "tf32" and CHI == 32:
        # the counters were taken on the canonical build; the zip-up build writes no R factors
        if ENV_DRAM_BYTES_PER_SITE_STEP is not None and getattr(a, "compression", "canonical") == "canonical":
            env_traffic = ENV_DRAM_BYTES_PER_SITE_STEP * a.R * (L - 1) * L
        if SAMPLE_TC_DRAM_BYTES_PER_PROPOSAL_SITE is not None:
            samp_traffic = SAMPLE_TC_DRAM_BYTES_PER_PROPOSAL_SITE * a.R * items * L * L
    return dict(kernel="env_build_kernel", bound="alu", achieved=build_tf, peak=alu_peak, unit="TFLOP/s",
                frac=build_tf / alu_peak, traffic=env_traffic,
                traffic_source=("ncu capture at L=128, 16 realizations, scaled per site step"
                                if env_traffic is not None else None),
                peak_source=("derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"
                             + (" / 64 (FP64 rate of this part)" if a.precision == "fp64" else "")),
                algorithmic_flops_per_site_step=site_flops, algorithmic_flops_per_launch=build_flops,
                launches=K, per_launch_ms=per_launch_ms, busy_ms=build_union_ms,
                jacobi_mean_sweeps=mean_sweeps,
                sampler=dict(kernel="sample_tc_kernel" if M == 128 else "sample_kernel", bound="hbm",
                             achieved=samp_gbs, peak=hbm, unit="GB/s", frac=samp_gbs / hbm,
                             algorithmic_bytes_per_launch=samp_bytes, busy_ms=samp_union_ms,
                             traffic=samp_traffic,
                             peak_source="measured" if "hbm_gbs" in peaks else "fallback"))


def run_periodic(a):
    """Periodic boundaries by a pinned pair of lines (Sec. IV): R tori of side L, --chains chains,
    --n steps each (one region proposal of (L-1)^2 spins per step and chain, each with its own
    environment build).  Prints one JSON line: region spins proposed per second, acceptance and
    the torus observables."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06538_gb300 as tn
    torch.cuda.set_device(0)
    beta = tn.nishimori_beta(a.p)
    seeds = list(range(1000, 1000 + a.R))
    J = tn.torus_couplings_pmj(a.L, seeds, a.p)
    ctx = tn.TNMCPeriodic(a.L, J, [beta] * a.R, seeds, a.chi, precision=a.precision, n_chains=a.chains,
                          n_therm=a.warmup)
    ctx.step(a.warmup, 0)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    t0.record()
    ctx.step(a.n, a.warmup)
    t1.record()
    torch.cuda.synchronize()
    el = t0.elapsed_time(t1) / 1e3
    ck = clocks.stop()
    obs = ctx.observables()
    dav = tn.disorder_average(obs, a.L, beta)
    spins = a.R * a.chains * a.n * (a.L - 1) ** 2
    line = dict(metric="region spins proposed/s, periodic boundaries (pinned pair of lines per step)",
                value=spins / el, unit=UNIT, mode="periodic", n_gpus=1, steps=a.n, warmup=a.warmup,
                ms_per_step=1e3 * el / a.n, higher_is_better=True, dtype=a.precision, data="synthetic",
                config=dict(workload=f"periodic TNMC, {a.R} tori of L={a.L}, chi={a.chi}, p={a.p} Nishimori beta, "
                                     f"{a.chains} chains, {a.n} steps", L=a.L, chi=a.chi, p=a.p, R=a.R,
                            chains=a.chains, precision=a.precision),
                gpu_launches=ctx.launch_count() - l0, clocks=ck, acceptance=dav["acceptance"],
                failed_realizations=dav["n_dropped"],
                observables={k: dav[k] for k in ("E", "m2", "q2", "U_m", "Q_q")},
                nishimori_E=-2 * a.L * a.L * (1 - 2 * a.p))
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_serve(a):
    """Poisson stream of independent requests (seed, L, p, beta, chi, n_samples): L uniform over
    --serve-Ls, p uniform in [0.09, 0.13] with beta on the Nishimori line, chi = min(chi_max,
    2^(L/2)), n_samples uniform in [100, 1000].  Prints one JSON line: proposed spins per second
    over the makespan (first arrival to last completion) and per-request latency percentiles."""
    # one hardware queue per in-flight batch: with fewer queues than streams, a short batch
    # can wait behind a long one that shares its queue
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06538_gb300 as tn
    torch.cuda.set_device(0)
    rng = np.random.default_rng(20240911)
    Ls = [int(x) for x in a.serve_Ls.split(",")]
    N = a.serve_requests
    gaps = rng.exponential(1.0 / a.serve_rate, N)
    reqs = []
    for k in range(N):
        L = int(rng.choice(Ls))
        p = float(rng.uniform(0.09, 0.13))
        chi = int(min(a.serve_chi_max, 2 ** (L // 2)))
        reqs.append((10_000 + k, L, chi, p, tn.nishimori_beta(p), int(rng.integers(100, 1001))))
    clocks = Clocks(0)
    srv = tn.TNMCServer(a.precision, a.chains, 0, chunk=256, max_batch=64, max_inflight=a.serve_inflight,
                        linger_us=int(a.serve_linger_ms * 1000))
    clocks.start()
    t0 = srv.now()
    ids = []
    for k, r in enumerate(reqs):
        target = t0 + gaps[: k + 1].sum()
        while srv.now() < target:
            time.sleep(min(0.001, max(0.0, target - srv.now())))
        ids.append(srv.submit(*r))
    srv.drain()
    res = {}
    while len(res) < N:
        for r in srv.poll(512):
            res[r["id"]] = r
    st = srv.stats()
    last_err = srv.last_error()
    srv.close()
    ck = clocks.stop()
    bad = [r for r in res.values() if r["status"] != 0]
    L_of = {i: reqs[k][1] for k, i in enumerate(ids)}
    fails = {}
    for r in bad:
        key = f"L={L_of[r['id']]} status={r['status']}"
        fails[key] = fails.get(key, 0) + 1
    lat = np.array([res[i]["latency"] for i in ids])
    t_first = min(r["t_submit"] for r in res.values())
    t_last = max(r["t_done"] for r in res.values())
    span = t_last - t_first
    spins = sum(res[i]["n_prop"] * reqs[k][1] ** 2 for k, i in enumerate(ids))
    acc = sum(res[i]["n_acc"] for i in ids)
    by_L = {}
    for k, i in enumerate(ids):
        by_L.setdefault(reqs[k][1], []).append(res[i]["latency"])
    line = {
        "metric": "spins proposed/s under a Poisson request stream (continuous batching)",
        "value": spins / span, "unit": UNIT, "mode": "serve", "n_gpus": 1, "higher_is_better": True,
        "dtype": {"tf32": "f32+tf32", "fp32": "f32", "fp64": "f64", "bf16": "f32+bf16"}[a.precision],
        "data": "synthetic",
        "config": {"workload": f"Poisson {a.serve_rate:g} req/s, {N} requests, L in {Ls}, "
                               f"chi=min({a.serve_chi_max},2^(L/2)), p in [0.09,0.13] Nishimori, "
                               f"n_samples in [100,1000], {a.chains} chains, {a.precision}",
                   "max_inflight": a.serve_inflight, "linger_ms": a.serve_linger_ms, "chunk": 256,
                   "max_batch": 64},
        "makespan_s": span, "accepted_per_s": acc / span, "failed": len(bad), "failures": fails,
        "last_error": last_err,
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "latency_p50_by_L": {str(L): float(np.median(v)) for L, v in sorted(by_L.items())},
        "server": st, "gpu_launches": st["launches"], "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    # a realization whose proposals met a doubly clamped site fails with TNMC_ERR_NUMERIC by
    # design and is reported above; any other failure is an error of the run
    return 0 if all(r["status"] == 4 for r in bad) else 1


def _finish(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
