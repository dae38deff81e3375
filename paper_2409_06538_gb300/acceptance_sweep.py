"""Acceptance probability p_a of the tensor-network proposals against lattice size, bond
dimension and temperature on the Nishimori line (Sec. III.B, acceptance of the tensor-network
proposals, Fig. fig:pa): for every (L, chi, p) it builds the environments of R seeded realizations,
draws n proposals per chain (two chains) and runs the Metropolis filter, then prints one JSON
line with p_a = accepted / proposed (each chain's unconditional first state excluded), its
standard error over realizations, tau ~ 1/p_a and the wall time.  Realizations whose proposals
met a doubly clamped site (TNMC_ERR_NUMERIC) are counted and left out of p_a.

    python -m paper_2409_06538_gb300.acceptance_sweep --Ls 8,16,32 --chis 8,16 --ps 0.10926

``tune_chi`` picks the bond dimension with the least time per accepted proposal from pilots.

Synthetic disorder only (seeded +-J bonds); every step runs in libtnmc.so."""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import tnmc as tn


def run_one(L, chi, p, R, n, precision, seed0):
    beta = tn.nishimori_beta(p)
    seeds = np.arange(seed0, seed0 + R, dtype=np.uint64)
    t0 = time.perf_counter()
    J = tn.couplings_pmj(L, seeds, p)
    ctx = tn.TNMC(L, J, [beta] * R, seeds, chi, precision=precision, n_chains=2)
    ctx.build_env(return_logz=False)
    ctx.propose(n, 0, outputs=False)
    ctx.accept()
    obs = ctx.observables(allow_numeric=True)
    status = ctx.realization_status()
    ctx.close()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ok = [o for o, s in zip(obs, status) if s == 0]
    rates = np.array([o["n_acc"] / max(1, o["n_tests"]) for o in ok])
    pa = float(rates.mean()) if len(rates) else float("nan")
    se = float(rates.std(ddof=1) / math.sqrt(len(rates))) if len(rates) > 1 else 0.0
    return dict(L=L, chi=chi, p=p, T=1.0 / beta, R=R, proposals_per_chain=n, precision=precision,
                p_a=pa, p_a_se=se, tau=(1.0 / pa if pa > 0 else float("inf")),
                failed_realizations=int((status != 0).sum()), clamps=int(sum(o["clamps"] for o in ok)),
                wall_s=wall)


def tune_chi(L, p, chis=(4, 8, 16, 32), R=8, n=100, precision="tf32", seed0=9000):
    """Bond dimension for (L, p) on the Nishimori line that costs least per accepted proposal.

    The paper notes that the time per sweep grows as D^2 while p_a grows with D, so D (chi
    here) is worth tuning against p_a (Sec. IV).  Each candidate runs a pilot of R realizations
    x 2 chains x n proposals; its cost is the pilot's wall time per accepted proposal
    (wall / (p_a * 2 R n)), infinite if any realization met a doubly clamped site.  Returns
    (best chi, list of the pilot records with their cost)."""
    table = []
    for chi in sorted(chis):
        r = run_one(L, chi, p, R, n, precision, seed0)
        ok = r["failed_realizations"] == 0 and r["p_a"] > 0
        r["s_per_accepted"] = r["wall_s"] / (r["p_a"] * 2 * R * n) if ok else float("inf")
        table.append(r)
    best = min(table, key=lambda r: (r["s_per_accepted"], r["chi"]))
    return best["chi"], table


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--Ls", default="8,16,32,64")
    ap.add_argument("--chis", default="4,8,16")
    ap.add_argument("--ps", default="0.10926", help="points on the Nishimori line")
    ap.add_argument("--R", type=int, default=16, help="realizations per point")
    ap.add_argument("--n", type=int, default=200, help="proposals per chain")
    ap.add_argument("--precision", default="tf32", choices=["fp64", "fp32", "bf16", "tf32"])
    ap.add_argument("--max-L-for-chi", default="", help="e.g. '32:256' skips chi=32 above L=256")
    ap.add_argument("--seed0", type=int, default=5000)
    a = ap.parse_args(argv)
    limits = dict(tuple(int(x) for x in kv.split(":")) for kv in a.max_L_for_chi.split(",") if kv)
    rows = []
    for p in [float(x) for x in a.ps.split(",")]:
        for chi in [int(x) for x in a.chis.split(",")]:
            for L in [int(x) for x in a.Ls.split(",")]:
                if chi in limits and L > limits[chi]:
                    continue
                r = run_one(L, chi, p, a.R, a.n, a.precision, a.seed0)
                rows.append(r)
                print(json.dumps(r), flush=True)
    return rows


if __name__ == "__main__":
    main()
