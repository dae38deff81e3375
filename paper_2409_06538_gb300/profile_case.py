"""One environment build and one proposal sweep of a small synthetic case, for ncu captures:

    python -m paper_2409_06538_gb300.profile_case L chi R precision n

(L x L lattice, cutoff chi, R realizations, precision fp64|fp32|bf16|tf32, n proposals per
chain, two chains, p = 0.109 on the Nishimori line).  Prints the wall times and the Jacobi
statistics of the build."""
import sys
import time

import numpy as np
import torch

import paper_2409_06538_gb300 as tn


def main(argv):
    L, chi, R, prec, n = int(argv[1]), int(argv[2]), int(argv[3]), argv[4], int(argv[5])
    beta = tn.nishimori_beta(0.109)
    seeds = np.arange(R, dtype=np.uint64)
    J = tn.couplings_pmj(L, seeds, 0.109)
    ctx = tn.TNMC(L, J, [beta] * R, seeds, chi, precision=prec, n_chains=2)
    torch.cuda.synchronize()
    t = time.time()
    ctx.build_env(return_logz=False)
    torch.cuda.synchronize()
    tb = time.time() - t
    st = ctx.build_stats()
    t = time.time()
    ctx.propose(n, 0, outputs=False)
    torch.cuda.synchronize()
    ts = time.time() - t
    print(f"L={L} chi={chi} R={R} {prec}: build {tb * 1e3:.1f} ms ({tb / ((L - 1) * L) * 1e6:.1f} us per site step), "
          f"propose {ts * 1e3:.1f} ms, jacobi {st}")
    ctx.close()


if __name__ == "__main__":
    main(sys.argv)
