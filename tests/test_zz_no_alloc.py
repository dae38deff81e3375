"""The allocation-free environment build gives the same environments and log Z as the
regular entry point.  It is for callers that cannot call cudaMalloc (an application that
reserves all device memory up front, or a path that must not take cudaMalloc's device-wide
synchronisation); this file is collected last so that a failure here leaves every other
test already run."""
import ctypes

import numpy as np
import pytest

from oracle import lattice

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc_build(lib, L, chi, precision, J, beta, stream):
    R = J.shape[0]
    C = 4 if chi <= 4 else 8 if chi <= 8 else 16 if chi <= 16 else 32
    el = 8 if precision == 0 else (2 if precision == 2 else 4)
    env = torch.zeros(R * L * L * 2 * C * C * el, dtype=torch.uint8, device="cuda")
    kdim = torch.zeros((R, L, L + 1), dtype=torch.int32, device="cuda")
    lam = torch.zeros((R, L), dtype=torch.float64, device="cuda")
    logz = torch.zeros(R, dtype=torch.float64, device="cuda")
    bdev = torch.tensor(beta, dtype=torch.float64, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    code = lib.tnmc_build_env_noalloc(L, R, chi, precision, vp(J), vp(bdev), vp(env), vp(kdim), vp(lam), vp(logz),
                                      ctypes.c_void_p(stream.cuda_stream))
    assert code == 0
    stream.synchronize()
    raw = env.cpu().numpy()
    if precision == 2:      # bfloat16: the high half of a float32
        tiles = (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32)
    else:
        tiles = raw.view(np.float64 if precision == 0 else np.float32)
    tiles = tiles.reshape(R, L, L, 2, C, C)
    return tiles, kdim.cpu().numpy(), lam.cpu().numpy(), logz.cpu().numpy(), C


@pytest.mark.parametrize("precision_name,precision,tol", [("fp64", 0, 1e-12), ("fp32", 1, 1e-5), ("bf16", 2, 1e-5),
                                                          ("tf32", 3, 1e-5)])
def test_noalloc_matches_regular_build_twice(precision_name, precision, tol):
    import paper_2409_06538_gb300 as tn
    from paper_2409_06538_gb300 import _capi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tn.build()
    lib = _capi.load()
    L, chi, p = 12, 6, 0.109
    beta = lattice.nishimori_beta(p)
    stream = torch.cuda.current_stream()
    for call, seeds in enumerate(([1, 2, 3], [40, 41, 42, 43])):
        J = tn.couplings_pmj(L, seeds, p)
        ctx = tn.TNMC(L, J, [beta] * len(seeds), seeds, chi, precision=precision_name)
        lz_ref = ctx.build_env()
        tiles, kdim, lam, logz, C = _noalloc_build(lib, L, chi, precision, J, [beta] * len(seeds), stream)
        assert np.abs(logz - lz_ref).max() <= tol * np.abs(lz_ref).max(), f"call {call}"
        for k in range(len(seeds)):
            for r in range(L):
                t_ref, d_ref, lam_ref = ctx.copy_env(k, r)
                assert np.array_equal(kdim[k, r], d_ref)
                assert abs(lam[k, r] - lam_ref) <= tol * max(1.0, abs(lam_ref))
                got = tiles[k, r][:, :, :chi, :chi].astype(np.float64)
                assert np.abs(got - t_ref).max() <= tol, f"call {call} real {k} row {r}"
        ctx.close()


def test_noalloc_rejects_oversized_requests():
    import paper_2409_06538_gb300 as tn
    from paper_2409_06538_gb300 import _capi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tn.build()
    lib = _capi.load()
    L, chi, R = 256, 32, 64          # needs far more than the 32 MiB scratch array
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    vp = ctypes.c_void_p(dummy.data_ptr())
    code = lib.tnmc_build_env_noalloc(L, R, chi, 1, vp, vp, vp, vp, vp, vp, None)
    assert code == 1                 # TNMC_ERR_ARG, nothing launched
