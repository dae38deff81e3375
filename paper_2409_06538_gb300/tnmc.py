"""Python binding of the TNMC C ABI.  PyTorch provides device buffers and the CUDA stream;
all arithmetic of the method runs in libtnmc.so."""
import ctypes
import math

import numpy as np
import torch

from . import _capi

_c = ctypes


def _ptr(t):
    return _c.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return _c.c_void_p(stream.cuda_stream)


def nishimori_beta(p):
    """Inverse temperature on the Nishimori line exp(-2/T) = p/(1-p), |J| = 1."""
    return 0.5 * math.log((1.0 - p) / p)


def env_build_occupancy(L, chi, precision="tf32"):
    """(realizations per SM, SM count) for the environment build on the current device."""
    lib = _capi.load()
    per, sms = _c.c_int32(0), _c.c_int32(0)
    _capi.check(lib.tnmc_env_build_occupancy(int(L), int(chi), _capi.PRECISIONS[precision], _c.byref(per),
                                             _c.byref(sms)))
    return per.value, sms.value


def couplings_pmj(L, seeds, p, stream=None):
    """Seeded +-J couplings of len(seeds) realizations on the device: int8 [R, 2L(L-1)]."""
    lib = _capi.load()
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    out = torch.empty((len(seeds), 2 * L * (L - 1)), dtype=torch.int8, device="cuda")
    _capi.check(lib.tnmc_couplings_pmj(L, len(seeds), seeds.ctypes.data_as(_capi.c_uint64_p), float(p),
                                       _ptr(out), _stream_handle(stream)))
    return out


class TNMC:
    """n_real realizations of one (L, chi) bucket behind one library context."""

    def __init__(self, L, couplings, beta, seeds, chi, precision="fp64", n_chains=2, n_therm=0, stream=None):
        self.lib = _capi.load()
        self.L, self.chi, self.n_chains = int(L), int(chi), int(n_chains)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        self.n_real = len(seeds)
        beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.n_real,)))
        if isinstance(couplings, torch.Tensor):
            J = couplings.contiguous()
            jp = _c.c_void_p(J.data_ptr())
        else:
            J = np.ascontiguousarray(np.asarray(couplings, dtype=np.int8))
            jp = _c.c_void_p(J.ctypes.data)
        self._keep = (J, beta, seeds)
        opts = _capi.Opts(_capi.PRECISIONS[precision], self.n_chains, int(n_therm),
                          _stream_handle(self.stream))
        ctx = _c.c_void_p()
        code = self.lib.tnmc_create(self.L, self.n_real, jp, beta.ctypes.data_as(_capi.c_double_p),
                                    seeds.ctypes.data_as(_capi.c_uint64_p), self.chi, _c.byref(opts),
                                    _c.byref(ctx))
        _capi.check(code, None)
        self.ctx = ctx
        self.precision = precision
        self.last_n = 0

    def set_couplings(self, couplings, beta, seeds):
        """New realizations for this context (host numpy/pinned tensor or device tensor)."""
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.n_real,)))
        if isinstance(couplings, torch.Tensor):
            J = couplings.contiguous()
            jp = _c.c_void_p(J.data_ptr())
        else:
            J = np.ascontiguousarray(np.asarray(couplings, dtype=np.int8))
            jp = _c.c_void_p(J.ctypes.data)
        self._chk(self.lib.tnmc_set_couplings(self.ctx, jp, beta.ctypes.data_as(_capi.c_double_p),
                                              seeds.ctypes.data_as(_capi.c_uint64_p)))
        self._keep = (J, beta, seeds)

    def set_realizations(self, seeds, beta, p):
        """New realizations from seeds: couplings generated on the device, asynchronously."""
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.n_real,)))
        self._chk(self.lib.tnmc_set_realizations(self.ctx, seeds.ctypes.data_as(_capi.c_uint64_p),
                                                 beta.ctypes.data_as(_capi.c_double_p), float(p)))

    def _chk(self, code):
        _capi.check(code, self.ctx)

    def build_env(self, return_logz=True):
        if return_logz:
            lz = np.zeros(self.n_real)
            self._chk(self.lib.tnmc_build_env(self.ctx, lz.ctypes.data_as(_capi.c_double_p)))
            return lz
        self._chk(self.lib.tnmc_build_env(self.ctx, None))
        return None

    def propose(self, n, step0=0, outputs=True):
        """Draw n proposals per chain; returns device tensors [R, chains, n] (or None)."""
        shape = (self.n_real, self.n_chains, n)
        if outputs:
            lq = torch.empty(shape, dtype=torch.float64, device="cuda")
            E = torch.empty(shape, dtype=torch.int32, device="cuda")
            M = torch.empty(shape, dtype=torch.int32, device="cuda")
            self._chk(self.lib.tnmc_propose(self.ctx, n, step0, _ptr(lq), _ptr(E), _ptr(M)))
            self.last_n = n
            return dict(logq=lq, energy=E, magnet=M)
        self._chk(self.lib.tnmc_propose(self.ctx, n, step0, None, None, None))
        self.last_n = n
        return None

    def spins(self):
        out = torch.empty((self.n_real, self.n_chains, self.last_n, self.L, self.L), dtype=torch.int8, device="cuda")
        self._chk(self.lib.tnmc_get_spins(self.ctx, _ptr(out)))
        return out

    def eval_conditionals(self, spins, want_qplus=True):
        """Teacher-forced q on spins (int8 cuda [R, n, L, L]); returns (logq [R,n], qplus [R,n,L,L])."""
        spins = spins.contiguous()
        R, n = spins.shape[0], spins.shape[1]
        assert R == self.n_real
        lq = torch.empty((R, n), dtype=torch.float64, device="cuda")
        qp = torch.empty((R, n, self.L, self.L), dtype=torch.float64, device="cuda") if want_qplus else None
        self._chk(self.lib.tnmc_eval_conditionals(self.ctx, n, _ptr(spins), _ptr(lq), _ptr(qp)))
        return lq, qp

    def accept(self, flags=False, count=False):
        acc = torch.empty((self.n_real, self.n_chains, self.last_n), dtype=torch.uint8, device="cuda") if flags else None
        cnt = _c.c_int64(0)
        self._chk(self.lib.tnmc_accept(self.ctx, _ptr(acc), _c.byref(cnt) if count else None))
        return dict(flags=acc, count=cnt.value if count else None)

    def observables(self, allow_numeric=False):
        """Per-realization thermal means.  With allow_numeric, a numeric failure of some
        realizations does not raise: check realization_status() to drop them."""
        arr = (_capi.Obs * self.n_real)()
        code = self.lib.tnmc_observables(self.ctx, arr)
        if not (allow_numeric and code == 4):
            self._chk(code)
        return [{k: getattr(o, k) for k, _ in _capi.Obs._fields_} for o in arr]

    def reset_chains(self):
        self._chk(self.lib.tnmc_reset_chains(self.ctx))

    def copy_env(self, real, row):
        tiles = np.zeros((self.L, 2, self.chi, self.chi))
        dims = np.zeros(self.L + 1, dtype=np.int32)
        lam = np.zeros(1)
        self._chk(self.lib.tnmc_copy_env(self.ctx, real, row, tiles.ctypes.data_as(_capi.c_double_p),
                                         dims.ctypes.data_as(_capi.c_int32_p), lam.ctypes.data_as(_capi.c_double_p)))
        return tiles, dims, float(lam[0])

    def build_stats(self):
        """Jacobi statistics of the last environment build (max sweeps, unconverged, total
        sweeps, number of truncating SVDs)."""
        out = (_c.c_int64 * 4)()
        self._chk(self.lib.tnmc_build_stats(self.ctx, out))
        return dict(max_sweeps=out[0], unconverged=out[1], total_sweeps=out[2], svds=out[3],
                    mean_sweeps=out[2] / max(1, out[3]))

    def realization_status(self):
        """Per-realization status codes (0 ok, 4 = a numeric failure in its proposals)."""
        out = np.zeros(self.n_real, dtype=np.int32)
        self._chk(self.lib.tnmc_realization_status(self.ctx, out.ctypes.data_as(_capi.c_int32_p)))
        return out

    def device_bytes(self):
        return int(self.lib.tnmc_device_bytes(self.ctx))

    def env_bytes(self):
        return int(self.lib.tnmc_env_bytes(self.ctx))

    def launch_count(self):
        return int(self.lib.tnmc_launch_count(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.tnmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def disorder_average(obs, L=None, beta=None):
    """Disorder means [.] and standard errors over per-realization thermal means, with the
    Binder ratios U_m = [<m^4>]/[<m^2>]^2 and Q_q = [<q^4>]/[<q^2>]^2, and given L (and beta)
    the susceptibilities chi_q = (L^2/T)([<q^2>] - [<q>]^2) and chi_edge = L [<m_edge^2>]
    (Sec. III.C, Eq. eq:susEA)."""
    keys = ["E", "E2", "m_abs", "m2", "m4", "q", "q_abs", "q2", "q4", "m_edge", "m_edge_abs", "m_edge2"]
    keys = [k for k in keys if k in obs[0]]
    R = len(obs)
    out = {}
    for k in keys:
        x = np.array([o[k] for o in obs])
        out[k] = (float(x.mean()), float(x.std(ddof=1) / math.sqrt(R)) if R > 1 else 0.0)
    out["U_m"] = out["m4"][0] / out["m2"][0] ** 2 if out["m2"][0] > 0 else float("nan")
    out["Q_q"] = out["q4"][0] / out["q2"][0] ** 2 if out["q2"][0] > 0 else float("nan")
    nacc = sum(o["n_acc"] for o in obs)
    nprop = sum(o["n_prop"] for o in obs)
    out["acceptance"] = nacc / max(1, nprop)
    out["clamps"] = int(sum(o["clamps"] for o in obs))
    if L is not None and beta is not None:
        out["chi_q"] = L * L * beta * (out["q2"][0] - out["q"][0] ** 2)
    if L is not None and "m_edge2" in out:
        out["chi_edge"] = L * out["m_edge2"][0]
    return out
