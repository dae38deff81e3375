"""Python binding of the TNMC C ABI.  PyTorch provides device buffers and the CUDA stream;
all arithmetic of the method runs in libtnmc.so."""
import ctypes

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


class _TorchAllocator:
    """Device memory for a context from PyTorch's caching allocator (tnmc_opts.alloc / free):
    stream-ordered blocks on the context's stream, returned to PyTorch's cache on release."""

    def __init__(self, device):
        self.device = int(device)

        def alloc(nbytes, stream, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=int(stream or 0))
            except Exception:          # out of memory: the library reports TNMC_ERR_OOM
                return None

        def free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _capi.ALLOC_FN(alloc)
        self.free = _capi.FREE_FN(free)


def nishimori_beta(p):
    """Inverse temperature on the Nishimori line, exp(-2/T) = p/(1-p) (tnmc_nishimori_beta)."""
    out = _c.c_double(0.0)
    _capi.check(_capi.load().tnmc_nishimori_beta(float(p), _c.byref(out)))
    return out.value


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

    def __init__(self, L, couplings, beta, seeds, chi, precision="fp64", n_chains=2, n_therm=0, stream=None,
                 allocator="torch", compression="canonical"):
        """allocator: "torch" -- device buffers come from PyTorch's caching allocator through the
        library's allocator hooks; "library" -- the library allocates them itself.
        compression: "canonical" (QR + SVD sweeps) or "zipup" (tnmc_compression)."""
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
        opts.compression = _capi.COMPRESSIONS[compression]
        if allocator == "torch":
            # kept alive with the context: the library calls it until tnmc_destroy
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            opts.alloc, opts.free = self._alloc.alloc, self._alloc.free
        elif allocator != "library":
            raise ValueError(f"unknown allocator {allocator!r}")
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

    def realization_status_async(self, out):
        """Queue a copy of the per-realization status words into `out` (int32 cuda tensor of
        n_real; 0 = no failure) on this context's stream, without synchronising."""
        assert out.is_cuda and out.dtype == torch.int32 and out.numel() >= self.n_real
        self._chk(self.lib.tnmc_realization_status_async(self.ctx, _ptr(out)))

    def set_fields(self, fields):
        """External fields in units of beta (int8 [R, L, L], host array or cuda tensor; None
        removes them): the weight gains exp(beta sum k s).  Build the environments again."""
        if fields is None:
            self._chk(self.lib.tnmc_set_fields(self.ctx, None))
            return
        if isinstance(fields, torch.Tensor):
            f = fields.contiguous()
            self._chk(self.lib.tnmc_set_fields(self.ctx, _ptr(f)))
        else:
            f = np.ascontiguousarray(np.asarray(fields, dtype=np.int8))
            self._chk(self.lib.tnmc_set_fields(self.ctx, _c.c_void_p(f.ctypes.data)))

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


def torus_couplings_pmj(L, seeds, p, stream=None):
    """Seeded +-J couplings of len(seeds) L x L tori on the device: int8 [R, 2 L^2]."""
    lib = _capi.load()
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    out = torch.empty((len(seeds), 2 * L * L), dtype=torch.int8, device="cuda")
    _capi.check(lib.tnmc_torus_couplings_pmj(L, len(seeds), seeds.ctypes.data_as(_capi.c_uint64_p), float(p),
                                             _ptr(out), _stream_handle(stream)))
    return out


class TNMCPeriodic:
    """n_real torus realizations sampled with a pinned pair of lines per step (Sec. IV), behind
    tnmc_periodic_*."""

    def __init__(self, L, couplings, beta, seeds, chi, precision="fp64", n_chains=2, n_therm=0, stream=None,
                 allocator="torch"):
        self.lib = _capi.load()
        self.L, self.chi, self.n_chains = int(L), int(chi), int(n_chains)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        self.n_real = len(seeds)
        beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.n_real,)))
        J = couplings.contiguous() if isinstance(couplings, torch.Tensor) else \
            np.ascontiguousarray(np.asarray(couplings, dtype=np.int8))
        jp = _c.c_void_p(J.data_ptr() if isinstance(J, torch.Tensor) else J.ctypes.data)
        opts = _capi.Opts(_capi.PRECISIONS[precision], self.n_chains, int(n_therm), _stream_handle(self.stream))
        if allocator == "torch":
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            opts.alloc, opts.free = self._alloc.alloc, self._alloc.free
        ctx = _c.c_void_p()
        code = self.lib.tnmc_periodic_create(self.L, self.n_real, jp, beta.ctypes.data_as(_capi.c_double_p),
                                             seeds.ctypes.data_as(_capi.c_uint64_p), self.chi, _c.byref(opts),
                                             _c.byref(ctx))
        if code != 0:
            msg = self.lib.tnmc_periodic_last_error(None)
            raise _capi.TnmcError(code, msg.decode() if msg else "")
        self.ctx = ctx
        self._keep = (J, beta, seeds)

    def _chk(self, code):
        if code != 0:
            msg = self.lib.tnmc_periodic_last_error(self.ctx)
            raise _capi.TnmcError(code, msg.decode() if msg else "")

    def step(self, n, step0=0):
        self._chk(self.lib.tnmc_periodic_step(self.ctx, int(n), int(step0)))

    def spins(self):
        out = torch.empty((self.n_real, self.n_chains, self.L, self.L), dtype=torch.int8, device="cuda")
        self._chk(self.lib.tnmc_periodic_get_spins(self.ctx, _ptr(out)))
        return out

    def observables(self):
        arr = (_capi.Obs * self.n_real)()
        self._chk(self.lib.tnmc_periodic_observables(self.ctx, arr))
        return [{k: getattr(o, k) for k, _ in _capi.Obs._fields_} for o in arr]

    def launch_count(self):
        return int(self.lib.tnmc_periodic_launch_count(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.tnmc_periodic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def disorder_average(obs, L, beta):
    """Disorder averages of per-realization thermal means (tnmc_disorder_average): for each
    quantity (mean, standard error), the Binder ratios U_m and Q_q, [<q^2>^2], the
    susceptibilities chi_q and chi_edge and the acceptance rate, over the realizations whose
    status is 0 (n_used; n_dropped were flagged).  obs: dicts as TNMC.observables() returns."""
    lib = _capi.load()
    arr = (_capi.Obs * len(obs))()
    for o, d in zip(arr, obs):
        for k, _ in _capi.Obs._fields_:
            if k in d:
                setattr(o, k, d[k])
    res = _capi.Disorder()
    code = lib.tnmc_disorder_average(arr, len(obs), int(L), float(beta), _c.byref(res))
    if code not in (0, 4):
        _capi.check(code)
    out = {k: (res.mean[i], res.se[i]) for i, k in enumerate(_capi.DIS_KEYS)}
    for k in ("U_m", "Q_q", "q2_sq", "chi_q", "chi_edge", "acceptance", "n_used", "n_dropped", "n_prop",
              "n_tests", "n_acc", "clamps"):
        out[k] = getattr(res, k)
    return out
