"""Python binding of the TNMC request server (continuous batching of independent
realizations, one scheduler thread in libtnmc.so).  Marshalling only."""
import ctypes

from . import _capi

_c = ctypes


def _result_dict(r):
    d = {k: getattr(r.obs, k) for k, _ in _capi.Obs._fields_}
    d.update(id=r.id, status=r.status, batch_size=r.batch_size, log_z=r.log_z,
             build_stats=list(r.build_stats), t_submit=r.t_submit, t_start=r.t_start, t_done=r.t_done,
             latency=r.t_done - r.t_submit)
    return d


class TNMCServer:
    """Submit (seed, L, chi, p, beta, n_samples) requests from any thread; results come back
    per request as their batch finishes.  A request's result is the same alone or in any mix."""

    def __init__(self, precision="tf32", n_chains=2, n_therm=0, chunk=256, max_batch=64, max_inflight=4,
                 linger_us=0, device=0, mem_budget=0):
        self.lib = _capi.load()
        opts = _capi.ServerOpts(_capi.PRECISIONS[precision], int(n_chains), int(n_therm), int(chunk),
                                int(max_batch), int(max_inflight), int(linger_us), int(device), int(mem_budget))
        h = _c.c_void_p()
        code = self.lib.tnmc_server_create(_c.byref(opts), _c.byref(h))
        if code != 0:
            raise _capi.TnmcError(code, "tnmc_server_create: invalid options or device")
        self.h = h

    def _chk(self, code):
        if code != 0:
            msg = self.lib.tnmc_server_last_error(self.h)
            raise _capi.TnmcError(code, msg.decode() if msg else "")

    def submit(self, seed, L, chi, p, beta, n_samples):
        req = _capi.Request(int(seed), int(L), int(chi), float(p), float(beta), int(n_samples))
        rid = _c.c_int64(0)
        self._chk(self.lib.tnmc_server_submit(self.h, _c.byref(req), _c.byref(rid)))
        return rid.value

    def wait(self, rid, timeout=-1.0):
        r = _capi.Result()
        self._chk(self.lib.tnmc_server_wait(self.h, int(rid), float(timeout), _c.byref(r)))
        return _result_dict(r)

    def poll(self, max_results=256):
        arr = (_capi.Result * max_results)()
        n = self.lib.tnmc_server_poll(self.h, arr, max_results)
        return [_result_dict(arr[i]) for i in range(n)]

    def drain(self, timeout=-1.0):
        self._chk(self.lib.tnmc_server_drain(self.h, float(timeout)))

    def last_error(self):
        msg = self.lib.tnmc_server_last_error(self.h)
        return msg.decode() if msg else ""

    def now(self):
        return float(self.lib.tnmc_server_now(self.h))

    def stats(self):
        out = (_c.c_int64 * 8)()
        self._chk(self.lib.tnmc_server_stats(self.h, out))
        keys = ["submitted", "completed", "failed", "batches", "contexts_created", "contexts_evicted",
                "peak_bytes", "launches"]
        return dict(zip(keys, list(out)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.tnmc_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
