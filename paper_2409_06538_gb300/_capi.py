"""ctypes declarations of the C ABI in include/tnmc.h.  Marshalling only: every step of the
method runs in libtnmc.so.  Importing fails loudly when the library has not been built;
there is no fallback implementation."""
import ctypes
import os

from . import buildlib as _build

c_int, c_int64, c_size_t, c_double, c_void_p = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double, ctypes.c_void_p
c_uint64_p = ctypes.POINTER(ctypes.c_uint64)
c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64_p = ctypes.POINTER(ctypes.c_int64)

STATUS = {0: "TNMC_OK", 1: "TNMC_ERR_ARG", 2: "TNMC_ERR_OOM", 3: "TNMC_ERR_CUDA", 4: "TNMC_ERR_NUMERIC",
          5: "TNMC_ERR_TIMEOUT", 6: "TNMC_ERR_STATE", 7: "TNMC_ERR_UNSUPPORTED"}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "tf32": 3}

# Entry points declared in include/tnmc.h: name -> (restype, argtypes)
SIGNATURES = {
    "tnmc_version": (c_int, []),
    "tnmc_couplings_pmj": (c_int, [c_int, c_int, c_uint64_p, c_double, c_void_p, c_void_p]),
    "tnmc_create": (c_int, [c_int, c_int, c_void_p, c_double_p, c_uint64_p, c_int, c_void_p,
                            ctypes.POINTER(c_void_p)]),
    "tnmc_set_couplings": (c_int, [c_void_p, c_void_p, c_double_p, c_uint64_p]),
    "tnmc_set_realizations": (c_int, [c_void_p, c_uint64_p, c_double_p, c_double]),
    "tnmc_build_env": (c_int, [c_void_p, c_double_p]),
    "tnmc_propose": (c_int, [c_void_p, c_int, ctypes.c_uint64, c_void_p, c_void_p, c_void_p]),
    "tnmc_get_spins": (c_int, [c_void_p, c_void_p]),
    "tnmc_eval_conditionals": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "tnmc_accept": (c_int, [c_void_p, c_void_p, c_int64_p]),
    "tnmc_observables": (c_int, [c_void_p, c_void_p]),
    "tnmc_reset_chains": (c_int, [c_void_p]),
    "tnmc_destroy": (c_int, [c_void_p]),
    "tnmc_last_error": (ctypes.c_char_p, [c_void_p]),
    "tnmc_env_bytes": (c_size_t, [c_void_p]),
    "tnmc_copy_env": (c_int, [c_void_p, c_int, c_int, c_double_p, c_int32_p, c_double_p]),
    "tnmc_launch_count": (c_int64, [c_void_p]),
    "tnmc_build_stats": (c_int, [c_void_p, c_int64_p]),
    "tnmc_build_env_noalloc": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p]),
    "tnmc_device_bytes": (c_size_t, [c_void_p]),
    "tnmc_selftest_bounded_wait": (c_int, [c_int, c_int64_p]),
    "tnmc_env_build_occupancy": (c_int, [c_int, c_int, c_int, c_int32_p, c_int32_p]),
    "tnmc_realization_status": (c_int, [c_void_p, c_int32_p]),
    "tnmc_realization_status_async": (c_int, [c_void_p, c_void_p]),
    "tnmc_disorder_average": (c_int, [c_void_p, c_int, c_int, c_double, c_void_p]),
    "tnmc_nishimori_beta": (c_int, [c_double, c_double_p]),
    "tnmc_estimate_device_bytes": (c_size_t, [c_int, c_int, c_int, c_void_p, c_int]),
    "tnmc_set_fields": (c_int, [c_void_p, c_void_p]),
    "tnmc_torus_couplings_pmj": (c_int, [c_int, c_int, c_uint64_p, c_double, c_void_p, c_void_p]),
    "tnmc_periodic_create": (c_int, [c_int, c_int, c_void_p, c_double_p, c_uint64_p, c_int, c_void_p,
                                     ctypes.POINTER(c_void_p)]),
    "tnmc_periodic_step": (c_int, [c_void_p, c_int, ctypes.c_uint64]),
    "tnmc_periodic_observables": (c_int, [c_void_p, c_void_p]),
    "tnmc_periodic_get_spins": (c_int, [c_void_p, c_void_p]),
    "tnmc_periodic_launch_count": (c_int64, [c_void_p]),
    "tnmc_periodic_last_error": (ctypes.c_char_p, [c_void_p]),
    "tnmc_periodic_destroy": (c_int, [c_void_p]),
    "tnmc_server_create": (c_int, [c_void_p, ctypes.POINTER(c_void_p)]),
    "tnmc_server_submit": (c_int, [c_void_p, c_void_p, c_int64_p]),
    "tnmc_server_poll": (c_int, [c_void_p, c_void_p, c_int]),
    "tnmc_server_wait": (c_int, [c_void_p, c_int64, c_double, c_void_p]),
    "tnmc_server_drain": (c_int, [c_void_p, c_double]),
    "tnmc_server_stats": (c_int, [c_void_p, c_int64_p]),
    "tnmc_server_last_error": (ctypes.c_char_p, [c_void_p]),
    "tnmc_server_now": (c_double, [c_void_p]),
    "tnmc_server_destroy": (c_int, [c_void_p]),
}


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


COMPRESSIONS = {"canonical": 0, "zipup": 1}


class Opts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("n_chains", c_int), ("n_therm", c_int), ("stream", c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", c_void_p), ("compression", c_int)]


class Obs(ctypes.Structure):
    _fields_ = [("n_prop", c_int64), ("n_acc", c_int64), ("n_meas", c_int64), ("n_meas_q", c_int64),
                ("clamps", c_int64), ("E", c_double), ("E2", c_double), ("m_abs", c_double),
                ("m2", c_double), ("m4", c_double), ("q", c_double), ("q_abs", c_double),
                ("q2", c_double), ("q4", c_double), ("m_edge", c_double), ("m_edge_abs", c_double),
                ("m_edge2", c_double), ("n_tests", c_int64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


# order of the mean / se arrays of tnmc_disorder
DIS_KEYS = ["E", "E2", "m_abs", "m2", "m4", "q", "q_abs", "q2", "q4", "m_edge", "m_edge_abs", "m_edge2"]


class Disorder(ctypes.Structure):
    _fields_ = [("n_used", ctypes.c_int32), ("n_dropped", ctypes.c_int32),
                ("mean", c_double * len(DIS_KEYS)), ("se", c_double * len(DIS_KEYS)),
                ("U_m", c_double), ("Q_q", c_double), ("q2_sq", c_double), ("chi_q", c_double),
                ("chi_edge", c_double), ("acceptance", c_double), ("n_prop", c_int64), ("n_tests", c_int64),
                ("n_acc", c_int64), ("clamps", c_int64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("n_chains", c_int), ("n_therm", c_int), ("chunk", c_int),
                ("max_batch", c_int), ("max_inflight", c_int), ("linger_us", c_int), ("device", c_int),
                ("mem_budget", c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("L", c_int), ("chi", c_int), ("p", c_double), ("beta", c_double),
                ("n_samples", c_int)]


class Result(ctypes.Structure):
    _fields_ = [("id", c_int64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("log_z", c_double),
                ("obs", Obs), ("build_stats", c_int64 * 4), ("t_submit", c_double), ("t_start", c_double),
                ("t_done", c_double)]


class TnmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def load(path=None):
    """Load libtnmc.so (built in-tree by __graft_entry__.build() / build.py)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or _build.lib_path()
    if not os.path.exists(p):
        raise ImportError(f"libtnmc.so is not built ({p}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def check(code, ctx=None):
    if code != 0:
        lib = load()
        msg = lib.tnmc_last_error(ctx)
        raise TnmcError(code, msg.decode() if msg else "")
