"""Host-side checks of the request-server boundary: the ctypes structures match the C
layouts of include/tnmc.h (compiled here with the host compiler), the capacity estimate
behaves as the allocation formulas say, and invalid server options are refused without a
device."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "tnmc.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("tnmc_opts %zu\n", sizeof(tnmc_opts));
  printf("tnmc_obs %zu\n", sizeof(tnmc_obs));
  printf("tnmc_server_opts %zu\n", sizeof(tnmc_server_opts));
  printf("tnmc_request %zu\n", sizeof(tnmc_request));
  printf("tnmc_result %zu\n", sizeof(tnmc_result));
  F(tnmc_opts, stream); F(tnmc_obs, E); F(tnmc_obs, q4); F(tnmc_obs, m_edge2);
  F(tnmc_server_opts, linger_us); F(tnmc_server_opts, device); F(tnmc_server_opts, mem_budget);
  F(tnmc_request, L); F(tnmc_request, chi); F(tnmc_request, p); F(tnmc_request, beta); F(tnmc_request, n_samples);
  F(tnmc_result, status); F(tnmc_result, batch_size); F(tnmc_result, log_z); F(tnmc_result, obs);
  F(tnmc_result, build_stats); F(tnmc_result, t_submit); F(tnmc_result, t_done);
  return 0;
}
"""


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text(LAYOUT_C)
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_struct_layouts_match_the_header(c_layout):
    from paper_2409_06538_gb300 import _capi
    S = {"tnmc_opts": _capi.Opts, "tnmc_obs": _capi.Obs, "tnmc_server_opts": _capi.ServerOpts,
         "tnmc_request": _capi.Request, "tnmc_result": _capi.Result}
    for cname, py in S.items():
        assert ctypes.sizeof(py) == c_layout[cname], cname
    for key, off in c_layout.items():
        if "." not in key:
            continue
        cname, field = key.split(".")
        assert getattr(S[cname], field).offset == off, key


@pytest.fixture(scope="module")
def lib():
    from paper_2409_06538_gb300 import _capi, build
    build()
    return _capi.load()


def test_estimate_follows_the_allocation_formulas(lib):
    from paper_2409_06538_gb300 import _capi
    opts = _capi.Opts(_capi.PRECISIONS["fp64"], 2, 0, None)
    est = lambda L, R, chi, n: lib.tnmc_estimate_device_bytes(L, R, chi, ctypes.byref(opts), n)
    L, chi = 16, 8
    env = L * L * 2 * chi * chi * 8                      # environment tiles of one realization
    one = est(L, 1, chi, 0)
    assert one > env
    # linear in the number of realizations up to the shared sampler workspace
    d1 = est(L, 2, chi, 0) - est(L, 1, chi, 0)
    d2 = est(L, 3, chi, 0) - est(L, 2, chi, 0)
    assert d1 == d2 and d1 > env
    # proposal buffers: packed spins + log q + energy + magnetisation + current index
    words = (L * L + 31) // 32
    assert est(L, 1, chi, 10) - one == 2 * 10 * (4 * words + 8 + 4 + 4 + 4)
    # chi is rounded up to the compiled tile (8 here); FP64 above 32, any path above 64 and bad
    # arguments give 0; chi = 64 in FP32 adds the M scratch of the environment build
    assert est(L, 1, 7, 0) == one
    assert est(L, 1, 33, 0) == 0 and est(1, 1, chi, 0) == 0 and est(L, 0, chi, 0) == 0
    o32 = _capi.Opts(_capi.PRECISIONS["fp32"], 2, 0, None)
    e64 = lib.tnmc_estimate_device_bytes(L, 1, 64, ctypes.byref(o32), 0)
    assert e64 >= L * L * 2 * 64 * 64 * 4 + 128 * 128 * 4
    assert lib.tnmc_estimate_device_bytes(L, 1, 65, ctypes.byref(o32), 0) == 0


def test_server_refuses_bad_options_without_a_device(lib):
    from paper_2409_06538_gb300 import _capi
    h = ctypes.c_void_p()
    bad = _capi.ServerOpts(0, 0, 0, 256, 8, 2, 0, 0, 0)    # n_chains = 0
    assert lib.tnmc_server_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    assert lib.tnmc_server_create(None, ctypes.byref(h)) == 1
    assert lib.tnmc_server_submit(None, None, None) == 1
    assert lib.tnmc_server_poll(None, None, 1) == 0
    assert lib.tnmc_server_destroy(None) == 0
