"""Host-side checks of the C ABI: the library builds for sm_103a, loads,
exports every symbol include/rt.h declares, the ctypes mirror matches the C
struct layout, and calls with bad arguments fail cleanly (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rt.h")


@pytest.fixture(scope="module")
def L():
    from paper_2606_02413_gb300 import _abi, build
    build.build()
    return _abi.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:rt_status|void|const char\*)\s+(rt_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(L):
    from paper_2606_02413_gb300 import _abi
    names = declared_functions()
    assert len(names) >= 10
    assert sorted(_abi.EXPORTS) == names
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2606_02413_gb300", "librt.so")],
                         capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_struct_layout_matches_header(tmp_path):
    from paper_2606_02413_gb300 import _abi
    probe = tmp_path / "probe.c"
    probe.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rt.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("rt_grid_desc %zu\nrt_view %zu\nrt_options %zu\nrt_ray_diag %zu\nrt_stats %zu\n",
         sizeof(rt_grid_desc), sizeof(rt_view), sizeof(rt_options), sizeof(rt_ray_diag), sizeof(rt_stats));
  P(rt_options, eta) P(rt_options, tau_stop) P(rt_options, max_steps) P(rt_options, tbc_K)
  P(rt_options, precision) P(rt_view, x0) P(rt_grid_desc, dtype) P(rt_ray_diag, steps)
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(probe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(got["rt_grid_desc"]) == C.sizeof(_abi.GridDesc)
    assert int(got["rt_view"]) == C.sizeof(_abi.View)
    assert int(got["rt_options"]) == C.sizeof(_abi.Options)
    assert int(got["rt_ray_diag"]) == C.sizeof(_abi.RayDiag)
    assert int(got["rt_stats"]) == C.sizeof(_abi.Stats)
    for key, (cls, field) in {"rt_options.eta": (_abi.Options, "eta"), "rt_options.tau_stop": (_abi.Options, "tau_stop"),
                              "rt_options.max_steps": (_abi.Options, "max_steps"),
                              "rt_options.tbc_K": (_abi.Options, "tbc_K"),
                              "rt_options.precision": (_abi.Options, "precision"), "rt_view.x0": (_abi.View, "x0"),
                              "rt_grid_desc.dtype": (_abi.GridDesc, "dtype"),
                              "rt_ray_diag.steps": (_abi.RayDiag, "steps")}.items():
        assert int(got[key]) == getattr(cls, field).offset, key


def test_defaults_and_strings(L):
    import paper_2606_02413_gb300 as rt
    o = rt.options()
    assert o.dtau == 2e-3 and o.n_nb == 4 and o.eta == 0.5 and o.tau_stop == 30.0 and o.emission == 1
    assert L.rt_status_string(0) == b"RT_OK"
    assert L.rt_status_string(-2) == b"RT_ERR_GRID"


def test_null_arguments_fail_cleanly(L):
    from paper_2606_02413_gb300 import _abi
    assert L.rt_trace_image(None, None, None, None, 1, None, None, None, None) == _abi.RT_ERR_ARG
    assert b"NULL" in L.rt_last_error()
    assert L.rt_load_grid(None, None, None, None, None, None) == _abi.RT_ERR_ARG
    assert L.rt_create(None, 0) == _abi.RT_ERR_ARG
    assert L.rt_destroy(None) == _abi.RT_ERR_ARG
    assert L.rt_sync(None, None) == _abi.RT_ERR_ARG
    assert L.rt_get_stats(None, None, None) == _abi.RT_ERR_ARG
    assert L.rt_trace_image_tape(None, None, None, None, 1, None, 0, None, None, None, None) == _abi.RT_ERR_ARG
    assert L.rt_backward_tape(None, None, None, None, None) == _abi.RT_ERR_ARG
    assert L.rt_tape_info(None, None, None, None) == _abi.RT_ERR_ARG
    assert L.rt_tape_free(None) == _abi.RT_ERR_ARG


def test_no_gpu_is_an_error_not_a_fallback(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_02413_gb300 import _abi
    h = C.c_void_p()
    rc = L.rt_create(C.byref(h), 0)
    assert rc in (_abi.RT_ERR_CUDA, _abi.RT_ERR_ARG)
    assert not h.value
