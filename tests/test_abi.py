"""CPU checks of the C ABI: the library builds, loads, exports every entry
point declared in include/pasd.h, and the ctypes structs match the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pasd.h")


@pytest.fixture(scope="module")
def P():
    from paper_1712_09999_gb300 import build
    build.build()
    from paper_1712_09999_gb300 import pasd
    pasd.lib()
    return pasd


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pasd_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pasd_plan", "pasd_solve", "pasd_submit", "pasd_poll"):
        assert required in names


def test_library_exports_every_declared_symbol(P):
    lib = ctypes.CDLL(P.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pasd_\w+)", out))
    assert set(_declared_functions()) <= exported


def test_binding_covers_every_entry_point(P):
    for name in _declared_functions():
        assert name in P._SIGS, name
        assert callable(getattr(P, name)), name


def test_struct_layouts_match_c(P):
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "pasd.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(pasd_params), offsetof(pasd_params, lambda),
         offsetof(pasd_params, mu0), offsetof(pasd_params, flags), sizeof(pasd_result),
         offsetof(pasd_result, kept), offsetof(pasd_result, latency_s));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    p, r = P.pasd_params, P.pasd_result
    assert vals == [ctypes.sizeof(p), p.lambda_.offset, p.mu0.offset, p.flags.offset,
                    ctypes.sizeof(r), r.kept.offset, r.latency_s.offset]


def test_host_only_entry_points(P):
    assert P.pasd_status_string(P.OK) == "PASD_OK"
    assert P.pasd_status_string(P.ERR_NONFINITE) == "PASD_ERR_NONFINITE"
    p = P.pasd_params_default((50, 40, 30), (5, 4, 3))
    assert p.order == 3 and p.mu0 == 1e-4 and p.mu_max == 1e10 and p.rho == 1.1
    assert p.tol == 1e-5 and p.max_iter == 1000
    with pytest.raises(P.PasdError):
        P.pasd_params_default((50,), (5,))      # order < 2


def test_no_gpu_fails_loudly(P):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.PasdError):
        P.pasd_ctx_create(0)
