"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/fdcgks.h declares, the ctypes parameter struct matches the C
layout, and argument validation fails cleanly before any device call."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2606_17772_gb300 import build as fbuild
from paper_2606_17772_gb300 import fdcgks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fdcgks.h")


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return fdcgks.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdcgks_[a-z_]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fdcgks.EXPORTS) == names


def test_params_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "fdcgks.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(fdcgks_params), offsetof(fdcgks_params, bc),
         offsetof(fdcgks_params, flux_variant), offsetof(fdcgks_params, precision),
         offsetof(fdcgks_params, tau_c1), offsetof(fdcgks_params, tau_c2), offsetof(fdcgks_params, stream));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    P = fdcgks.Params
    assert vals == [ctypes.sizeof(P), P.bc.offset, P.flux_variant.offset, P.precision.offset, P.tau_c1.offset,
                    P.tau_c2.offset, P.stream.offset]


def test_side_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "fdcgks.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %d\n", sizeof(fdcgks_side), offsetof(fdcgks_side, kind),
         offsetof(fdcgks_side, split0), offsetof(fdcgks_side, split_speed), offsetof(fdcgks_side, prim),
         (int)FDCGKS_BC_FIXED);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    S = fdcgks.Side
    assert vals == [ctypes.sizeof(S), S.kind.offset, S.split0.offset, S.split_speed.offset, S.prim.offset,
                    fdcgks.BC_FIXED]


def test_line_params_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "fdcgks.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(fdcgks_line_params), offsetof(fdcgks_line_params, bc),
         offsetof(fdcgks_line_params, flux_variant), offsetof(fdcgks_line_params, tau_c1),
         offsetof(fdcgks_line_params, recon_vars), offsetof(fdcgks_line_params, stream),
         offsetof(fdcgks_line_params, cluster), offsetof(fdcgks_line_params, precision));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    P = fdcgks.LineParams
    assert vals == [ctypes.sizeof(P), P.bc.offset, P.flux_variant.offset, P.tau_c1.offset, P.recon_vars.offset,
                    P.stream.offset, P.cluster.offset, P.precision.offset]


@pytest.mark.parametrize("bad", [dict(n=2), dict(n=0), dict(batch=0), dict(bc=(0, 1)), dict(bc=(3, 3)),
                                 dict(flux_variant=63), dict(gamma=1.0), dict(recon_vars=2), dict(cluster=3),
                                 dict(cluster=16), dict(precision=2)])
def test_invalid_line_parameters_are_rejected_before_device_work(lib, bad):
    kw = dict(n=20, batch=1, bc=(1, 1))
    kw.update(bad)
    p = fdcgks.line_params(**kw)
    h = ctypes.c_void_p()
    assert lib.fdcgks_line_create(ctypes.byref(p), ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.fdcgks_line_last_error(None).decode()


def test_case_sides_marshalling():
    from paper_2606_17772_gb300 import inputs
    case = inputs.double_mach(16, 4)
    p = fdcgks.params_for_case(case)
    assert list(p.bc) == list(case.bc)
    arr = fdcgks.make_sides(case.sides)
    assert list(arr[3].kind) == [fdcgks.BC_FIXED, fdcgks.BC_FIXED]
    assert arr[3].split0 == case.sides[3]["split0"] and arr[3].split_speed == case.sides[3]["split_speed"]
    assert list(arr[3].prim[1]) == list(inputs.DMR_PRE) and list(arr[0].prim[0]) == list(inputs.DMR_POST)
    assert list(arr[2].kind) == [fdcgks.BC_TRANSMISSIVE, fdcgks.BC_SYMMETRY] and arr[2].split0 == 1.0 / 6.0
    with pytest.raises(ValueError):
        fdcgks.Ensemble.from_cases([case])


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-3), dict(gamma=1.0), dict(Pr=0.0), dict(mu=-1.0),
                                 dict(bc=(0, 1, 0, 0)), dict(flux_variant=63), dict(geno_variant=5),
                                 dict(precision=7), dict(grad_base=2), dict(x1=-1.0), dict(bc=(9, 9, 0, 0))])
def test_invalid_parameters_are_rejected_before_device_work(lib, bad):
    kw = dict(nx=8, ny=8)
    kw.update(bad)
    p = fdcgks.make_params(**kw)
    h = ctypes.c_void_p()
    st = lib.fdcgks_create(ctypes.byref(p), ctypes.byref(h))
    assert st == 1
    assert h.value is None
    assert lib.fdcgks_last_error(None).decode()


def test_batch_argument_validation(lib):
    p = fdcgks.make_params(8, 8)
    assert lib.fdcgks_iface_batch(ctypes.byref(p), 2, ctypes.c_double(0.1), 4, None, None) == 1
    assert lib.fdcgks_nodal_batch(ctypes.byref(p), ctypes.c_double(-1.0), 4, None, None) == 1
    assert lib.fdcgks_recon_batch(ctypes.byref(p), 3, ctypes.c_double(0.1), 4, None, None) == 1
    assert lib.fdcgks_recon_batch(ctypes.byref(p), 0, ctypes.c_double(0.1), 0, None, None) == 0   # empty batch


def test_null_context_calls(lib):
    assert lib.fdcgks_step(None, ctypes.c_double(0.1)) == 1
    assert lib.fdcgks_dims(None, None, None, None, None) == 1
    assert lib.fdcgks_set_sides(None, None) == 1
    assert lib.fdcgks_set_time(None, ctypes.c_double(0.0)) == 1
    assert lib.fdcgks_get_time(None, None) == 1
    assert lib.fdcgks_line_steps(None, ctypes.c_double(0.1), 1) == 1
    assert lib.fdcgks_line_check(None, None, None) == 1
    lib.fdcgks_line_destroy(None)
    lib.fdcgks_destroy(None)
    assert lib.fdcgks_status_string(3).decode() == "non-physical state"
