"""Host-side checks of libdvm that need no GPU: the C ABI loads and exports every declared symbol,
argument validation, and the library's own velocity quadratures (Golub-Welsch Gauss-Hermite,
trapezoid Newton-Cotes, the cubic grid of Eq. nonuniform_v) against numpy and the oracle."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1704_03126_gb300 import build as dvm_build
from paper_1704_03126_gb300 import dvm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    dvm_build.build()
    return dvm.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dvm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dvm_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "dvm_create" in names and "dvm_solve" in names and "dvm_batch_solve" in names
    L = dvm.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("n", [2, 8, 12, 16, 32, 48, 64])
def test_library_gauss_hermite_matches_numpy(n):
    x, w = dvm.velocity_grid("gh", n)
    xr, wr = np.polynomial.hermite.hermgauss(n)
    assert np.max(np.abs(x - xr)) < 1e-12 * max(1.0, np.abs(xr).max())
    # Golub-Welsch weights come from eigenvector components: absolute accuracy ~1e-15
    assert np.max(np.abs(w - wr / math.sqrt(math.pi))) < 5e-15
    assert np.all(x == -x[::-1])


@pytest.mark.parametrize("kind,n,vmax", [("nc", 32, 5.0), ("nc", 8, 4.0), ("cubic", 48, 4.0), ("cubic", 16, 4.0),
                                         ("gh", 24, 0.0)])
def test_library_grids_match_oracle(kind, n, vmax):
    x, w = dvm.velocity_grid(kind, n, vmax)
    xo, wo = oracle.quadrature(kind, n, vmax)
    assert np.max(np.abs(x - xo)) < 5e-14
    assert np.max(np.abs(w - wo)) < 5e-15
    assert np.all(x == -x[::-1])


def test_library_rejects_invalid_grids():
    for kind, n in [("gh", 7), ("nc", 1), ("cubic", 66)]:
        with pytest.raises(dvm.DvmError) as ei:
            dvm.velocity_grid(kind, n)
        assert ei.value.status == dvm.DVM_EINVAL


@pytest.mark.parametrize("kwargs", [
    dict(mask=np.zeros((8, 1), np.uint8), kn=1.0),                     # nx < 2
    dict(mask=np.ones((8, 8), np.uint8), kn=1.0),                      # no gas cell
    dict(mask=np.zeros((8, 8), np.uint8), kn=-1.0),                    # neither kn nor delta
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, quad=("gh", 7)),     # odd velocity grid
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, ly=0.0),             # bad height
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, accommodation=1.5),  # accommodation outside [0, 1]
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, accommodation=-0.1),
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, periodic_y=True, top_wall_u1=1.0),  # moving plate, periodic x2
    dict(mask=np.zeros((4, 8), np.uint8), kn=1.0, row_heights=np.full(4, 0.25)),      # row heights without dx1
    dict(mask=np.zeros((4, 8), np.uint8), kn=1.0, dx1=0.1, row_heights=np.array([0.3, 0.3, 0.0, 0.4])),
    dict(mask=np.zeros((4, 8), np.uint8), kn=1.0, dx1=0.1, row_heights=np.full(4, 0.25), storage="as_given"),
    dict(mask=np.zeros((4, 8), np.uint8), kn=1.0, dx1=-0.1),                           # negative x1 spacing
    dict(mask=np.zeros((8, 4096), np.uint8)[:, :2].repeat(2049, axis=1).repeat(512, axis=0), kn=1.0),  # > 16.8 M cells
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, anderson=9),                         # mixing depth above 8
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, anderson=-1),
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, anderson=3, accommodation=0.5),     # mixing with specular walls
    dict(mask=np.zeros((8, 8), np.uint8), kn=1.0, anderson=3, precision="fp32"),      # mixing with FP32 storage
])
def test_create_rejects_invalid_parameters(kwargs):
    with pytest.raises(dvm.DvmError) as ei:
        dvm.Solver(**kwargs)
    assert ei.value.status == dvm.DVM_EINVAL


def test_both_kn_and_delta_rejected_by_the_library():
    L = dvm.lib()
    p = dvm.Params()
    L.dvm_params_init(p)
    p.nx, p.ny, p.kn, p.delta = 4, 4, 1.0, 1.0
    mask = np.zeros((4, 4), np.uint8)
    import ctypes
    ctx = ctypes.c_void_p()
    st = L.dvm_create(mask.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p), None, ctypes.byref(ctx))
    assert st == dvm.DVM_EINVAL
    assert b"exactly one" in L.dvm_last_error(None)


def test_storage_order_is_validated_by_the_library():
    import ctypes
    L = dvm.lib()
    p = dvm.Params()
    L.dvm_params_init(p)
    assert p.storage == dvm.STORAGE["auto"]
    p.nx, p.ny, p.storage = 4, 4, 3
    mask = np.zeros((4, 4), np.uint8)
    ctx = ctypes.c_void_p()
    st = L.dvm_create(mask.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p), None, ctypes.byref(ctx))
    assert st == dvm.DVM_EINVAL
    assert b"storage" in L.dvm_last_error(None)


def test_status_strings():
    L = dvm.lib()
    assert L.dvm_status_string(0) == b"DVM_OK"
    assert L.dvm_status_string(4) == b"DVM_ENOCONV"


def test_selftest_wait_rejects_an_unknown_primitive():
    st, sec = dvm.selftest_wait(7, 10)
    assert st == dvm.DVM_EINVAL


def test_every_entry_point_rejects_null_handles():
    """No call dereferences a NULL context, batch or output pointer: each returns DVM_EINVAL (checked
    before any CUDA call, so this runs without a GPU)."""
    import ctypes
    L = dvm.lib()
    P = None
    d = ctypes.c_double()
    i = ctypes.c_int()
    f = ctypes.c_float()
    calls = {
        "dvm_reset": (P,),
        "dvm_set_delta_field": (P, P),
        "dvm_solve": (P, 1e-6, 10, ctypes.byref(i), ctypes.byref(d)),
        "dvm_iterate": (P, 1),
        "dvm_flowrate": (P, ctypes.byref(d), ctypes.byref(d)),
        "dvm_fields": (P, P, P, P, P),
        "dvm_get_info": (P, P),
        "dvm_distribution": (P, P, 0, P),
        "dvm_quadrature": (P, P, P),
        "dvm_adjoint": (P, 1e-6, 10, P, P, P),
        "dvm_set_schedule": (P, 0, 0),
        "dvm_get_schedule": (P, ctypes.byref(i), ctypes.byref(i)),
        "dvm_batch_create": (P, 0, P),
        "dvm_batch_run": (P, 1e-6, 10, P),
        "dvm_batch_iterate": (P, 1),
        "dvm_batch_enqueue": (P, 1),
        "dvm_batch_check": (P,),
        "dvm_batch_timing": (P, ctypes.byref(f), ctypes.byref(f)),
        "dvm_batch_set_schedule": (P, 0, 0),
        "dvm_batch_get_schedule": (P, ctypes.byref(i), ctypes.byref(i)),
        "dvm_batch_autotune": (P, 1, ctypes.byref(i), ctypes.byref(i), ctypes.byref(f)),
        "dvm_velocity_grid": (P, P, P),
        "dvm_params_init": (P,),
    }
    for name, args in calls.items():
        st = getattr(L, name)(*args)
        assert st == dvm.DVM_EINVAL, (name, st)
    # destroy functions accept NULL silently
    L.dvm_destroy(None)
    L.dvm_batch_destroy(None)


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures of the binding have the size and field offsets of dvm_params, dvm_info
    and dvm_quad as a C compiler lays them out from include/dvm.h."""
    import ctypes
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = {"dvm_params": dvm.Params, "dvm_info": dvm.Info, "dvm_quad": dvm.Quad}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dvm.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", include, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert c_layout[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert c_layout[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
