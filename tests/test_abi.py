"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every function include/hs.h declares, and its host-side validation and
helpers behave (no compute call needs a GPU here)."""
import ctypes
import os

import numpy as np
import pytest

from paper_1805_12258_gb300 import build as hsbuild
from paper_1805_12258_gb300 import hs


@pytest.fixture(scope="module")
def L():
    hsbuild.build()
    return hs.lib()


def test_header_declares_the_boundary():
    names = hs.header_functions()
    for n in ("hs_plan_create", "hs_run", "hs_run_checked", "hs_cand_sync", "hs_run_host",
              "hs_plan_destroy", "hs_status_str", "hs_last_error", "hs_pack_paper"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in hs.header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_record_layout():
    assert ctypes.sizeof(hs.hs_cand) == 16
    assert hs.CAND_DTYPE.itemsize == 16
    assert ctypes.sizeof(hs.hs_options) == 44


def test_status_strings(L):
    assert hs.hs_status_str(hs.HS_OK) == "ok"
    assert "overflow" in hs.hs_status_str(hs.HS_ERR_OVERFLOW)
    assert hs.hs_status_str(99) == "unknown status"


@pytest.mark.parametrize("nt,n,H,why", [
    (0, 100, 8, "odd"), (20, 100, 8, "odd"), (21, 0, 8, "n_bins"), (21, 100, 0, "H"),
    (21, 100, 33, "H"), (32769, 100, 8, "odd"), (21, 1 << 31, 8, "n_bins")])
def test_plan_create_rejects_bad_shapes(L, nt, n, H, why):
    ta = np.ones(max(H, 1) * max(nt, 1), np.float32)
    out = ctypes.c_void_p()
    st = L.hs_plan_create(ctypes.byref(out), nt, n, H, ta.ctypes.data, None)
    assert st == hs.HS_ERR_INVALID
    assert why in L.hs_last_error().decode()
    assert out.value is None


def test_plan_create_rejects_nonfinite_thresholds(L):
    ta = np.ones((8, 21), np.float32)
    ta[3, 4] = np.nan
    out = ctypes.c_void_p()
    assert L.hs_plan_create(ctypes.byref(out), 21, 100, 8, ta.ctypes.data, None) == \
        hs.HS_ERR_INVALID
    assert L.hs_plan_create(ctypes.byref(out), 21, 100, 8, None, None) == hs.HS_ERR_INVALID


def test_plan_create_rejects_bad_options(L):
    ta = np.ones((8, 21), np.float32)
    out = ctypes.c_void_p()
    opt = hs.hs_options(7, 0, 0, 0, 0, 0)
    assert L.hs_plan_create(ctypes.byref(out), 21, 100, 8, ta.ctypes.data,
                            ctypes.byref(opt)) == hs.HS_ERR_INVALID


@pytest.mark.parametrize("H,opts,why", [
    (13, dict(index=1, kernel=2), "harmonic-fraction"),              # H not compiled
    (16, dict(index=1, kernel=2, tile_bins=96), "harmonic-fraction"),  # tile width
    (16, dict(index=1, kernel=2, zround=1), "harmonic-fraction"),      # floor rounding
    (16, dict(index=1, kernel=2, row_pitch=1001), "harmonic-fraction"),  # rows not 16 B
    (16, dict(index=1, stages=3), "pipelined")])
def test_plan_create_refuses_missing_harmonic_fraction_kernels(L, H, opts, why):
    # the kernel choice is made before any device allocation: a staged
    # harmonic-fraction kernel is asked for where none is compiled
    ta = np.ones((H, 85), np.float32)
    opt = hs.hs_options(**opts)
    out = ctypes.c_void_p()
    st = L.hs_plan_create(ctypes.byref(out), 85, 1000, H, ta.ctypes.data, ctypes.byref(opt))
    assert st == hs.HS_ERR_UNSUPPORTED
    assert why in L.hs_last_error().decode()
    assert out.value is None


def test_run_rejects_null_plan_and_pointers(L):
    buf = hs.hs_cand_buf(None, None, 0)
    assert L.hs_run(None, None, None, ctypes.byref(buf)) == hs.HS_ERR_INVALID
    assert L.hs_cand_sync(None, None, None) == hs.HS_ERR_INVALID
    assert L.hs_plan_destroy(None) == hs.HS_OK


def test_pack_paper(L):
    # Section III: CL1 = F*2^24 + H*2^21 + B with F the row, H the 0-based
    # plane, B the bin; CL2 = amplitude.
    rec = np.zeros(1, hs.CAND_DTYPE)[0]
    rec["bin"], rec["z"], rec["k"], rec["power"] = 123456, -40, 8, 42.5
    cl1, cl2 = hs.hs_pack_paper(rec, 85)
    assert cl1 == (2 << 24) + (7 << 21) + 123456
    assert cl2 == 42.5
    rec["k"] = 9
    with pytest.raises(hs.HsError):
        hs.hs_pack_paper(rec, 85)
    rec["k"], rec["bin"] = 1, 1 << 21
    with pytest.raises(hs.HsError):
        hs.hs_pack_paper(rec, 85)


def test_c_struct_layouts_match_the_binding(tmp_path):
    """The header's structs as a C compiler lays them out equal the ctypes
    mirrors the binding passes across the boundary."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = ["hs_options", "hs_cand", "hs_cand_buf", "hs_beam", "hs_server_config",
             "hs_request", "hs_result", "hs_server_stats"]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include "hs.h"\nint main(void){\n' +
                   "".join(f'printf("%zu\\n", sizeof({n}));\n' for n in names) +
                   "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(hs.HEADER), str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                            text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(getattr(hs, n)) for n in names]


def test_server_and_generator_validate_before_touching_the_device(L):
    out = ctypes.c_void_p()
    assert L.hs_server_create(ctypes.byref(out), None) == hs.HS_ERR_INVALID
    cfg = hs.hs_server_config(85, 16, None, 4, 1000, 16, 0, 0)
    assert L.hs_server_create(ctypes.byref(out), ctypes.byref(cfg)) == hs.HS_ERR_INVALID
    assert L.hs_synth_fop(None, None, 0, 85, 100, 104, 1, 0, None) == hs.HS_ERR_INVALID
    assert L.hs_server_submit(None, None, None) == hs.HS_ERR_INVALID
    assert L.hs_server_destroy(None) == hs.HS_OK
    assert "busy" in hs.hs_status_str(hs.HS_ERR_BUSY)
    assert "bounds" in hs.hs_status_str(hs.HS_ERR_BOUNDS)
