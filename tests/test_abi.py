"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every function include/ctm.h declares, and its ctypes structures
match the header's layout.  No compute calls here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("ctm.h", "ctm_server.h")]


@pytest.fixture(scope="module")
def built():
    from paper_2604_07980_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    return build.build()


def _declared():
    txt = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ctm_\w+)\s*\(", txt, re.M)))


def test_header_declares_binding_exports():
    from paper_2604_07980_gb300 import binding as B
    assert sorted(B.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts():
    from paper_2604_07980_gb300 import binding as B
    assert ctypes.sizeof(B.ctm_params) == 21 * 4
    assert ctypes.sizeof(B.ctm_frame) == 48
    assert B.BLOCK_DTYPE.itemsize == B.BLOCK_BYTES == 48
    assert ctypes.sizeof(B.ctm_debug) == 24
    assert ctypes.sizeof(B.ctm_tuning) == 24
    assert ctypes.sizeof(B.ctm_geometry) == 136
    assert ctypes.sizeof(B.ctm_server_config) == 40
    assert ctypes.sizeof(B.ctm_request) == 80
    assert ctypes.sizeof(B.ctm_completion) == 56
    assert ctypes.sizeof(B.ctm_server_stats) == 72


def test_status_strings_and_defaults(built):
    from paper_2604_07980_gb300 import binding as B
    L = B.lib()
    assert L.ctm_status_str(0) == b"ok"
    assert b"invalid" in L.ctm_status_str(-1)
    p = B.make_params()
    assert (p.win_w, p.win_h, p.sentinel, p.far_side_px, p.close_factor) == (9, 7, 1, 40, 2)
    # argument checks that need no device
    assert L.ctm_default_params(None) == B.CTM_EINVAL
    assert L.ctm_census_build(None, 10, 10, 10, 1, 9, 7, 1, None, 10, None) == B.CTM_EINVAL
    h = ctypes.c_void_p()
    bad = B.make_params({"win_w": 8})
    assert L.ctm_create(ctypes.byref(h), ctypes.byref(bad), 1, 64, 64, 4) == B.CTM_EINVAL
    assert L.ctm_match_batch(None, None, None, None, None, None, None, None, 0, None) == B.CTM_EINVAL
    assert b"bounded device wait" in L.ctm_status_str(B.CTM_ETIMEOUT)
    assert L.ctm_probe_bounded_wait(None, None) == B.CTM_EINVAL


def test_create_and_noalloc_share_parameter_checks(built):
    """Parameters whose strip exceeds the matcher's shared-memory budget (12 disparities
    x 21 vertical offsets) are rejected with CTM_EINVAL by ctm_create and by
    ctm_match_boxes_noalloc alike, before either touches a device; so are other
    out-of-range fields."""
    torch = pytest.importorskip("torch")
    from paper_2604_07980_gb300 import binding as B
    L = B.lib()
    bad_sets = [{"far_dmax": 11, "close_dmax": 11, "dy_min": -10, "dy_max": 10},
                {"win_w": 8}, {"grid_g": 9}, {"trim_frac": 0.5}, {"max_occluders": 33}]
    for bad in bad_sets:
        p = B.make_params(bad)
        h = ctypes.c_void_p()
        assert L.ctm_create(ctypes.byref(h), ctypes.byref(p), 1, 64, 64, 4) == B.CTM_EINVAL, bad
        if torch.cuda.is_available():
            continue  # the no-GPU form below passes placeholder pointers
        fake = ctypes.c_void_p(256)
        st = L.ctm_match_boxes_noalloc(ctypes.byref(p), fake, fake, 64, 64, 64, fake, 1, 1.0, 1.0,
                                       fake, fake, fake, None)
        assert st == B.CTM_EINVAL, bad
    ok = B.make_params({"far_dmax": 11, "close_dmax": 11, "dy_min": -4, "dy_max": 4})
    h = ctypes.c_void_p()
    assert L.ctm_create(ctypes.byref(h), ctypes.byref(ok), 1, 64, 64, 4) != B.CTM_EINVAL
    if h.value:
        L.ctm_destroy(h)


def test_binding_refuses_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2604_07980_gb300 import binding as B
    with pytest.raises(B.CtmError):
        B.Context({}, 1, 64, 64, 4)


def test_server_argument_checks(built):
    """Server entry points reject bad arguments before touching a device."""
    from paper_2604_07980_gb300 import binding as B
    L = B.lib()
    cfg = B.ctm_server_config()
    assert L.ctm_server_default_config(ctypes.byref(cfg)) == B.CTM_OK
    assert (cfg.lanes, cfg.frames_per_batch, cfg.max_width, cfg.max_height) == (4, 8, 3840, 2160)
    assert L.ctm_server_default_config(None) == B.CTM_EINVAL
    p = B.make_params()
    h = ctypes.c_void_p()
    assert L.ctm_server_create(None, ctypes.byref(p), ctypes.byref(cfg)) == B.CTM_EINVAL
    for field, bad in (("lanes", 0), ("lanes", 9), ("frames_per_batch", 0), ("max_queue", 0),
                       ("image_budget_bytes", 0), ("plain", 2)):
        c = B.ctm_server_config.from_buffer_copy(cfg)
        setattr(c, field, bad)
        assert L.ctm_server_create(ctypes.byref(h), ctypes.byref(p), ctypes.byref(c)) == B.CTM_EINVAL
        assert not h.value
    req = B.ctm_request()
    assert L.ctm_server_submit(None, ctypes.byref(req)) == B.CTM_EINVAL
    n = ctypes.c_int32(7)
    assert L.ctm_server_poll(None, None, 0, 0, ctypes.byref(n)) == B.CTM_EINVAL
    assert L.ctm_server_destroy(None) == B.CTM_EINVAL
    assert L.ctm_server_now_ns() > 0


def test_tuning_argument_checks(built):
    from paper_2604_07980_gb300 import binding as B
    L = B.lib()
    t = B.ctm_tuning(128, 192, 0, 4096, 0)
    assert L.ctm_get_tuning(None, ctypes.byref(t)) == B.CTM_EINVAL
    assert L.ctm_set_tuning(None, ctypes.byref(t)) == B.CTM_EINVAL
    assert L.ctm_autotune(None, None, None, None, None, None, None, 3, None, None, None) == B.CTM_EINVAL


def test_box_points_argument_checks(built):
    from paper_2604_07980_gb300 import binding as B
    L = B.lib()
    assert L.ctm_box_points(None, None, None, 0, None, 0, None, None) == B.CTM_OK  # nothing to do
    assert L.ctm_box_points(None, None, None, 4, None, 1, None, None) == B.CTM_EINVAL
    assert L.ctm_box_points(None, None, None, -1, None, 0, None, None) == B.CTM_EINVAL


def test_struct_fields_match_the_c_headers():
    """Every field of every ctypes mirror (and of the numpy block and frame records)
    sits at the offset and has the size a C compiler gives the header's struct:
    a C program built from include/*.h prints offsetof/sizeof for each field."""
    import shutil
    import subprocess
    import numpy as np
    from paper_2604_07980_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    mirrors = {name: getattr(B, name) for name in
               ("ctm_params", "ctm_frame", "ctm_debug", "ctm_stats", "ctm_geometry", "ctm_tuning",
                "ctm_server_config", "ctm_request", "ctm_completion", "ctm_server_stats")}
    records = {"ctm_block": B.BLOCK_DTYPE, "ctm_frame": B.FRAME_DTYPE}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ctm_server.h"', "int main(void) {"]
    expect = {}
    for sname, cls in mirrors.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        expect[sname] = ctypes.sizeof(cls)
        for fname, _ in cls._fields_:
            key = f"{sname}.{fname}"
            lines.append(f'printf("{key} %zu %zu\\n", offsetof({sname}, {fname}), '
                         f'sizeof((({sname} *)0)->{fname}));')
            d = getattr(cls, fname)
            expect[key] = (d.offset, d.size)
    rec_expect = {}
    for sname, dt in records.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        rec_expect[sname] = dt.itemsize
        for fname in dt.names:
            key = f"{sname}.{fname}"
            lines.append(f'printf("{key} %zu %zu\\n", offsetof({sname}, {fname}), '
                         f'sizeof((({sname} *)0)->{fname}));')
            rec_expect[key] = (dt.fields[fname][1], dt.fields[fname][0].itemsize)
    lines += ["return 0;", "}"]
    out_dir = os.path.join(ROOT, "paper_2604_07980_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "abi_layout.c")
    exe = os.path.join(out_dir, "abi_layout")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
    got = {}
    for line in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines():
        parts = line.split()
        got[parts[0]] = int(parts[1]) if len(parts) == 2 else (int(parts[1]), int(parts[2]))
    for key, want in expect.items():
        assert got[key] == want, (key, got[key], want)
    for key, want in rec_expect.items():
        assert got[key] == want, (key, got[key], want)
    assert np.dtype(B.BLOCK_DTYPE).itemsize == B.BLOCK_BYTES
