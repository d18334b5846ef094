"""Host-only checks of the C ABI: the library loads without a GPU, exports
every function include/cog.h declares, and validates parameters."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cog():
    from paper_1705_09339_gb300.build import build
    build()
    from paper_1705_09339_gb300 import cog
    return cog


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cog_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(cog):
    names = _declared("cog.h")
    assert "cog_apply" in names and "cog_train_prior" in names and len(names) >= 15
    for n in names:
        assert hasattr(cog.lib, n), n


def test_struct_sizes_match_header(cog):
    import ctypes as C
    assert C.sizeof(cog.cog_params) == 4 * 24
    assert C.sizeof(cog.cog_stats) == 8 * 7 + 8
    assert C.sizeof(cog.cog_layout) == 8 * 12
    # 2 int32, 3 + 3 + 6 + 6 int64, 6 + 6 + 3 + 9 + 3 double
    assert C.sizeof(cog.cog_group_stats) == 8 + 8 * 18 + 8 * 27


def test_default_params_and_layout(cog):
    p = cog.cog_default_params(1920, 1080, 5, state_dtype="f16")
    assert (p.alpha, p.lambda_, p.T_bg) == (pytest.approx(0.01), 2.5, pytest.approx(0.7))
    assert p.flags == cog.COG_ALL and p.kde_bw == 4
    L = cog.cog_state_layout(p)
    P = 1920 * 1080
    Pp = (P + 4095) // 4096 * 4096
    assert L.rec_bytes == 80 and L.elem_bytes == 2
    assert L.kde_row == 256 and L.kde + P * 768 <= L.total
    for off in (L.jl, L.conf, L.s1, L.gmm, L.queue, L.kde):
        assert off % 256 == 0
    assert L.s1_bytes == 16 and L.gmm - L.s1 >= Pp * 16 and L.kde - L.queue >= Pp * 16
    # every first-kernel CTA (1024 pixels) may enqueue all its pixels into
    # segment cta % 32: each segment holds ceil(ctas / 32) whole tiles
    for (w, h) in [(1, 1), (64, 64), (1920, 1080), (4096, 1), (33 * 1024, 1)]:
        pp = cog.cog_default_params(w, h, 3)
        Lq = cog.cog_state_layout(pp)
        ctas = (w * h + 1023) // 1024
        cap = (ctas + 31) // 32 * 1024
        assert Lq.kde - Lq.queue >= 32 * cap * 16
    assert cog.cog_state_bytes(p) == L.total
    p32 = cog.cog_default_params(160, 120, 3)
    assert cog.cog_state_layout(p32).rec_bytes == 96 and cog.cog_state_layout(p32).s1_bytes == 32
    # per-channel mixtures: K x 9 values per record (K=5 FP16: 90 -> 96 bytes)
    pc = cog.cog_default_params(1920, 1080, 5, state_dtype="f16")
    pc.flags |= cog.COG_PERCHAN
    assert cog.cog_state_layout(pc).rec_bytes == 96
    # the 4-bit prior: 128-byte rows, half the 8-bit prior's 768 bytes per pixel
    p4 = cog.cog_default_params(1920, 1080, 5, state_dtype="f16", kde_bits=4)
    L4 = cog.cog_state_layout(p4)
    assert L4.kde_row == 128 and L4.kde == L.kde and L4.kde + P * 384 <= L4.total
    assert L.total - L4.total >= P * 384 - 256


@pytest.mark.parametrize("field,value", [("K", 0), ("K", 9), ("width", 0), ("alpha", 0.0), ("alpha", 1.5),
                                         ("var_min", 0.0), ("kde_bw", 0), ("kde_bw", 33), ("r2", -1),
                                         ("illum_permille", 1001), ("flags", 128), ("flags", 15 | 32 | 64),
                                         ("state_dtype", 3), ("skip_period", 0),
                                         ("w_illum", 1.0), ("T_bg", 1.5), ("kde_bits", 0), ("kde_bits", 6)])
def test_invalid_params_rejected(cog, field, value):
    p = cog.cog_default_params(64, 48, 3)
    setattr(p, field, value)
    with pytest.raises(cog.CogError) as e:
        cog.cog_state_bytes(p)
    assert e.value.status == cog.COG_ERR_INVALID_ARG
    assert cog.cog_last_error_string(None)


def test_null_context_calls_fail_cleanly(cog):
    assert cog.lib.cog_sync(None) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_destroy(None) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_apply(None, None, None, None, None) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_apply_clip(None, None, 4, None, None, None) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_clip_runs(None, None) == cog.COG_ERR_INVALID_ARG
    import ctypes as C
    w, ms = C.c_uint32(0), C.c_double(0.0)
    for bad in (0, 2001):
        assert cog.lib.cog_selftest_bounded_wait(bad, C.byref(w), C.byref(ms)) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_selftest_bounded_wait(10, None, None) == cog.COG_ERR_INVALID_ARG


def test_server_add_rejects_bad_arguments(cog):
    import ctypes as C
    idx = C.c_int32(0)
    assert cog.lib.cog_server_add(None, None, C.byref(idx)) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_server_remove(None, 0, None) == cog.COG_ERR_INVALID_ARG
    ptr = C.c_void_p()
    assert cog.lib.cog_host_alloc(0, C.byref(ptr)) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_host_alloc(16, None) == cog.COG_ERR_INVALID_ARG
    assert cog.lib.cog_host_free(None) == cog.COG_ERR_INVALID_ARG   # not a block of cog_host_alloc


def test_group_rejects_bad_arguments(cog):
    import ctypes as C
    st = cog.cog_group_stats()
    assert cog.lib.cog_group(None, None, 10, None, None, C.byref(st)) == cog.COG_ERR_INVALID_ARG


def test_probe_stream_rejects_bad_arguments(cog):
    """The streaming probe validates its arguments before any launch."""
    import numpy as np
    bufs = [np.zeros(64, dtype=np.uint8) for _ in range(6)]
    good = [b.ctypes.data + (-b.ctypes.data) % 16 for b in bufs]   # 16-byte aligned addresses
    # (no valid call is made here: every case below fails validation)
    for P in (0, -4, 6):
        assert cog.lib.cog_probe_stream(*good, P, None) == cog.COG_ERR_INVALID_ARG
    for i in range(6):
        args = list(good)
        args[i] = None
        assert cog.lib.cog_probe_stream(*args, 8, None) == cog.COG_ERR_INVALID_ARG
        args[i] = good[i] + 4
        assert cog.lib.cog_probe_stream(*args, 8, None) == cog.COG_ERR_INVALID_ARG


def test_header_compiles_as_c99_and_cpp11(tmp_path):
    """The C ABI header stands alone for C and C++ callers."""
    import shutil
    import subprocess
    inc = os.path.join(ROOT, "include")
    for cc, std, ext in (("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")):
        if not shutil.which(cc):
            pytest.skip(f"{cc} not found")
        src = tmp_path / f"h.{ext}"
        src.write_text('#include "cog.h"\nint main(void) { cog_group_stats s; (void)s; return 0; }\n')
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-I", inc, "-c", str(src), "-o",
                            str(tmp_path / f"h_{ext}.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_ctypes_structs_match_the_header(cog, tmp_path):
    """Every struct the binding mirrors has the size and field offsets the
    C compiler gives the header's declaration."""
    import ctypes as C
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    structs = {"cog_params": cog.cog_params, "cog_layout": cog.cog_layout, "cog_stats": cog.cog_stats,
               "cog_group_stats": cog.cog_group_stats, "cog_server_stats": cog.cog_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cog.h"', 'int main(void) {']
    for name, ct in structs.items():
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in ct._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'    printf("{name}.{f} %zu\\n", offsetof({name}, {cf}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "sz.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "sz"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for name, ct in structs.items():
        assert int(got[name]) == C.sizeof(ct), name
        for f, _ in ct._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(ct, f).offset, (name, f)
