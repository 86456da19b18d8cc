"""The C-ABI library builds, loads, and exports every function include/rbfd.h
declares; the ctypes mirrors of its structs match the C layout.  No GPU
needed: nothing here launches a kernel."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2107_13887_gb300 import build as B
from paper_2107_13887_gb300 import rbfd

HEADER = os.path.join(B.ROOT, "include", "rbfd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(rbfd_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["rbfd_create", "rbfd_greedy", "rbfd_get_level", "rbfd_deform", "rbfd_deform_f64",
                 "rbfd_destroy", "rbfd_last_error", "rbfd_options_default"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in rbfd.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_exports_are_plain_c(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    for n in declared_functions():
        assert n in exported  # unmangled


def test_version_and_defaults_without_gpu(lib):
    L = rbfd.load()
    assert L.rbfd_version().startswith(b"rbfd")
    o = rbfd.default_options()
    assert o.precision == rbfd.MIXED and o.basis == 2 and o.refine_iters == 3


def test_struct_layout_matches_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rbfd.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu\\n", sizeof(rbfd_options), offsetof(rbfd_options, nc_cap),'
        " offsetof(rbfd_options, stream), offsetof(rbfd_options, grid_ctas));\n"
        'printf("%zu %zu %zu %zu\\n", sizeof(rbfd_stats), offsetof(rbfd_stats, confirm_resumes),'
        " offsetof(rbfd_stats, persist_phase_ms), offsetof(rbfd_stats, wall_pairs_exact));\n"
        'printf("%zu %zu\\n", sizeof(rbfd_quality), offsetof(rbfd_quality, hist));\n'
        'printf("%zu %zu %zu\\n", sizeof(rbfd_job), offsetof(rbfd_job, opt), offsetof(rbfd_job, out));\n'
        'printf("%zu %zu %zu\\n", sizeof(rbfd_worklist_tune), offsetof(rbfd_worklist_tune, launch_ms),'
        " offsetof(rbfd_worklist_tune, items));\n"
        'printf("%zu %zu %zu\\n", sizeof(rbfd_server_options), offsetof(rbfd_server_options, max_queue),'
        " offsetof(rbfd_server_options, fuse_volume));\n"
        'printf("%zu %zu\\n", offsetof(rbfd_stats, newton_pairs_useful), offsetof(rbfd_stats, eq12_pairs));\n'
        'printf("%zu %zu %zu\\n", offsetof(rbfd_options, prune), offsetof(rbfd_stats, persist_grow_fma),'
        " offsetof(rbfd_stats, sweep_warps_skipped));\n"
        "return 0;}\n"
    )
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    a, b, c, d, e, f, g, h = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:8]
    so, onc, ost, ori = map(int, a.split())
    ss, ocr, ovp, owp = map(int, b.split())
    assert so == ctypes.sizeof(rbfd.rbfd_options)
    assert onc == rbfd.rbfd_options.nc_cap.offset
    assert ost == rbfd.rbfd_options.stream.offset
    assert ori == rbfd.rbfd_options.grid_ctas.offset
    assert ss == ctypes.sizeof(rbfd.rbfd_stats)
    assert ocr == rbfd.rbfd_stats.confirm_resumes.offset
    assert ovp == rbfd.rbfd_stats.persist_phase_ms.offset
    assert owp == rbfd.rbfd_stats.wall_pairs_exact.offset
    sq, oh = map(int, c.split())
    assert sq == ctypes.sizeof(rbfd.rbfd_quality) and oh == rbfd.rbfd_quality.hist.offset
    sj, oo, ou = map(int, d.split())
    assert sj == ctypes.sizeof(rbfd.rbfd_job)
    assert oo == rbfd.rbfd_job.opt.offset and ou == rbfd.rbfd_job.out.offset
    st, ol, oi = map(int, e.split())
    assert st == ctypes.sizeof(rbfd.rbfd_worklist_tune)
    assert ol == rbfd.rbfd_worklist_tune.launch_ms.offset and oi == rbfd.rbfd_worklist_tune.items.offset
    sso, omq, ofv = map(int, f.split())
    assert sso == ctypes.sizeof(rbfd.rbfd_server_options)
    assert omq == rbfd.rbfd_server_options.max_queue.offset and ofv == rbfd.rbfd_server_options.fuse_volume.offset
    onp, oeq = map(int, g.split())
    assert onp == rbfd.rbfd_stats.newton_pairs_useful.offset and oeq == rbfd.rbfd_stats.eq12_pairs.offset
    opr, ogf, obs = map(int, h.split())
    assert opr == rbfd.rbfd_options.prune.offset
    assert ogf == rbfd.rbfd_stats.persist_grow_fma.offset and obs == rbfd.rbfd_stats.sweep_warps_skipped.offset


def test_argument_checks_before_any_device_work(lib):
    """Calls with invalid arguments fail with RBFD_EINVAL and a message before
    they touch a device (no GPU here): bad sizes, bit counts and NULL arrays."""
    L = rbfd.load()
    i64 = ctypes.c_int64
    assert L.rbfd_sort_pairs(None, None, i64(-1), 32, None) == rbfd.EINVAL
    assert b"n out of range" in L.rbfd_last_error()
    assert L.rbfd_sort_pairs(None, None, i64(4), 0, None) == rbfd.EINVAL
    assert L.rbfd_sort_pairs(None, None, i64(4), 33, None) == rbfd.EINVAL
    assert b"key_bits" in L.rbfd_last_error()
    assert L.rbfd_sort_pairs(None, None, i64(0), 32, None) == rbfd.OK  # nothing to sort
    assert L.rbfd_sort_pairs(None, None, i64(4), 32, None) == rbfd.EINVAL  # NULL arrays
    assert b"device memory" in L.rbfd_last_error()
