"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/wg.h declares; the declared structs match the binding's."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:wg_status|void|const char\*|uint64_t)\s+(wg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libwg():
    from paper_2601_04370_gb300 import build
    build.build()
    from paper_2601_04370_gb300 import wg
    return wg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("wg_init", "wg_shutdown", "wg_create_design", "wg_set_params", "wg_destroy_design",
              "wg_eval_coating", "wg_trace_forward", "wg_trace_backward", "wg_loss", "wg_last_error",
              "wg_submit", "wg_poll", "wg_cancel", "wg_autotune"):
        assert n in names


def test_library_exports_every_declared_symbol(libwg):
    missing = [n for n in declared_functions() if not hasattr(libwg, n)]
    assert not missing, missing


def test_exports_with_nm():
    from paper_2601_04370_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(wg_\w+)", out))
    assert set(declared_functions()) <= exported


def test_version_and_error_string_without_gpu(libwg):
    from paper_2601_04370_gb300 import wg
    assert "sm_103a" in wg.version()
    assert isinstance(libwg.wg_last_error(), bytes)


def test_struct_sizes_match_header():
    """Layout of the ctypes mirrors against a C compile of the header."""
    from paper_2601_04370_gb300 import wg
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "wg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(wg_init_opts), sizeof(wg_design_desc), sizeof(wg_trace_cfg),
         sizeof(wg_stats), sizeof(wg_ray_record));
  printf("%zu %zu %zu\n", offsetof(wg_trace_cfg, stream), offsetof(wg_trace_cfg, ray_records),
         offsetof(wg_stats, kernel_ms));
  printf("%zu %zu %zu %zu\n", sizeof(wg_request), sizeof(wg_result), offsetof(wg_request, cfg),
         offsetof(wg_result, stats));
  return 0;
}
'''
    import tempfile
    tmp = tempfile.mkdtemp(prefix="wg_abi_")
    c = os.path.join(tmp, "abi_sizes.c")
    exe = os.path.join(tmp, "abi_sizes")
    open(c, "w").write(code)
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
    a, b, c2 = subprocess.check_output([exe], text=True).strip().splitlines()
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(wg.InitOpts), ctypes.sizeof(wg.DesignDesc), ctypes.sizeof(wg.TraceCfg),
                     ctypes.sizeof(wg.Stats), wg.RAY_RECORD_DTYPE.itemsize]
    assert offs == [wg.TraceCfg.stream.offset, wg.TraceCfg.ray_records.offset, wg.Stats.kernel_ms.offset]
    assert [int(x) for x in c2.split()] == [ctypes.sizeof(wg.Request), ctypes.sizeof(wg.Result),
                                             wg.Request.cfg.offset, wg.Result.stats.offset]
