"""The C ABI library builds, loads without a GPU and exports every entry point that
include/*.h declares; the header itself is valid C.  No compute call is made."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(ipg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_2010_01542_gb300 as ipg
    from paper_2010_01542_gb300 import _build

    _build.build()
    return ipg.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ipg_graph_create", "ipg_graph_create_dev", "ipg_graph_destroy", "ipg_pagerank",
                     "ipg_pagerank_dev", "ipg_hashmin_cc", "ipg_hashmin_cc_dev", "ipg_sssp", "ipg_sssp_dev",
                     "ipg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_pure_host_calls(lib):
    import paper_2010_01542_gb300 as ipg

    assert ipg.ipg_version() >= 100
    assert lib.ipg_status_string(0) == b"IPG_OK"
    assert lib.ipg_status_string(7) == b"IPG_EOVERFLOW"
    assert lib.ipg_status_string(8) == b"IPG_ECANCELED"
    assert ipg.STATUS_NAMES[ipg.IPG_ECANCELED] == "IPG_ECANCELED"
    assert lib.ipg_server_cancel(None, 0, None) == 1
    # a NULL graph is rejected on the host, before any CUDA call
    assert lib.ipg_graph_info(None, None, None, None, None) == 1
    assert b"NULL" in lib.ipg_last_error()
    assert lib.ipg_graph_create(None, None, None, 0, 0, 1, None) == 1
    assert lib.ipg_graph_check_symmetric(None, None, None) == 1


def test_header_is_valid_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "ipg.h"\nint main(void){ ipg_stats s = {0}; (void)s; return (int)IPG_OK; }\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I",
                           os.path.join(ROOT, "include"), str(src)])


def test_missing_library_fails_loudly(tmp_path):
    import paper_2010_01542_gb300 as ipg

    with pytest.raises(ipg.IpgLibraryMissing):
        ipg.load_library(str(tmp_path / "nope.so"))


def test_host_alloc_argument_checks(lib):
    """ipg_host_alloc / ipg_host_free reject bad arguments on the host, before any CUDA call."""
    alloc, free = lib.ipg_host_alloc, lib.ipg_host_free
    alloc.argtypes, alloc.restype = [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int
    free.argtypes, free.restype = [ctypes.c_void_p], ctypes.c_int
    assert alloc(16, None) == 1
    p = ctypes.c_void_p(1234)
    assert alloc(0, ctypes.byref(p)) == 0 and p.value is None  # empty request: NULL, no mapping
    assert free(None) == 0
    junk = ctypes.create_string_buffer(64)
    assert free(ctypes.addressof(junk)) == 1  # not from ipg_host_alloc: refused, nothing released
    assert b"ipg_host_alloc" in lib.ipg_last_error()


def test_plain_c_program_links_and_calls_the_library(tmp_path, lib):
    """A C99 program built against include/ipg.h and linked with libipg.so calls the
    host-side entry points (no GPU needed): version, status names, argument errors."""
    from paper_2010_01542_gb300 import _build

    libdir = os.path.dirname(_build.library_path())
    src = tmp_path / "use_ipg.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "ipg.h"
int main(void) {
    if (ipg_version() < 100) return 1;
    if (strcmp(ipg_status_string(IPG_EINVAL), "IPG_EINVAL") != 0) return 2;
    if (ipg_graph_info(NULL, NULL, NULL, NULL, NULL) != IPG_EINVAL) return 3;
    if (strlen(ipg_last_error()) == 0) return 4;
    ipg_graph* g = NULL;
    if (ipg_graph_create(NULL, NULL, NULL, 0, 0, 1, &g) != IPG_EINVAL || g != NULL) return 5;
    void* p = (void*)1;
    if (ipg_host_alloc(0, &p) != IPG_OK || p != NULL) return 6;
    if (ipg_server_cancel(NULL, 0, NULL) != IPG_EINVAL) return 7;
    ipg_graph_destroy(NULL);
    puts("ok");
    return 0;
}
''')
    exe = tmp_path / "use_ipg"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-L", libdir, "-lipg", "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
