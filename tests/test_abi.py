"""The C ABI library builds, loads without a GPU and exports every entry point that
include/*.h declares; the header itself is valid C.  No compute call is made."""
import ctypes
import glob
import os
import re
import subprocess
import sys

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
    assert lib.ipg_graph_create_profile(None, None) == 1
    assert lib.ipg_sssp_batch_info(None, None) == 1


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


_NULL_PROBE = r'''
import ctypes, re, sys
import paper_2010_01542_gb300 as ipg
lib = ipg.load_library()
text = re.sub(r"/\*.*?\*/", "", open(sys.argv[1]).read(), flags=re.S)
bad = []
seen = 0
for m in re.finditer(r"^\s*(ipg_status|uint32_t|double|void)\s+(ipg_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M):
    ret, name, params = m.groups()
    ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
    if not ps or not re.search(r"\b(ipg_graph|ipg_server)\s*\*", ps[0]):
        continue
    fn = getattr(lib, name)
    fn.argtypes = None
    fn.restype = {"ipg_status": ctypes.c_int, "uint32_t": ctypes.c_uint32, "double": ctypes.c_double}.get(ret)
    args = [ctypes.c_void_p(None) if "*" in p else ctypes.c_double(0) if "double" in p
            else ctypes.c_uint64(0) if "64" in p else ctypes.c_uint32(0) for p in ps]
    r = fn(*args)
    seen += 1
    if ret == "ipg_status" and r != 1:
        bad.append((name, r))
    if ret in ("uint32_t", "double") and r != 0:
        bad.append((name, r))
print(seen, bad)
'''


def test_every_handle_entry_point_rejects_null(tmp_path, lib):
    """Each entry point whose first argument is a graph or server handle, called with NULL
    for every pointer and 0 for every number, returns IPG_EINVAL (or 0 / nothing) on the
    host before any CUDA call, and nothing crashes.  Runs in a child process."""
    script = tmp_path / "null_probe.py"
    script.write_text(_NULL_PROBE)
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, str(script), os.path.join(ROOT, "include", "ipg.h")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    seen, bad = r.stdout.strip().rsplit("\n", 1)[-1].split(" ", 1)
    assert int(seen) >= 20 and bad == "[]", r.stdout


def test_no_cpu_fallback_without_a_gpu(lib):
    """With no CUDA device the product path refuses to run (IPG_ECUDA), never computing on
    the host instead: graph creation from valid host arrays and the host allocator."""
    import numpy as np
    import torch

    import paper_2010_01542_gb300 as ipg

    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    offsets = np.array([0, 1, 2], dtype=np.uint64)
    cols = np.array([1, 0], dtype=np.uint32)
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_graph_create(offsets, cols, None, 2, 2, False)
    assert e.value.status == ipg.IPG_ECUDA
    with pytest.raises(ipg.IpgError) as e:
        ipg.host_empty(1 << 20, np.uint32)
    assert e.value.status in (ipg.IPG_ECUDA, ipg.IPG_ENOMEM)
