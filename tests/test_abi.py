"""C-ABI checks that need no GPU: the library loads, exports every entry point
that include/*.h declares, the ctypes mirrors of the header's structs have
the C layout, and compute entry points refuse to run without a device (no CPU
fallback)."""
import ctypes
import glob
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    path = os.path.join(ROOT, "paper_1702_04458_b300", "libdbp.so")
    if not os.path.exists(path):
        import importlib.util
        spec = importlib.util.spec_from_file_location(
            "dbp_build", os.path.join(ROOT, "paper_1702_04458_b300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
    import paper_1702_04458_b300 as p
    return p


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(dbp_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dbp_create", "dbp_destroy", "dbp_uplink_admm", "dbp_uplink_cg",
                     "dbp_downlink_admm"):
        assert required in names


def test_library_exports_every_declared_symbol(pkg):
    lib = ctypes.CDLL(pkg.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(dbp_\w+)", out))
    assert set(_declared_functions()) <= exported


def test_struct_layouts_match_header(pkg):
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "dbp.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(dbp_frame_desc), sizeof(dbp_config), sizeof(dbp_tuning));
  printf("%zu %zu %zu %zu %zu\n", offsetof(dbp_frame_desc, flags), offsetof(dbp_frame_desc, rho),
         offsetof(dbp_frame_desc, Es), offsetof(dbp_frame_desc, box_r), offsetof(dbp_frame_desc, eps));
  printf("%zu\n", offsetof(dbp_config, hbm_budget_bytes));
  printf("%zu %zu\n", offsetof(dbp_tuning, kernel), offsetof(dbp_tuning, prefactor));
  printf("%zu %zu %zu %zu\n", sizeof(dbp_request), offsetof(dbp_request, channel_key),
         sizeof(dbp_result), offsetof(dbp_result, finish_us));
  printf("%zu %zu %zu\n", sizeof(dbp_graph_item), offsetof(dbp_graph_item, H), offsetof(dbp_graph_item, beta_out));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        vals = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in vals]
    D = pkg.dbp_frame_desc
    assert vals[:3] == [ctypes.sizeof(D), ctypes.sizeof(pkg.dbp_config), ctypes.sizeof(pkg.dbp_tuning)]
    assert vals[3:8] == [D.flags.offset, D.rho.offset, D.Es.offset, D.box_r.offset, D.eps.offset]
    assert vals[8] == pkg.dbp_config.hbm_budget_bytes.offset
    assert vals[9:11] == [pkg.dbp_tuning.kernel.offset, pkg.dbp_tuning.prefactor.offset]
    R = pkg.dbp_request
    assert vals[11:15] == [ctypes.sizeof(R), R.channel_key.offset, ctypes.sizeof(pkg.dbp_result),
                          pkg.dbp_result.finish_us.offset]
    G = pkg.dbp_graph_item
    assert vals[15:18] == [ctypes.sizeof(G), G.H.offset, G.beta_out.offset]


def test_enum_values_match_the_header(pkg):
    """Every DBP_* enumerator the binding defines has the header's value."""
    names = sorted(n for n in dir(pkg) if n.startswith("DBP_") and isinstance(getattr(pkg, n), int))
    body = "".join(f'  printf("%lld\\n", (long long){n});\n' for n in names)
    prog = "#include <stdio.h>\n#include \"dbp.h\"\nint main(void) {\n" + body + "  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "e.c")
        exe = os.path.join(d, "e")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [getattr(pkg, n) for n in names]
    assert "DBP_PATH_BCAST" in names


def test_version_string(pkg):
    assert "sm_103a" in pkg.dbp_version()


def test_no_cpu_fallback_without_device(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; this checks the CPU-only refusal")
    with pytest.raises(pkg.DbpError) as ei:
        pkg.dbp_create(0)
    assert ei.value.status == pkg.DBP_ERR_CUDA


def test_null_handle_is_rejected(pkg):
    lib = ctypes.CDLL(pkg.LIB_PATH)
    lib.dbp_uplink_admm.restype = ctypes.c_int
    lib.dbp_uplink_admm.argtypes = [ctypes.c_void_p] * 7
    assert lib.dbp_uplink_admm(None, None, None, None, None, None, None) == pkg.DBP_ERR_INVALID_ARG
    lib.dbp_last_error.restype = ctypes.c_char_p
    lib.dbp_last_error.argtypes = [ctypes.c_void_p]
    assert lib.dbp_last_error(None) == b"NULL handle"


def test_every_header_is_a_build_dependency():
    """An object older than any header a translation unit may include is
    rebuilt: the kernels' .cuh, the library's internal .h (which holds the
    handle's struct) and the public header.  A stale object with an old
    struct layout would read the handle at wrong offsets."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "dbp_build_deps", os.path.join(ROOT, "paper_1702_04458_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    newest = mod._deps_mtime()
    csrc = os.path.join(ROOT, "paper_1702_04458_b300", "csrc")
    headers = (glob.glob(os.path.join(csrc, "*.h")) + glob.glob(os.path.join(csrc, "*.cuh")) +
               glob.glob(os.path.join(ROOT, "include", "*.h")))
    assert any(h.endswith("dbp_internal.h") for h in headers)
    assert newest == max(os.path.getmtime(h) for h in headers)
