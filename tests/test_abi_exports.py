"""The C ABI boundary on the host, with no GPU: the header is plain C, liblt.so
loads, and it exports exactly the functions include/*.h declares (no compute call
is made).  The library is built first if it is missing or stale (nvcc
cross-compiles without a device)."""
import ctypes
import glob
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))

_DECL = re.compile(r"^[A-Za-z_][\w \t\*]*?\b(lt_\w+)\s*\(", re.M)


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def declared():
    names = set()
    for h in HEADERS:
        for m in _DECL.finditer(_strip_comments(open(h).read())):
            line = m.group(0)
            if line.lstrip().startswith(("typedef", "#", "struct", "enum")):
                continue
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build liblt.so")
    from paper_2202_12567_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    names = declared()
    assert len(names) >= 20, names
    for must in ("lt_create", "lt_sample_pass1", "lt_sample_pass2", "lt_eval_entries", "lt_complete",
                 "lt_render", "lt_eval_entries_noalloc", "lt_complete_adm", "lt_rgb_setup", "lt_expand_rgb", "lt_make_slices_split", "lt_split_slice_count", "lt_sample_pass1_target", "lt_mesh_upload", "lt_mesh_bvh"):
        assert must in names


def test_header_is_plain_c():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    for h in HEADERS:
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-x", "c", h],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_library_loads_and_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, f"declared in include/ but not exported: {missing}"


def test_library_exports_nothing_undeclared(libpath):
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if re.search(r"\bT lt_\w+$", ln)}
    assert exported == declared()


def test_binding_wraps_every_declared_symbol():
    pytest.importorskip("torch")
    from paper_2202_12567_gb300 import lt
    assert set(lt.EXPORTED) == declared()


def test_status_strings_without_a_device(libpath):
    lib = ctypes.CDLL(libpath)
    lib.lt_status_str.restype = ctypes.c_char_p
    lib.lt_status_str.argtypes = [ctypes.c_int32]
    assert lib.lt_status_str(0) == b"ok"
    assert lib.lt_status_str(1) == b"invalid argument"
    assert lib.lt_status_str(99) == b"unknown status"
    lib.lt_last_error.restype = ctypes.c_char_p
    lib.lt_last_error.argtypes = [ctypes.c_void_p]
    assert lib.lt_last_error(None) == b"null context"
    lib.lt_create.restype = ctypes.c_int32
    lib.lt_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.lt_create(None, 0, None) == 1  # null output handle: LT_EINVAL, nothing touched


def test_split_slice_count_is_host_only_and_matches_the_oracle(libpath):
    """lt_split_slice_count plans the recursive split on the host (no device needed);
    its slice count equals the oracle's leaf sizes for many (m, target)."""
    from oracle import slices
    lib = ctypes.CDLL(libpath)
    f = lib.lt_split_slice_count
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int64, ctypes.c_int32]
    rng = np.random.default_rng(0)
    cases = [(1, 1), (7, 2), (1000, 100), (65536, 800), (262144, 800)]
    cases += [(int(rng.integers(1, 200000)), int(rng.integers(1, 5000))) for _ in range(40)]
    for m, target in cases:
        assert f(m, target) == len(slices.split_sizes(m, target)), (m, target)
    assert f(0, 10) == -1 and f(10, 0) == -1


def test_binding_structs_match_the_c_layout(tmp_path):
    """Every struct the binding mirrors has the C size and field offsets (compiled
    with the system C compiler against include/lt.h)."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_2202_12567_gb300 import lt
    structs = {"lt_tree": lt.lt_tree, "lt_frame": lt.lt_frame, "lt_samples": lt.lt_samples,
               "lt_factors": lt.lt_factors, "lt_rgb": lt.lt_rgb, "lt_params": lt.lt_params,
               "lt_tuning": lt.lt_tuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lt.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for row in out:
        if not row:
            continue
        name, what, value = row.split()
        cls = structs[name]
        want = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert int(value) == want, (name, what, int(value), want)
        seen += 1
    assert seen == sum(1 + len(c._fields_) for c in structs.values())
