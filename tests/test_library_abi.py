"""The C ABI without a GPU: the in-tree library loads, exports every function that
include/aplicur.h declares, the Python binding declares exactly those, and the ctypes
structs have the C layout (sizes and field offsets printed by a small C program
compiled against the header)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aplicur.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(aplicur_\w+)\s*\(", src)
    typedefs = set(re.findall(r"typedef\s+[^;]*?\b(aplicur_\w+)\s*;", src))
    return sorted(set(names) - typedefs)


@pytest.fixture(scope="module")
def lib():
    from paper_2604_05065_gb300 import build as B
    if not os.path.exists(B.LIB):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and no nvcc")
        B.build_library()
    return C.CDLL(B.LIB)


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("aplicur_create", "aplicur_solve", "aplicur_backward", "aplicur_destroy",
                 "aplicur_batch_create", "aplicur_batch_solve", "aplicur_dense_atx_noalloc"):
        assert must in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_exactly_the_header(lib):
    from paper_2604_05065_gb300 import aplicur as A
    assert sorted(A.SIGNATURES) == _declared()


def test_status_strings_without_gpu(lib):
    lib.aplicur_status_string.restype = C.c_char_p
    assert lib.aplicur_status_string(0) == b"ok"
    assert lib.aplicur_status_string(5) == b"factorisation breakdown"


def test_struct_layouts_match_c(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2604_05065_gb300 import aplicur as A
    structs = {"aplicur_matrix": A.Matrix, "aplicur_options": A.Options, "aplicur_stats": A.Stats,
               "aplicur_profile": A.Profile, "aplicur_batch_stats": A.BatchStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-o", str(exe), str(c)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, what, val = line.split()
        got[(cname, what)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_build_compiles_every_cuda_source():
    """Every .cu file under csrc is a translation unit of the library (a kernel file left
    out of the build would leave its entry points undefined only at load time)."""
    from paper_2604_05065_gb300 import build as B
    csrc = os.path.join(ROOT, "paper_2604_05065_gb300", "csrc")
    on_disk = sorted(f for f in os.listdir(csrc) if f.endswith(".cu"))
    assert sorted(B.SOURCES) == on_disk
