"""The C-ABI library builds, loads without a GPU and exports every function
that include/zr.h declares; the Python binding names the same set."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "zr.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    names = set()
    for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(zr_\w+)\s*\(", src, flags=re.M):
        if "typedef" in src[m.start():m.end()]:
            continue
        names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("zr_create", "zr_vandermonde_solve_batched", "zr_newton_batched", "zr_zippel_step", "zr_reconstruct",
              "zr_serve_create", "zr_serve_submit", "zr_serve_wait", "zr_serve_destroy"):
        assert f in names
    assert len(names) > 30


def test_library_exports_every_declared_symbol():
    from paper_2505_24256_gb300 import build as zb
    from paper_2505_24256_gb300 import zr

    path = zb.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for each of them, and nothing else
    assert set(zr.SIGNATURES) == declared_functions()
    # host-only calls work without a device
    assert lib.zr_status_string(0)


def test_struct_layouts_match_the_header():
    """Every struct the binding mirrors has the header's size and field
    offsets (a C program built from include/zr.h with gcc reports them)."""
    import subprocess
    import tempfile

    from paper_2505_24256_gb300 import zr

    structs = {name: getattr(zr, name) for name in dir(zr)
               if name.startswith("zr_") and isinstance(getattr(zr, name), type)
               and issubclass(getattr(zr, name), ctypes.Structure)}
    assert {"zr_blackbox", "zr_recon_params", "zr_result", "zr_request", "zr_poly", "zr_vsys", "zr_step_desc",
            "zr_serve_stats", "zr_peaks"} <= set(structs)
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "zr.h"', "int main(void) {"]
    for name, cls in sorted(structs.items()):
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[tuple(parts[:2])] = int(parts[2])
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
