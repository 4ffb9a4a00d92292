"""The boundary from C: `include/pc.h` compiles on its own as strict C99 and as
C++17, and a C program linked against the library gets, from host-only calls
(no GPU needed), the same sizes, version and status strings as the Python
binding, and the argument errors the header documents.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "pc.h"

int main(void) {
    pc_config cfg;
    uint64_t bound = 0, ws = 0, ws_perm = 0, dws = 0, big = 0;
    memset(&cfg, 0, sizeof cfg);
    cfg.leaf_size = 777;
    int a = pc_compress_bound(1000003, PC_F64, &cfg, &bound);
    int b = pc_compress_workspace_size(1000003, PC_F64, &cfg, 0, &ws);
    int c = pc_compress_workspace_size(1000003, PC_F64, &cfg, 1, &ws_perm);
    int d = pc_decompress_workspace_size(1000003, &dws);
    int e = pc_compress_bound(PC_MAX_PARTICLES + 1, PC_F32, &cfg, &big);
    cfg.leaf_size = PC_MAX_LEAF_SIZE + 1;
    int f = pc_compress_bound(1000, PC_F32, &cfg, &big);
    printf("%d %d %d %d %d %d\n", a, b, c, d, e, f);
    printf("%llu %llu %llu %llu\n", (unsigned long long)bound, (unsigned long long)ws,
           (unsigned long long)ws_perm, (unsigned long long)dws);
    printf("%d\n", pc_format_version());
    printf("%s\n", pc_error_string(PC_ERR_ARG));
    printf("%s\n", pc_error_string(PC_ERR_CORRUPT));
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    import paper_2404_02826_gb300 as pc

    pc.load()  # raises when the library is not built
    return pc


def _need(tool):
    if shutil.which(tool) is None:
        pytest.skip(f"{tool} not found")


@pytest.mark.parametrize("compiler,flags", [("gcc", ["-x", "c", "-std=c99"]), ("g++", ["-x", "c++", "-std=c++17"])])
def test_header_compiles_alone(tmp_path, compiler, flags):
    _need(compiler)
    src = tmp_path / "only_header.src"
    src.write_text('#include "pc.h"\nint pc_header_probe(void) { return PC_OK + PC_F32 + PC_EB_ABS; }\n')
    r = subprocess.run([compiler, *flags, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", INC, "-c", str(src),
                        "-o", str(tmp_path / "only_header.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_matches_the_binding(tmp_path, lib):
    _need("gcc")
    pc = lib
    src = tmp_path / "sizes.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "sizes"
    libdir = os.path.dirname(pc.LIB_PATH)
    name = os.path.basename(pc.LIB_PATH)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", INC, str(src), "-o", str(exe),
                        "-L", libdir, "-l:" + name, "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr
    lines = run.stdout.splitlines()
    status = [int(x) for x in lines[0].split()]
    assert status[:4] == [pc.PC_OK] * 4
    assert status[4:] == [pc.PC_ERR_ARG, pc.PC_ERR_ARG]
    sizes = [int(x) for x in lines[1].split()]
    assert sizes == [pc.pc_compress_bound(1000003, pc.PC_F64, 777),
                     pc.pc_compress_workspace_size(1000003, pc.PC_F64, 777, False),
                     pc.pc_compress_workspace_size(1000003, pc.PC_F64, 777, True),
                     pc.pc_decompress_workspace_size(1000003)]
    # room for the input indices is always planned: the permutation needs it, and
    # so do lossless axes (Sec. 4.1), which only the value range reveals
    assert sizes[2] == sizes[1]
    assert int(lines[2]) == pc.pc_format_version()
    assert lines[3] == pc.pc_error_string(pc.PC_ERR_ARG) and lines[4] == pc.pc_error_string(pc.PC_ERR_CORRUPT)


LAYOUT_STRUCTS = ("pc_config", "pc_info", "pc_compress_item", "pc_decompress_item", "pc_sweep_point", "pc_request",
                  "pc_completion", "pc_tuned_class")


def test_struct_layouts_match_the_binding(tmp_path, lib):
    """Every struct of the header, as a C compiler lays it out (size and the
    offset of each field), equals the binding's ctypes declaration."""
    _need("gcc")
    pc = lib
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pc.h"', "int main(void) {"]
    for name in LAYOUT_STRUCTS:
        st = getattr(pc, name)
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in st._fields_:
            lines.append(f'    printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", INC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr
    import ctypes

    seen = 0
    for line in run.stdout.splitlines():
        name, field, value = line.split()
        st = getattr(pc, name)
        want = ctypes.sizeof(st) if field == "size" else getattr(st, field).offset
        assert int(value) == want, (name, field)
        seen += 1
    assert seen == sum(len(getattr(pc, s)._fields_) + 1 for s in LAYOUT_STRUCTS)
