"""CPU-side checks of the C-ABI library: it builds, loads, and exports every symbol that
include/poslo.h declares (no compute calls: there is no GPU here)."""
import os
import re
import subprocess

import pytest

from paper_2506_08781_gb300 import build, poslo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "poslo.h")).read()
    return sorted(set(re.findall(r"\b(poslo_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    try:
        build.build()
    except RuntimeError as e:   # nvcc missing: the library cannot exist
        pytest.skip(str(e))
    return poslo.load_library()


def test_header_and_binding_agree():
    assert sorted(poslo.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (poslo_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    for s in _declared():
        assert hasattr(lib, s)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(poslo.PosloError):
        poslo.Context(device=0)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(poslo, "_lib", None)
    with pytest.raises(ImportError):
        poslo.load_library(str(tmp_path / "nope.so"))


def test_noalloc_rejects_misaligned_device_pointers_before_any_cuda_call(lib):
    """Device-resident offsets are read as 8-byte words and e_t written as 16-byte vectors:
    misaligned addresses are refused on the host (EINVAL) before the device is touched, so
    this runs without a GPU.  The addresses are never dereferenced."""
    import ctypes as C
    import struct
    ds = (C.c_uint8 * 24).from_buffer_copy(struct.pack("<II", 4, 0) + bytes(16))
    base = 1 << 20                               # 256-byte aligned fake device addresses
    for offs, e_out in [(base + 4, base), (base, base + 8), (base + 1, base + 1)]:
        b = poslo.Batch()
        b.variant, b.n2, b.Y, b.msgs, b.offs, b.s, b.R = poslo.VARIANT_F, 16, base, base, offs, base, base
        b.n, b.first_index, b.R_count, b.ds, b.ds_nodes, b.on_device = 8, 0, 8, C.addressof(ds), 1, 1
        assert lib.poslo_hash_entries_noalloc(C.byref(b), e_out, None) == -1


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/poslo.h compiles as C99 and a C program links against the library and gets a
    clean status from it (no GPU here: poslo_create reports POSLO_EDEVICE or another error,
    poslo_last_error(NULL) answers, and invalid arguments are refused)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include "poslo.h"
int main(void) {
  poslo_params p = {0};
  poslo_ctx* ctx = (poslo_ctx*)1;
  int rc = poslo_create(&p, &ctx);
  if (rc == POSLO_OK || ctx != NULL) return 2;
  if (poslo_create(&p, NULL) != POSLO_EINVAL) return 3;
  if (poslo_last_error(NULL) == NULL) return 4;
  poslo_destroy(NULL);
  printf("%d\n", rc);
  return 0;
}
''')
    exe = tmp_path / "use"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    build.LIB, "-Wl,-rpath," + os.path.dirname(build.LIB)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert int(r.stdout.strip()) < 0


def test_product_path_never_imports_the_oracle():
    """The package (binding, inputs, build) imports nothing from oracle/, statically or at
    run time: the oracle is test infrastructure only."""
    import ast
    import sys
    pkg = os.path.join(ROOT, "paper_2506_08781_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom) and node.module:
                    names = [node.module]
                assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (f, names)
    code = ("import sys; import paper_2506_08781_gb300.poslo, paper_2506_08781_gb300.synth; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "False", r.stderr


def test_binding_structures_match_the_header(tmp_path):
    """Every C structure of include/poslo.h and its ctypes mirror in the binding agree in size
    and in the offset of every field (compiled by the host C compiler; no GPU needed)."""
    import ctypes as C
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    pairs = {"poslo_params": poslo.Params, "poslo_batch": poslo.Batch, "poslo_multi_batch": poslo.MultiBatch,
             "poslo_partial": poslo.Partial, "poslo_request": poslo.Request, "poslo_batch_record": poslo.BatchRecord,
             "poslo_ccd_c": poslo.CcdC}
    lines = []
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "poslo.h"\nint main(void) {\n' +
                   "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            parts = ln.split()
            got[tuple(parts[:-1])] = int(parts[-1])
    for cname, py in pairs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
