"""The C ABI without a GPU: the library builds, loads and exports every
function that include/gbbc.h declares; the binding names the same calls; the
header's documented constants match the binding's."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbbc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(bc_[a-z_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_05718_gb300 import _build, gbbc
    _build.build()
    return gbbc.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bc_graph_create", "bc_compute", "bc_read"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2008_05718_gb300 import _build
    out = subprocess.check_output(["nm", "-D", "--defined-only", _build.LIB]).decode()
    exported = set(re.findall(r" T (bc_[a-z_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_covers_header():
    from paper_2008_05718_gb300 import gbbc
    assert sorted(gbbc.EXPORTS) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(gbbc, n))


def test_status_strings_and_options_without_gpu(lib):
    from paper_2008_05718_gb300 import gbbc
    assert gbbc.bc_status_string(0) == "GBBC_OK"
    assert gbbc.bc_status_string(5) == "GBBC_ERR_CAPACITY"
    o = gbbc.bc_options_init()
    import ctypes
    assert o.struct_size == ctypes.sizeof(gbbc.gbbc_options)
    assert o.batch_width == 0 and o.policy == 0


def test_enum_values_match_header():
    from paper_2008_05718_gb300 import gbbc
    text = open(HEADER).read()
    for name, val in [("GBBC_OK", 0), ("GBBC_ERR_INVALID", 1), ("GBBC_ERR_OOM", 2), ("GBBC_ERR_CUDA", 3),
                      ("GBBC_ERR_TIMEOUT", 4), ("GBBC_ERR_CAPACITY", 5), ("GBBC_ERR_STATE", 6)]:
        assert re.search(rf"{name}\s*=\s*{val}\b", text)
        assert getattr(gbbc, name) == val
    for name, val in gbbc.POLICY.items():
        assert re.search(rf"GBBC_POLICY_{name.upper()}\s*=\s*{val}\b", text)


def test_create_without_device_fails_cleanly(lib):
    # no GPU here: the call must return a status, not crash
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    from paper_2008_05718_gb300 import gbbc
    with pytest.raises(gbbc.GbbcError) as e:
        gbbc.bc_graph_create(2, 2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32))
    assert e.value.status == gbbc.GBBC_ERR_CUDA


def test_product_path_has_no_oracle_dependency():
    # the CUDA library and its binding never reference the oracle
    pkg = os.path.join(ROOT, "paper_2008_05718_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".c", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_header_is_plain_c_and_links(lib, tmp_path):
    # a C99 program includes the header, links libgbbc.so and calls the
    # entry points that need no GPU
    from paper_2008_05718_gb300 import _build
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "gbbc.h"
int main(void) {
    gbbc_options o;
    bc_options_init(&o);
    if (o.struct_size != sizeof(gbbc_options) || o.schedule != GBBC_SCHEDULE_AUTO || o.streams != 0) return 1;
    if (strcmp(bc_status_string(GBBC_ERR_CAPACITY), "GBBC_ERR_CAPACITY") != 0) return 2;
    if (bc_mlp_param_count(2) <= 0 || bc_mlp_param_count(1) >= bc_mlp_param_count(2)) return 3;
    gbbc_graph* g = (gbbc_graph*)0;
    int32_t rp[2] = {0, 0};
    if (bc_graph_create(-1, 0, rp, (const int32_t*)0, &o, (void*)0, &g) != GBBC_ERR_INVALID || g) return 4;
    if (bc_compute((gbbc_graph*)0, (const int32_t*)0, 0, (void*)0) != GBBC_ERR_INVALID) return 5;
    printf("ok %d %d\n", GBBC_MAX_WEIGHT, GBBC_NOALLOC_MAX_VERTICES);
    return 0;
}
''')
    exe = tmp_path / "use"
    libdir = os.path.dirname(_build.LIB)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-L", libdir, "-l:" + os.path.basename(_build.LIB), "-Wl,-rpath," + libdir,
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stderr[-500:])
    assert out.stdout.split() == ["ok", "64", "16384"]
