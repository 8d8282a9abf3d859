"""The C-ABI library loads and exports every symbol include/*.h declares, and
host-side argument checks reject bad inputs without touching a GPU (no GPU)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_07936_gb300 import build, mg
    build.build()
    return mg.load()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mg_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mg_setup", "mg_solve", "mg_vcycle", "mg_load_prolong_weights",
                     "mg_solve_batched", "mg_destroy", "mg_set_options", "mg_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2403_07936_gb300 import mg
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in mg.SIGNATURES, f"{name} has no binding signature"


def test_status_strings(lib):
    assert lib.mg_status_string(0) == b"MG_OK"
    assert lib.mg_status_string(8) == b"MG_ERR_NONFINITE"


@pytest.mark.parametrize("levels,N", [(4, 63), (4, 6), (0, 64), (1, 64), (9, 64), (20, 2048)])
def test_setup_rejects_invalid_sizes(lib, levels, N):
    h = C.c_void_p(123)
    st = lib.mg_setup(levels, N, C.byref(h))
    assert st == 1  # MG_ERR_INVALID_ARG
    assert h.value is None
    assert lib.mg_last_error()


def test_weights_blob_layout_matches_generator_shapes():
    from paper_2403_07936_gb300 import sr
    from synthetic.weights import random_weights, weight_shapes
    w = random_weights(0)
    blob = sr.pack_weights(w)
    n_params = sum(int(__import__("numpy").prod(s)) for _, s in weight_shapes())
    assert len(blob) == 64 + 4 * n_params
    assert blob[:8] == b"MGSRW001"


@pytest.mark.parametrize("args", [(1 << 30, -1, 2, 2, 10, 1e-10), (1 << 30, 2, 5, 2, 10, 1e-10),
                                  (1 << 30, 2, 2, -1, 10, 1e-10), (1 << 30, 2, 2, 17, 10, 1e-10),
                                  (1 << 30, 2, 2, 2, 0, 1e-10),
                                  (1 << 30, 2, 2, 2, 10, float("nan"))])
def test_server_create_rejects_invalid_options(lib, args):
    h = C.c_void_p(123)
    st = lib.mg_server_create(*args, None, C.byref(h))
    assert st == 1
    assert h.value is None


def test_server_calls_reject_null_server(lib):
    from paper_2403_07936_gb300 import mg
    f = (C.c_double * 64)()
    assert lib.mg_server_submit(None, 0, 8, f, None, None) == 1
    assert lib.mg_server_tick(None, None, None, None) == 1
    r, got = mg.ServerResult(), C.c_int()
    assert lib.mg_server_poll(None, C.byref(r), C.byref(got)) == 1


def test_tile_variant_table_host_logic(lib):
    """The tile-variant table is host state: set, read back, reject bad entries (no GPU)."""
    from paper_2403_07936_gb300 import mg
    old_d, old_u = mg.get_tile_variant(0, 4096, 3), mg.get_tile_variant(1, 4096, 3)
    assert old_d in range(4) and old_u in range(8)
    try:
        mg.set_tile_variant(1, 4096, 3, 6)
        assert mg.get_tile_variant(1, 4096, 3) == 6
        mg.set_tile_variant(0, 4096, 3, 3)
        assert mg.get_tile_variant(0, 4096, 3) == 3
        for bad in [(0, 4096, 3, 4), (1, 4096, 3, 8), (1, 4096, 3, -1), (2, 4096, 3, 0), (1, 96, 3, 0),
                    (1, 64, 3, 0), (1, 4096, 5, 0)]:
            with pytest.raises(mg.MGError):
                mg.set_tile_variant(*bad)
    finally:
        mg.set_tile_variant(0, 4096, 3, old_d)
        mg.set_tile_variant(1, 4096, 3, old_u)


def test_empty_batch_is_a_no_op(lib):
    """A batch of zero right-hand sides succeeds without touching a device."""
    from paper_2403_07936_gb300 import mg
    H, F, X = (C.c_void_p * 1)(), (C.c_void_p * 1)(), (C.c_void_p * 1)()
    infos = (mg.SolveInfo * 1)()
    assert lib.mg_solve_batched(H, F, X, 0, 1e-10, 0, infos) == 0
    assert lib.mg_solve_batched(H, F, X, -1, 1e-10, 0, infos) == 1


def test_binding_fails_loudly_without_the_library():
    """No CPU fallback: a missing libmg.so is an ImportError naming the build step."""
    import subprocess
    import sys
    code = ("from paper_2403_07936_gb300 import mg\n"
            "mg.load('" + os.path.join(ROOT, "no_such_dir", "libmg.so") + "')\n")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=120)
    assert p.returncode != 0
    assert "ImportError" in p.stderr and "no CPU fallback" in p.stderr


def test_every_declared_function_is_documented():
    """Each entry point of include/mg.h is preceded by its comment block."""
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        lines = open(h).read().split("\n")
        for i, line in enumerate(lines):
            m = re.match(r"^(?:mg_status|const char \*|void|unsigned long long|int)\s+\**(mg_\w+)\s*\(", line)
            if m:
                assert "*/" in "\n".join(lines[max(0, i - 3):i]), f"{m.group(1)} has no comment block"


def test_allocation_free_entry_point_source_calls_no_allocator():
    """The translation unit of mg_op_vcycle_static names no CUDA allocation call."""
    import re
    src = open(os.path.join(ROOT, "paper_2403_07936_gb300", "csrc", "mg_noalloc.cu")).read()
    code = "\n".join(line.split("//")[0] for line in src.splitlines())
    assert not re.search(r"cuda(Malloc|Free|MallocAsync|FreeAsync|MallocHost|HostAlloc|MallocManaged)\s*\(", code)
