"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function that
include/ef.h declares; argument checks that need no device return the documented codes."""
import ctypes
import os
import re

import paper_1704_07369_gb300 as ef

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ef.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(ef_[A-Za-z0-9_]+)\s*\(", src))


def test_library_exports_every_declared_symbol():
    ef.build()
    lib = ef.lib()
    names = _declared()
    assert names == set(ef.SYMBOLS)
    for n in names:
        assert hasattr(lib, n), n


def test_host_side_argument_checks():
    lib = ef.lib()
    h = ctypes.c_void_p()
    assert lib.ef_plan_create(4, 16, 8.0, 0, 16, 0, ctypes.byref(h)) == ef.EF_ERR_INVALID_ARG
    assert b"d must be" in lib.ef_last_error()
    assert lib.ef_plan_create(3, 16, -1.0, 1, 32, 0, ctypes.byref(h)) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_plan_create(2, 16, 8.0, 1, 16, 0, ctypes.byref(h)) == ef.EF_ERR_UNSUPPORTED
    assert lib.ef_plan_create(2, 16, 8.0, 0, 15, 0, ctypes.byref(h)) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_plan_create(3, 16, 8.0, 1, 30, 0, ctypes.byref(h)) == ef.EF_ERR_UNSUPPORTED
    assert lib.ef_plan_create(3, 16, 8.0, 1, 32, 0, None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_collide(None, None, None, 1, None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_plan_destroy(None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_status_string(ef.EF_ERR_POSITIVITY) == b"EF_ERR_POSITIVITY"
    Ns = (ctypes.c_int * 3)(24, 32, 24)
    sp = ctypes.c_void_p()
    assert lib.ef_stream_plan_create(3, 3, Ns, 8.0, 1, 32, 0, 0, ctypes.byref(sp)) == ef.EF_ERR_INVALID_ARG
    assert b"nchunks" in lib.ef_last_error()
    assert lib.ef_stream_plan_create(3, 0, Ns, 8.0, 1, 32, 0, 2, ctypes.byref(sp)) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_stream_plan_create(3, 3, Ns, 8.0, 1, 32, 0, 2, None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_stream_plan_destroy(None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_stream_euler_step(None, None, 0.01, 1, None, None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_rk3_step(None, None, 0.01, 1, None, 1, None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_transport_step(None, None, None, 4, 0.1, 0.01, None) == ef.EF_ERR_INVALID_ARG
    c = ctypes.c_void_p()
    assert lib.ef_classical_create(7, 8.0, 0.0, 1, ctypes.byref(c)) == ef.EF_ERR_INVALID_ARG      # odd N
    assert lib.ef_classical_create(130, 8.0, 0.0, 1, ctypes.byref(c)) == ef.EF_ERR_INVALID_ARG    # N > 128
    assert lib.ef_classical_create(16, -1.0, 0.0, 1, ctypes.byref(c)) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_classical_create(16, 8.0, 0.0, 1, None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_classical_collide(None, None, None, 1, None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_classical_destroy(None) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_plan_reserve(None, 4) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_mlp_status(None, 0, 0) == ef.EF_ERR_INVALID_ARG
    assert lib.ef_status_string(ef.EF_ERR_TIMEOUT) == b"EF_ERR_TIMEOUT"


def test_no_operation_allocates_or_synchronises():
    """The operations of a plan take every buffer from the plan (made at creation or by
    ef_plan_reserve): no allocation, free or device synchronisation inside them.  Checked on the
    source of the operation bodies: every cudaMalloc / cudaFree / cudaDeviceSynchronize sits in a
    create, reserve, destroy, status, autotune or table-building function."""
    allowed = re.compile(r"^(ef_plan_create\w*|ef_plan_reserve|ef_plan_destroy|ef_plan_status|ef_mlp_status|"
                         r"ef_mlp_create|ef_mlp_destroy|ef_mlp_params|ef_surrogate_create|ef_surrogate_destroy|ef_surrogate_set_checker|"
                         r"ef_surrogate_stats|ef_stream_plan_create|ef_stream_plan_destroy|ef_classical_create|"
                         r"ef_classical_destroy|ef_galerkin_create|gfree|choose_shape|upload_table|build_class|alloc_workspaces|"
                         r"destroy_plan|finish_plan|cfree|\w*_free)$")
    csrc = os.path.join(ROOT, "paper_1704_07369_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if not fn.endswith((".cpp", ".cu")):
            continue
        with open(os.path.join(csrc, fn)) as f:
            lines = f.read().split("\n")
        func = None
        for ln in lines:
            m = re.match(r"^(?:static\s+)?[A-Za-z_][\w:<>\s\*&]*?\b(\w+)\s*\([^;]*$", ln)
            if m and not ln.startswith((" ", "\t", "#", "//")) and m.group(1) not in ("if", "for", "while", "switch"):
                func = m.group(1)
            code = ln.split("//")[0]
            if re.search(r"\b(cudaMalloc|cudaFree|cudaDeviceSynchronize|cudaMallocAsync)\s*\(", code):
                assert func is not None and allowed.match(func), (fn, func, ln.strip())


def test_oracle_is_not_on_the_product_path():
    """The package never imports the oracle (only tests, smoke and the bench's CPU legs do)."""
    pkg = os.path.join(ROOT, "paper_1704_07369_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".cpp", ".h", ".inc")):
                with open(os.path.join(dirpath, fn)) as f:
                    src = f.read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), fn
                assert "ef_oracle" not in src and "liboracle" not in src, fn
