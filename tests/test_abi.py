"""The C ABI library loads on a machine without a GPU and exports every symbol include/ddg.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = ""
    inc = os.path.join(ROOT, "include")
    for name in sorted(os.listdir(inc)):
        if name.endswith(".h"):
            with open(os.path.join(inc, name)) as fh:
                text += fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ddg_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("ddg_create", "ddg_mesh_upload", "ddg_assemble_poly", "ddg_partition",
                     "ddg_model_create", "ddg_setup_precond", "ddg_precondition", "ddg_fcg_solve"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    import paper_2402_08296_b300 as ddg
    lib = ctypes.CDLL(ddg.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert isinstance(ddg.ddg_last_error(), str)


def test_binding_covers_every_symbol():
    import paper_2402_08296_b300 as ddg
    for n in declared_symbols():
        assert hasattr(ddg, n), n


def test_null_handles_are_refused_with_a_status():
    """Every entry point returns a status for NULL handles and outputs, with a message, before
    it touches a device: no abort and no exception crosses the boundary (runs without a GPU)."""
    import paper_2402_08296_b300 as ddg
    lib = ddg.lib
    nul = None
    calls = {
        "ddg_create": (0, 0, nul),
        "ddg_memory_in_use": (nul, nul),
        "ddg_get_stream": (nul, nul),
        "ddg_launch_count": (nul,),
        "ddg_mesh_upload": (nul, 3, nul, 1, nul, nul, nul),
        "ddg_assemble_poly": (nul, nul),
        "ddg_assemble_nodal": (nul, nul, nul),
        "ddg_problem_info": (nul, nul),
        "ddg_matrix_download": (nul, nul, nul, nul, nul),
        "ddg_partition": (nul, 4, 1, nul),
        "ddg_partition_download": (nul, nul, nul, nul, nul),
        "ddg_graph_download": (nul, nul, nul, nul, nul, nul),
        "ddg_coarse_download": (nul, nul, nul),
        "ddg_model_create": (nul, 30, 10, 1e-3, nul, 0, 0, nul),
        "ddg_model_get_weights": (nul, nul, 0),
        "ddg_model_set_weights": (nul, nul, 0),
        "ddg_setup_precond": (nul, ddg.DDG_DDM_LU, nul, 0),
        "ddg_precondition": (nul, nul, nul, nul),
        "ddg_local_corrections": (nul, nul, nul, nul, nul),
        "ddg_apply_A": (nul, nul, nul, nul),
        "ddg_apply_A_dot_noalloc": (nul, nul, nul, nul, nul),
        "ddg_train_local_model": (nul, nul, nul, nul),
        "ddg_train_loss_grad": (nul, nul, nul, nul, 1, nul, nul),
        "ddg_submit": (nul, 3, nul, 1, nul, nul, nul, nul),
        "ddg_poll": (nul, 1, nul, nul),
        "ddg_serve_config": (nul, 1, 0, 1),
        "ddg_serve_stats": (nul, nul),
        "ddg_fcg_solve": (nul, nul, 1e-6, 10, 10, nul, nul),
        "ddg_fcg_history": (nul, nul, 0, nul),
        "ddg_probe_fma_peaks": (0, nul, nul),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == ddg.DDG_INVALID_ARG, name
        assert ddg.ddg_last_error(), name
    for name in ("ddg_destroy", "ddg_problem_destroy", "ddg_model_destroy"):
        assert getattr(lib, name)(nul) == ddg.DDG_OK, name
    declared = set(declared_symbols()) - {"ddg_last_error"}
    assert declared <= set(calls) | {"ddg_destroy", "ddg_problem_destroy", "ddg_model_destroy"}


def test_status_codes_match_the_header():
    import paper_2402_08296_b300 as ddg
    with open(os.path.join(ROOT, "include", "ddg.h")) as fh:
        text = fh.read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(DDG_[A-Z_]+)\s*=\s*(-?\d+)", text)}
    for name in ("DDG_OK", "DDG_INVALID_ARG", "DDG_OOM", "DDG_CUDA_ERROR", "DDG_NOT_CONVERGED",
                 "DDG_BREAKDOWN", "DDG_BUSY", "DDG_TIMEOUT", "DDG_PENDING", "DDG_BAD_MESH",
                 "DDG_TOO_LARGE", "DDG_INTERNAL"):
        assert getattr(ddg, name) == codes[name], name
        if codes[name] < 0:
            assert codes[name] in ddg.STATUS_NAMES, name
