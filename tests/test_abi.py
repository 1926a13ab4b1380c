"""The C ABI library loads on a machine without a GPU and exports every symbol include/ddg.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "ddg.h")) as fh:
        text = fh.read()
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
