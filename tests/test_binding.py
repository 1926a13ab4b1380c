"""The Python binding refuses arrays of the wrong shape, length, dtype or device before it
calls the library, which reads and writes exactly the sizes it expects (runs without a GPU)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def ddg():
    import paper_2402_08296_b300 as m
    return m


def test_host_arrays_of_the_wrong_shape_are_refused(ddg):
    xy = np.zeros((4, 2))
    tri = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    with pytest.raises(ValueError, match="xy"):
        ddg.ddg_mesh_upload(None, xy.ravel(), tri)
    with pytest.raises(ValueError, match="tri"):
        ddg.ddg_mesh_upload(None, xy, tri.ravel())
    with pytest.raises(ValueError, match="dirichlet"):
        ddg.ddg_mesh_upload(None, xy, tri, dirichlet=np.zeros(3, np.uint8))
    with pytest.raises(ValueError, match="r"):
        ddg.ddg_assemble_poly(None, np.zeros(8))
    with pytest.raises(ValueError, match="w"):
        ddg.ddg_model_create(None, 30, 10, 1e-3, np.zeros(10, np.float32))
    with pytest.raises(ValueError, match="xy"):
        ddg.ddg_submit(None, xy.ravel(), tri, np.zeros(9), ddg.DDG_DDM_LU)
    with pytest.raises(ValueError, match="r"):
        ddg.ddg_submit(None, xy, tri, np.zeros(3), ddg.DDG_DDM_LU)


def test_device_arrays_of_the_wrong_kind_are_refused(ddg):
    import torch
    cpu64 = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError, match="not on a CUDA device"):
        ddg.ddg_precondition(None, cpu64, cpu64)
    with pytest.raises(TypeError, match="float64"):
        ddg.ddg_apply_A(None, torch.zeros(8, dtype=torch.float32), cpu64)
    with pytest.raises(TypeError, match="CUDA torch tensor"):
        ddg.ddg_local_corrections(None, np.zeros(8), cpu64, cpu64)
    with pytest.raises(ValueError, match="not on a CUDA device"):
        ddg.ddg_apply_A_dot_noalloc(None, cpu64, cpu64, cpu64)


def test_poll_buffer_is_sized_from_the_submitted_mesh(ddg):
    key = (0x1234, 7)
    ddg._TICKET_NODES[key] = 100
    try:
        with pytest.raises(ValueError, match="100 nodes"):
            ddg.ddg_poll(ctypes.c_void_p(0x1234), 7, 50)
    finally:
        ddg._TICKET_NODES.pop(key, None)
