"""riesz_apply_noalloc against riesz_apply through the C ABI.

riesz_apply_noalloc is for callers that must not allocate device memory on
their hot path; its scratch is a fixed array inside the library.  This file
is collected last so that, if it fails, a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [rz.APPLY_ELEMENT, rz.APPLY_MATRIX_FREE])
def test_noalloc_apply_matches_apply_twice(mode):
    verts, cells = kuhn_mesh(3, 0.1, 21)
    s = rz.Riesz("N1curl", 3, verts, cells, apply_mode=mode)
    for seed in (1, 2):  # two calls in a row, different inputs
        x = torch.tensor(normal_vector(s.N, seed), device="cuda")
        y_ref = torch.zeros_like(x)
        y_new = torch.full_like(x, float("nan"))
        s.apply(x, y_ref)
        s.apply_noalloc(x, y_new)
        torch.cuda.synchronize()
        a, b = y_ref.cpu().numpy(), y_new.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_noalloc_apply_rejects_meshes_beyond_its_scratch():
    verts, cells = kuhn_mesh(16, 0.0, 0)
    s = rz.Riesz("N1curl", 5, verts, cells, apply_mode=rz.APPLY_MATRIX_FREE)
    assert (s.nref - s.nint_cell) * s.ncells > 1 << 21
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    rc = s.lib.riesz_apply_noalloc(s.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None)
    assert rc == 1
    assert b"exceeds the fixed scratch" in s.lib.riesz_last_error()
