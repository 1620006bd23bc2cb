"""Setup autotuner: the residency of the patch factorisation changes only the
schedule, never the factors."""
import numpy as np
import pytest

from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def precond_of(s, r):
    z = torch.zeros_like(r)
    s.precond(r, z)
    torch.cuda.synchronize()
    return z


def test_autotuned_factors_equal_untuned():
    verts, cells = kuhn_mesh(6, 0.1, 2)  # 343 vertex patches: between 1 and 24 per SM
    tuned = rz.Riesz("N1curl", 2, verts, cells)
    plain = rz.Riesz("N1curl", 2, verts, cells, autotune=0)
    t = tuned.tuning()
    assert t["candidates_timed"] == 8 and t["cholesky_ctas_per_sm"] in (0, 2, 3, 4)
    assert t["cholesky_ctas_per_patch"] in (1, 2)
    tp = plain.tuning()
    assert tp["cholesky_ctas_per_sm"] == 0 and tp["candidates_timed"] == 0
    r = torch.tensor(normal_vector(tuned.N, 3), device="cuda")
    assert torch.equal(precond_of(tuned, r), precond_of(plain, r))
    # the same for every residency after a geometry update
    verts_d = torch.tensor(verts, device="cuda")
    tuned.update_geometry(verts_d)
    assert torch.equal(precond_of(tuned, r), precond_of(plain, r))


def test_autotune_skipped_for_few_patches():
    verts, cells = kuhn_mesh(2, 0.1, 2)  # 27 patches
    s = rz.Riesz("CG", 3, verts, cells)
    assert s.tuning()["candidates_timed"] == 0


def test_cluster_factorisation_equals_single_cta():
    """Two CTAs per patch (a cluster sharing panel tiles and trailing tile pairs) give the same factors
    bitwise as one CTA per patch."""
    for space, p, n in [("N1curl", 3, 3), ("RT", 2, 4), ("CG", 4, 2)]:
        verts, cells = kuhn_mesh(n, 0.1, 5)
        s2 = rz.Riesz(space, p, verts, cells, autotune=2)
        s1 = rz.Riesz(space, p, verts, cells, autotune=0)
        assert s2.tuning()["cholesky_ctas_per_patch"] == 2 and s1.tuning()["cholesky_ctas_per_patch"] == 1
        r = torch.tensor(normal_vector(s1.N, 9), device="cuda")
        assert torch.equal(precond_of(s1, r), precond_of(s2, r))
