"""Failures made on the host and reported as statuses, never as a GPU fault: an open
(non-manifold) input mesh, a forced cycle cap of one cycle (partial results with
their residuals), and a NaN-poisoned start block."""
import numpy as np
import pytest

from paper_1511_07042_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_open_mesh_is_rejected(gpu_bmg):
    v, t = inputs.icosahedron()
    with pytest.raises(gpu_bmg.BmgError) as e:
        gpu_bmg.Problem(v, t[:-1], 2)          # one face removed: three edges on one triangle
    assert e.value.code == 7                   # BMG_ERR_MESH
    with pytest.raises(gpu_bmg.BmgError) as e:
        gpu_bmg.Problem(v, np.vstack([t, t[:1]]), 2)   # a face twice: its edges on three triangles
    assert e.value.code == 7


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cycle_cap_of_one_returns_partial_results(gpu_bmg, precision):
    v, t = inputs.icosahedron()
    p = gpu_bmg.Problem(v, t, 3)
    p.hierarchy(3)
    X0 = inputs.gaussian_block(inputs.n_vertices(2), 20, 3)
    ev, U, rs, info = p.solve(X0, 20, 16, 0.0, 1e-10, gpu_bmg.options(max_cycles=1, precision=precision))
    assert info.converged == 0
    assert info.total_cycles == 6 + 1 and list(info.cycles[:2]) == [6, 1]
    assert np.all(np.isfinite(ev)) and np.all(np.isfinite(rs)) and np.all(np.isfinite(U))
    assert info.max_resid == rs.max() > 1e-10
    assert np.all(np.diff(ev) >= -1e-12 * np.abs(ev).max())    # ascending Ritz values near sigma = 0


def test_nan_start_block_is_reported(gpu_bmg):
    v, t = inputs.icosahedron()
    p = gpu_bmg.Problem(v, t, 3)
    p.hierarchy(3)
    X0 = inputs.gaussian_block(inputs.n_vertices(2), 20, 3)
    X0[7, :] = np.nan
    with pytest.raises(gpu_bmg.BmgError) as e:
        p.solve(X0, 20, 16, 0.0, 1e-10, gpu_bmg.options(precision="fp32"))
    assert e.value.code in (4, 6)              # BMG_ERR_SINGULAR or BMG_ERR_NONFINITE
