"""Checkpoint and resume of the BFMG solve (Alg. 4) at a cycle boundary.

A solve stopped after c cycles, its state moved to another problem handle built from
the same mesh and resumed, must give outputs bit-identical to the uninterrupted solve:
every kernel reduces in a fixed order, the row-kernel shapes and CUDA-graph replay do
not change results, so the continued cycles repeat the same arithmetic.  The stops
fall on level 2, on level 3, on the first cycle of the finest level (state taken just
after the prolongation) and inside it, in both arithmetics (the precision form's
hand-over to float64 included)."""
import numpy as np
import pytest

from paper_1511_07042_gb300 import inputs

pytestmark = pytest.mark.gpu
R, K, NW, TOL = 4, 20, 12, 1e-10


def problem(bmg, r=R):
    v, t = inputs.icosahedron()
    p = bmg.Problem(v, t, r)
    p.hierarchy(r)
    return p


def opts(bmg, precision, **kw):
    return bmg.options(precision=precision, smoother="mcsgs", nu=1, omega=1.0, **kw)


@pytest.fixture(scope="module")
def reference(gpu_bmg):
    out = {}
    X0 = inputs.gaussian_block(inputs.n_vertices(2), K, 17)
    for precision in ("fp64", "fp32"):
        ev, U, rs, info = problem(gpu_bmg).solve(X0, K, NW, 0.0, TOL, opts(gpu_bmg, precision))
        assert info.converged == 1
        out[precision] = (X0, ev, U, rs, info)
    return out


@pytest.mark.parametrize("precision,stop", [("fp64", 3), ("fp64", 8), ("fp64", 12), ("fp64", 17),
                                            ("fp32", 10), ("fp32", 12), ("fp32", 20)])
def test_resume_is_bit_identical(gpu_bmg, reference, precision, stop):
    X0, ev, U, rs, info = reference[precision]
    assert info.total_cycles > stop
    p1 = problem(gpu_bmg)
    ev1, _, rs1, info1 = p1.solve(X0, K, NW, 0.0, TOL, opts(gpu_bmg, precision, stop_after_cycles=stop),
                                  evecs=False)
    assert info1.converged == 0 and info1.total_cycles == stop
    assert info1.history() == info.history()[:stop]
    state = p1.get_state(K)
    p2 = problem(gpu_bmg)
    p2.set_state(K, state)
    ev2, U2, rs2, info2 = p2.solve(None, K, NW, 0.0, TOL, opts(gpu_bmg, precision, resume=True))
    assert info2.converged == 1
    assert np.array_equal(ev2, ev) and np.array_equal(rs2, rs) and np.array_equal(U2, U)
    assert (info2.total_cycles, info2.fp32_cycles) == (info.total_cycles, info.fp32_cycles)
    assert list(info2.cycles) == list(info.cycles)
    assert info2.history() == info.history()
    assert info2.max_dense_err == info.max_dense_err


def test_state_errors(gpu_bmg, reference):
    X0 = reference["fp64"][0]
    p = problem(gpu_bmg)
    with pytest.raises(gpu_bmg.BmgError) as e:
        p.get_state(K)                                   # nothing stopped yet
    assert e.value.code == 8
    with pytest.raises(gpu_bmg.BmgError) as e:
        p.solve(None, K, NW, 0.0, TOL, opts(gpu_bmg, "fp64", resume=True))
    assert e.value.code == 8                             # no state given
    p.solve(X0, K, NW, 0.0, TOL, opts(gpu_bmg, "fp64", stop_after_cycles=5), evecs=False)
    state = p.get_state(K)
    with pytest.raises(gpu_bmg.BmgError) as e:
        p.set_state(K, state[:-8])                       # truncated
    assert e.value.code == 1
    with pytest.raises(gpu_bmg.BmgError) as e:
        problem(gpu_bmg, 3).set_state(K, state)          # another hierarchy
    assert e.value.code == 1
    p.set_state(K, state)
    with pytest.raises(gpu_bmg.BmgError) as e:
        p.solve(None, K, NW, 1.0, TOL, opts(gpu_bmg, "fp64", resume=True))
    assert e.value.code == 1                             # sigma differs from the state's
