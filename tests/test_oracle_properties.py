"""Property tests of the oracle over random small geometries (CPU).

Each example draws a plan (planes, rows, columns, angle, scan step, pixel)
and checks facts that hold for every geometry: the row-wise gather equals
the matrix built entry by entry from the interpolation kernel, the adjoint
is its transpose, and the output extent holds exactly the columns that carry
weight (readings 2-7).
"""
import numpy as np
import pytest

import oracle as O

hyp = pytest.importorskip("hypothesis")
st = hyp.strategies
given, settings = hyp.given, hyp.settings

geometries = st.tuples(
    st.integers(2, 9),                                   # nscan
    st.integers(1, 5),                                   # nrows
    st.integers(1, 3),                                   # ncols
    st.sampled_from([15.0, 30.0, 35.0, 45.0, 60.0, 72.5, 90.0]),
    st.sampled_from([0.05, 0.1, 0.2, 0.3, 0.4, 0.7]),    # scan step
    st.sampled_from([0.1, 0.115, 0.2]),                  # pixel
)


def _small(shape):
    g = O.geometry(*shape)
    return g if g.nz * g.ny * g.nx * g.nscan * g.nrows * g.ncols <= 1_500_000 else None


@settings(max_examples=60, deadline=None, derandomize=True)
@given(geometries, st.integers(0, 2**31 - 1), st.sampled_from([O.LINEAR, O.NEAREST]))
def test_gather_equals_entrywise_matrix(shape, seed, interp):
    g = _small(shape)
    hyp.assume(g is not None)
    R = np.random.default_rng(seed).standard_normal((g.nscan, g.nrows, g.ncols))
    A = O.explicit_matrix(g, interp)
    np.testing.assert_allclose(O.deskew(R, g, interp).ravel(), A @ R.ravel(), rtol=0, atol=1e-12)


@settings(max_examples=60, deadline=None, derandomize=True)
@given(geometries, st.integers(0, 2**31 - 1))
def test_adjoint_is_transpose(shape, seed):
    g = _small(shape)
    hyp.assume(g is not None)
    Y = np.random.default_rng(seed).standard_normal((g.nz, g.ny, g.nx))
    A = O.explicit_matrix(g)
    np.testing.assert_allclose(O.skew_adjoint(Y, g).ravel(), A.T @ Y.ravel(), rtol=0, atol=1e-12)


@settings(max_examples=200, deadline=None, derandomize=True)
@given(geometries)
def test_extent_is_exactly_the_weighted_columns(shape):
    """Every column of [0, ny) carries weight from some plane of some row,
    and no column past the last does: the extent formula is tight on the
    right and covers every sample (reading 6).  The exception: when one row
    step moves a column by more than nscan + 1 planes (cos(theta) x
    pixel/step > nscan + 1, a thin stack sampled by coarse rows), a column's
    rows can step over the whole stack, so inside the grid some columns
    carry no weight (the last one among them); the first column still does."""
    g = O.geometry(*shape)
    k = np.arange(g.nz)[:, None]
    def weighted(j):
        nf = O.plane_coord(g, np.asarray(j)[None, :], k)          # [nz, len(j)]
        return np.any((nf > -1.0 + 1e-9) & (nf < g.nscan - 1e-9), axis=0)
    w = weighted(np.arange(g.ny))
    if g.c * g.pixel / g.step <= g.nscan + 1:
        assert w.all()
    else:
        assert w[0] and w.any()
    assert not weighted(np.arange(g.ny, g.ny + 3)).any()
    # every raw sample reaches some output column with a non-zero weight,
    # unless columns step over whole planes (pixel >= 2 step, reading 6)
    if g.pixel >= 2.0 * g.step:
        return
    for r in range(g.nrows):
        nf = O.plane_coord(g, np.arange(g.ny), r)
        for n in range(g.nscan):
            assert np.any(np.abs(nf - n) < 1.0 - 1e-12), (r, n)


@settings(max_examples=200, deadline=None, derandomize=True)
@given(geometries)
def test_extent_is_tight_on_the_left(shape):
    """Column 0 carries weight and the column before it would not: J0 puts
    the first weighted column of the grid at index 0 (reading 6)."""
    g = O.geometry(*shape)
    k = np.arange(g.nz)
    def weighted(j):
        nf = O.plane_coord(g, j, k)
        return bool(np.any((nf > -1.0 + 1e-9) & (nf < g.nscan - 1e-9)))
    assert weighted(0)
    assert not weighted(-1)
