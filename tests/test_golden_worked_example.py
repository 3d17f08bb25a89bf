"""The paper's printed worked example of the remapped display size against
the sheet-frame extent (oracle and library host code).  The scan step of
that example is not printed, so the shear per image it implies is derived
from the printed sizes and the check is one of consistency: the extent
formula must reproduce the printed display exactly for that shear, and the
printed micrometre sizes must equal the pixel counts times the pixel."""
import json
import os

import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_example_display.json")


@pytest.fixture(scope="module")
def ex():
    with open(GOLDEN) as f:
        return json.load(f)


def test_oracle_extent_reproduces_printed_display(ex):
    n, rows = ex["images_per_stack"], ex["roi_rows"]
    shear = (ex["display_rows"] - rows) / (n - 1)          # rows per image implied by the example
    assert O.sheet_rows(n, rows, shear) == ex["display_rows"]
    # a shear whose last image lands one row lower gives one row less
    assert O.sheet_rows(n, rows, (ex["display_rows"] - rows - 1) / (n - 1)) == ex["display_rows"] - 1
    # the displayed width is the camera ROI width (no remap across columns)
    assert ex["display_cols"] == ex["roi_cols"]


def test_printed_micrometres_match_pixels(ex):
    um_y, um_x = ex["display_um"]
    assert abs(ex["display_rows"] * ex["pixel_um"] - um_y) < 0.5
    assert abs(ex["display_cols"] * ex["pixel_um"] - um_x) < 0.5


def test_library_extent_matches(ex, tmp_path):
    import paper_2211_00645_gb300 as lib
    if not os.path.exists(lib.LIB_PATH):
        pytest.skip("libopm.so not built")
    n, rows = ex["images_per_stack"], ex["roi_rows"]
    shear = (ex["display_rows"] - rows) / (n - 1)
    assert lib.opm_sheet_rows(n, rows, shear) == ex["display_rows"]
