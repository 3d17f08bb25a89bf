"""The seeded input generator (CPU): deterministic bytes, plane-by-plane
production identical to the whole stack, the stated intensity model, and the
serving shape mix."""
import numpy as np

import opm_synth as S


def _small(seed=3, blobs=6, background=100.0, amp=(200.0, 5000.0), sigma=(1.5, 4.0)):
    return S.StackConfig("t", 12, 40, 56, 35.0, 0.3, 0.1, n_blobs=blobs, sigma=sigma, amp=amp,
                         background=background, seed=seed)


def test_raw_stack_is_deterministic_and_seed_dependent():
    a = S.raw_stack(_small())
    b = S.raw_stack(_small())
    c = S.raw_stack(_small(seed=4))
    assert a.dtype == np.uint16 and a.shape == (12, 40, 56)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_plane_ranges_equal_the_whole_stack():
    cfg = _small()
    whole = S.raw_stack(cfg)
    out = np.empty((5, 40, 56), dtype=np.uint16)
    part = S.raw_stack(cfg, out=out, planes=(4, 9))
    assert part is out
    assert np.array_equal(part, whole[4:9])


def test_background_is_poisson_with_the_stated_mean():
    cfg = _small(blobs=0, background=100.0)
    R = S.raw_stack(cfg).astype(np.float64)
    # Poisson(100): mean 100, variance 100
    assert abs(R.mean() - 100.0) < 0.5
    assert abs(R.var() - 100.0) < 5.0


def test_blob_peak_follows_its_amplitude():
    cfg = _small(blobs=1, background=0.0, amp=(4000.0, 4000.0), sigma=(3.0, 3.0))
    centres, _, _ = S.blob_params(cfg)
    c = centres[0]
    R = S.raw_stack(cfg).astype(np.float64)
    n, r, x = (int(round(v)) for v in c)
    n, r, x = min(n, 11), min(r, 39), min(x, 55)
    d2 = ((n - c[0]) ** 2 + (r - c[1]) ** 2 + (x - c[2]) ** 2) / (2 * 9.0)
    lam = 4000.0 * np.exp(-d2)
    assert abs(R[n, r, x] - lam) < 6 * np.sqrt(lam) + 1
    # far from the blob the stack is empty (background 0)
    far = np.ones(R.shape, dtype=bool)
    far[max(0, n - 13):n + 14, max(0, r - 13):r + 14, max(0, x - 13):x + 14] = False
    assert R[far].max() == 0


def test_counts_clip_to_uint16():
    cfg = _small(blobs=3, background=70000.0)
    assert S.raw_stack(cfg).max() == 65535


def test_serve_shapes_draw_from_the_stated_sets():
    shapes = S.serve_shapes(500, seed=7)
    assert shapes == S.serve_shapes(500, seed=7)
    planes = {s[0] for s in shapes}
    assert planes <= set(range(50, 401, 50)) and len(planes) == 8
    assert {s[1] for s in shapes} == set(S.SERVE_ROWS)
    assert {s[2] for s in shapes} == set(S.SERVE_COLS)
    assert {s[3] for s in shapes} == {2}


def test_tiled_stack_repeats_one_tile():
    t = S.tiled_stack((120, 300, 600), seed=5)
    assert t.shape == (120, 300, 600) and t.dtype == np.uint16 and t.flags.c_contiguous
    assert np.array_equal(t[:50, :128, :256], t[50:100, 128:256, 256:512])


def test_gaussian_vectors_are_seeded_standard_normal():
    a = S.gaussian((200, 300), 9)
    assert np.array_equal(a, S.gaussian((200, 300), 9))
    assert abs(a.mean()) < 0.02 and abs(a.std() - 1.0) < 0.02
