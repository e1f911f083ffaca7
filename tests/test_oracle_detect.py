"""Pins of the detection oracle (score normalisation and candidate
extraction, Section 3.3) to closed forms, brute force and statistics."""
import collections

import numpy as np
import pytest

from oracle import detect as od


def _all_valid(shape):
    return np.zeros(shape, dtype=np.int32)


def test_spike_closed_form():
    # one value a among zeros: mean a/n, variance a^2 (n-1)/n^2, so the spike
    # sits at z = sqrt(n - 1) and every other pixel of its window at
    # -1/sqrt(n - 1); with z = s / sigma the spike is at n / sqrt(n - 1)
    H, W, w = 40, 50, 15
    s = np.zeros((H, W))
    y, x, a = 20, 25, 3.7
    s[y, x] = a
    for fn in (od.local_stats, od.local_stats_direct):
        n, mean, sd = fn(s, _all_valid(s.shape), w)
        assert n[y, x] == w * w
        z, flag = od.normalise(s, _all_valid(s.shape), n, mean, sd, 3.0)
        assert z[y, x] == pytest.approx(np.sqrt(w * w - 1), rel=1e-12)
        assert z[y, x - 3] == pytest.approx(-1 / np.sqrt(w * w - 1), rel=1e-12)
        assert z[y, x + 8] == 0.0  # window of (y, x + 8) misses the spike: constant, sigma 0
        assert flag.sum() == 1
        zl, _ = od.normalise(s, _all_valid(s.shape), n, mean, sd, 3.0, subtract_mean=False)
        assert zl[y, x] == pytest.approx(w * w / np.sqrt(w * w - 1), rel=1e-12)


def test_clipped_window_counts():
    # a spike in a corner: its square holds (R + 1)^2 in-image pixels
    H, W, w = 30, 30, 11
    R = w // 2
    s = np.zeros((H, W))
    s[0, 0] = 1.0
    n, mean, sd = od.local_stats(s, _all_valid(s.shape), w)
    assert n[0, 0] == (R + 1) ** 2
    assert n[0, 3] == (R + 1) * (R + 4)
    assert n[H // 2, W // 2] == w * w
    z, _ = od.normalise(s, _all_valid(s.shape), n, mean, sd, 3.0)
    assert z[0, 0] == pytest.approx(np.sqrt((R + 1) ** 2 - 1), rel=1e-12)


def test_invalid_pixels_are_left_out():
    g = np.random.default_rng(1)
    s = g.normal(size=(25, 27))
    a = np.where(g.random(s.shape) < 0.2, -1, 3).astype(np.int32)
    n, mean, sd = od.local_stats(s, a, 7)
    # the same statistics with the invalid pixels' scores changed
    s2 = np.where(a < 0, 1e6, s)
    n2, mean2, sd2 = od.local_stats(s2, a, 7)
    np.testing.assert_array_equal(n, n2)
    np.testing.assert_allclose(mean, mean2, rtol=0, atol=1e-9)
    np.testing.assert_allclose(sd ** 2, sd2 ** 2, rtol=0, atol=1e-9)
    z, flag = od.normalise(s, a, n, mean, sd, -100.0)
    assert not flag[a < 0].any() and (z[a < 0] == 0).all()


@pytest.mark.parametrize("w", [1, 3, 7, 255])
def test_summed_area_matches_definition(w):
    g = np.random.default_rng(w)
    s = g.normal(2.0, 0.5, size=(23, 31))
    a = np.where(g.random(s.shape) < 0.1, -1, 0).astype(np.int32)
    n0, m0, d0 = od.local_stats_direct(s, a, w)
    n1, m1, d1 = od.local_stats(s, a, w)
    np.testing.assert_array_equal(n0, n1)
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-12)
    # the variance as mean square minus squared mean resolves ~1e-15 of the
    # mean square (sigma itself only its square root near 0)
    np.testing.assert_allclose(d1 ** 2, d0 ** 2, rtol=0, atol=1e-12)
    big = d0 > 1e-3
    np.testing.assert_allclose(d1[big], d0[big], rtol=1e-9)
    if w == 1:
        z, flag = od.normalise(s, a, n1, m1, d1, 0.0)
        assert (z == 0).all() and not flag.any()  # one pixel per window: no sigma


def test_affine_invariance_and_constant():
    g = np.random.default_rng(2)
    s = g.normal(size=(33, 29))
    a = _all_valid(s.shape)
    z0, f0 = od.normalise(s, a, *od.local_stats(s, a, 9), 1.5)
    s2 = 4.0 * s + 7.0
    z1, f1 = od.normalise(s2, a, *od.local_stats(s2, a, 9), 1.5)
    np.testing.assert_allclose(z1, z0, rtol=1e-9, atol=1e-9)
    c = np.full((10, 10), 2.5)
    z2, f2 = od.normalise(c, a[:10, :10], *od.local_stats(c, a[:10, :10], 5), 0.0)
    assert (z2 == 0).all() and not f2.any()


def _flood(flag):
    """Components by breadth-first flood fill over 8 neighbours."""
    H, W = flag.shape
    lab = np.zeros((H, W), dtype=np.int64)
    cur = 0
    for y in range(H):
        for x in range(W):
            if flag[y, x] and not lab[y, x]:
                cur += 1
                lab[y, x] = cur
                q = collections.deque([(y, x)])
                while q:
                    cy, cx = q.popleft()
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            ny, nx = cy + dy, cx + dx
                            if 0 <= ny < H and 0 <= nx < W and flag[ny, nx] and not lab[ny, nx]:
                                lab[ny, nx] = cur
                                q.append((ny, nx))
    return lab, cur


@pytest.mark.parametrize("p", [0.1, 0.35, 0.6])
def test_components_match_flood_fill(p):
    g = np.random.default_rng(int(p * 100))
    flag = g.random((40, 37)) < p
    lab, count = od.components(flag)
    ref, rcount = _flood(flag)
    assert count == rcount
    # same partition: a one-to-one map between the labels
    pairs = set(zip(lab[flag].tolist(), ref[flag].tolist()))
    assert len(pairs) == count == len({a for a, _ in pairs}) == len({b for _, b in pairs})


def test_diagonal_touch_is_one_component():
    flag = np.eye(6, dtype=bool)
    assert od.components(flag)[1] == 1
    chk = (np.add.outer(np.arange(8), np.arange(8)) % 2) == 0
    assert od.components(chk)[1] == 1


def test_detection_peak_and_order():
    # two blobs; the first has two pixels of equal z: the smaller index wins
    H, W = 60, 60
    s = np.zeros((H, W))
    s[10, 10] = s[10, 11] = 5.0
    s[11, 10] = 4.0
    s[40, 40] = 6.0
    s[40, 41] = 1.0
    a = np.full((H, W), 2, dtype=np.int32)
    a[40, 40] = 7
    det, z, flag = od.detections(s, a, window=255, threshold=3.0)
    assert len(det) == 2
    assert (det[0]["y"], det[0]["x"], det[0]["k"]) == (40, 40, 7)
    assert (det[1]["y"], det[1]["x"], det[1]["npix"]) == (10, 10, 3)
    assert det[0]["z"] > det[1]["z"] > 3.0
    assert det[0]["z"] == pytest.approx(z[40, 40])
    assert det[0]["npix"] == flag[39:42, 39:43].sum()


def test_noise_statistics():
    # pure N(0, 1) scores: local mean ~0 and sigma ~1, and the share of
    # pixels above 3 sigma near the normal tail 1.35e-3
    g = np.random.default_rng(5)
    s = g.normal(size=(512, 512))
    a = _all_valid(s.shape)
    n, mean, sd = od.local_stats(s, a, 255)
    c = (slice(128, 384), slice(128, 384))
    assert abs(mean[c]).max() < 0.02
    assert abs(sd[c] - 1).max() < 0.02
    z, flag = od.normalise(s, a, n, mean, sd, 3.0)
    frac = flag.mean()
    assert abs(frac - 1.3499e-3) < 5 * np.sqrt(1.35e-3 / s.size)
