"""Pins of the oracle's system matrix (the strip-integral projector) against
closed forms, an exact identity and brute-force integration."""
import math

import numpy as np
import pytest

import oracle


def _problem(nx, ny, V, D, angles=None, **kw):
    y = np.zeros((V, D))
    return oracle.Problem(nx, ny, V, D, y, np.ones((V, D)), view_angles=angles, **kw)


def test_column_sums_equal_pixel_area():
    """sum_c A[c, s] * dd = dx^2 for every pixel whose footprint is on the
    detector (the strip integrals of one pixel partition its area)."""
    for dx, dd in [(1.0, 1.0), (1.0, 0.8), (0.7, 1.1)]:
        P = _problem(9, 7, 17, 31, pixel_pitch=dx, channel_pitch=dd)
        for m in range(17):
            for i in range(7):
                for j in range(9):
                    c0, v = P.footprint(m, i, j)
                    assert 1 <= len(v) <= 3
                    assert abs(v.sum() * dd - dx * dx) < 1e-14
                    assert np.all(v > 0)


def test_theta_zero_box():
    """theta = 0: the profile is a box of width dx; odd image on an odd detector
    puts every pixel exactly on one channel (value 1); an even image straddles
    two channels (1/2, 1/2)."""
    P = _problem(5, 5, 4, 11)
    for j in range(5):
        c0, v = P.footprint(0, 2, j)
        assert len(v) == 1 and v[0] == 1.0
        assert c0 == j - 2 + 5   # x = j - 2, channel holding [x + 5.5 - 0.5, ...)
    P = _problem(4, 4, 4, 11)
    for j in range(4):
        c0, v = P.footprint(0, 1, j)
        np.testing.assert_array_equal(v, [0.5, 0.5])


def test_theta_quarter_pi_triangle():
    """theta = pi/4: the profile is a triangle of half-width 1/sqrt(2); a pixel
    centred on a channel gets sqrt(2) - 1/2 there and 3/4 - 1/sqrt(2) on each
    side (areas of the triangle's pieces)."""
    P = _problem(5, 5, 4, 11)
    c0, v = P.footprint(1, 2, 2)   # centre pixel, view 1 of 4 = pi/4
    assert len(v) == 3
    side = 0.75 - 1.0 / math.sqrt(2.0)
    np.testing.assert_allclose(v, [side, math.sqrt(2.0) - 0.5, side], rtol=0, atol=1e-15)


def test_brute_force_integration():
    """Strip integrals against direct integration of the pixel indicator over
    a fine grid (2x2 image, random angles, non-unit pitches)."""
    rng = np.random.default_rng(4)
    angles = rng.uniform(0, np.pi, 6)
    dx, dd, off = 1.0, 0.9, 0.23
    P = _problem(2, 2, 6, 7, angles=angles, pixel_pitch=dx, channel_pitch=dd, channel_offset=off)
    K = 1200
    u = (np.arange(K) + 0.5) / K - 0.5
    for m, th in enumerate(angles):
        for i in range(2):
            for j in range(2):
                xc = (j - 0.5) * dx
                yc = (0.5 - i) * dx
                X = xc + dx * u[None, :]
                Y = yc + dx * u[:, None]
                t = X * math.cos(th) + Y * math.sin(th)
                q = (t - off) / dd + 3.5
                ch = np.floor(q).astype(int)
                counts = np.bincount(ch.ravel(), minlength=7)
                brute = counts * (dx * dx / (K * K)) / dd
                c0, v = P.footprint(m, i, j)
                ref = np.zeros(7)
                ref[c0:c0 + len(v)] = v
                assert np.abs(ref - brute).max() < 3e-3


def test_dense_matches_footprints():
    P = _problem(6, 5, 8, 13)
    A = P.dense_A()
    for m in range(8):
        for i in range(5):
            for j in range(6):
                c0, v = P.footprint(m, i, j)
                col = A[m * 13:(m + 1) * 13, i * 6 + j]
                ref = np.zeros(13)
                ref[c0:c0 + len(v)] = v
                np.testing.assert_array_equal(col, ref)


def test_detector_clipping():
    """Pixels whose footprint leaves a too-narrow detector keep only the
    channels that exist (run length may drop to 0)."""
    P = _problem(16, 16, 4, 5)
    seen_short = False
    for m in range(4):
        for i in range(16):
            for j in range(16):
                c0, v = P.footprint(m, i, j)
                if len(v):
                    assert 0 <= c0 and c0 + len(v) <= 5
                seen_short |= len(v) == 0
    assert seen_short


def test_interleaved_partition():
    """J_i = {m : m mod N = i} (0-based reading of Sec. II-A)."""
    P = oracle.Problem(4, 4, 10, 7, np.zeros((10, 7)), np.ones((10, 7)), n_agents=4)
    assert P.agent_views(0).tolist() == [0, 4, 8]
    assert P.agent_views(3).tolist() == [3, 7]
    allv = np.concatenate([P.agent_views(g) for g in range(4)])
    assert sorted(allv.tolist()) == list(range(10))
