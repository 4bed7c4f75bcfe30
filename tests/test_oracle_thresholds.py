"""Pins for the oracle's thresholding operators (Section 2.2).

Four independent checks: hand-derived values (tests/golden), the textbook
rules they reduce to at d = 1 (Fan & Li 2001 SCAD rule, Gao & Bruce firm
threshold for MCP), continuity at every region boundary, and brute-force
minimisation of the per-coordinate surrogate 1/2 d b^2 - u b + P(b) on a fine
grid (the update is the proximal map of P, Section 2.1 M-step).
"""
import math
import os

import numpy as np
import pytest

from oracle import (Penalty, penalty_value, threshold_enet, threshold_group_lasso,
                    threshold_lasso, threshold_mcp, threshold_scad)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                out.append(line.split())
    return out


def _apply(kind, u, wl, par, d):
    u = np.array([u])
    if kind == "lasso":
        return threshold_lasso(u, wl, d)[0]
    if kind == "enet":
        return threshold_enet(u, wl, par, d)[0]
    if kind == "mcp":
        return threshold_mcp(u, wl, par, d)[0]
    if kind == "scad":
        return threshold_scad(u, wl, par, d)[0]
    raise ValueError(kind)


def test_golden_scalar_thresholds():
    rows = _rows("thresholds.txt")
    assert len(rows) >= 20
    for kind, u, wl, par, d, exp in rows:
        got = _apply(kind, float(u), float(wl), float(par), float(d))
        assert got == pytest.approx(float(exp), abs=1e-14, rel=1e-14), (kind, u, wl, par, d)


def test_golden_group_threshold():
    for u1, u2, cl, d, b1, b2 in _rows("group_thresholds.txt"):
        u = np.array([float(u1), float(u2)])
        got = threshold_group_lasso(u, [np.array([0, 1])], np.array([float(cl)]), float(d))
        assert got == pytest.approx([float(b1), float(b2)], abs=1e-15)


def _fan_li(z, lam, a):
    # Fan & Li (2001), Eq. (2.8): the SCAD thresholding rule for an orthonormal design.
    if abs(z) <= 2 * lam:
        return math.copysign(max(abs(z) - lam, 0.0), z)
    if abs(z) <= a * lam:
        return ((a - 1) * z - math.copysign(a * lam, z)) / (a - 2)
    return z


def _firm(z, lam, g):
    # Firm threshold (Gao & Bruce 1997; MCP solution for an orthonormal design, Zhang 2010).
    if abs(z) <= g * lam:
        return math.copysign(max(abs(z) - lam, 0.0), z) / (1.0 - 1.0 / g)
    return z


@pytest.mark.parametrize("lam", [0.3, 1.0, 2.5])
def test_reduce_to_textbook_rules_at_d1(lam):
    zs = np.linspace(-12, 12, 2401)
    for a in (2.5, 3.0, 3.7, 6.0):
        got = threshold_scad(zs, lam, a, 1.0)
        exp = np.array([_fan_li(z, lam, a) for z in zs])
        np.testing.assert_allclose(got, exp, rtol=0, atol=1e-12)
    for g in (1.5, 3.0, 8.0):
        got = threshold_mcp(zs, lam, g, 1.0)
        exp = np.array([_firm(z, lam, g) for z in zs])
        np.testing.assert_allclose(got, exp, rtol=0, atol=1e-12)
    exp = np.sign(zs) * np.maximum(np.abs(zs) - lam, 0)
    np.testing.assert_allclose(threshold_lasso(zs, lam, 1.0), exp, atol=1e-15)


def test_continuity_at_region_boundaries():
    eps = 1e-9
    for d in (1.0, 2.0, 3.3):
        wl, g = 0.7, 3.7
        for b in ((d + 1) * wl, wl * g * d, wl):
            lo = threshold_scad(np.array([b - eps]), wl, g, d)[0]
            hi = threshold_scad(np.array([b + eps]), wl, g, d)[0]
            assert abs(hi - lo) < 1e-7
        g = 3.0
        for b in (wl * g * d, wl):
            lo = threshold_mcp(np.array([b - eps]), wl, g, d)[0]
            hi = threshold_mcp(np.array([b + eps]), wl, g, d)[0]
            assert abs(hi - lo) < 1e-7
        b = 0.5 * wl
        lo = threshold_enet(np.array([b - eps]), wl, 0.5, d)[0]
        hi = threshold_enet(np.array([b + eps]), wl, 0.5, d)[0]
        assert abs(hi - lo) < 1e-7


@pytest.mark.parametrize("kind,par", [("lasso", 0.0), ("enet", 0.5), ("enet", 0.0),
                                      ("mcp", 3.0), ("mcp", 1.5), ("scad", 3.7), ("scad", 2.5)])
def test_threshold_is_prox_by_grid_search(kind, par):
    """beta = argmin_b 1/2 d b^2 - u b + P(b), checked by brute force on a grid."""
    rng = np.random.default_rng(5)
    grid = np.linspace(-12, 12, 480001)   # spacing 5e-5
    for _ in range(40):
        d = float(rng.uniform(1.0, 3.0))
        lam = float(rng.uniform(0.1, 1.5))
        u = float(rng.uniform(-10, 10))
        pen = Penalty(kind, alpha=par if kind == "enet" else 1.0,
                      gamma=par if kind in ("mcp", "scad") else 3.0)
        if kind == "mcp" and par * d <= 1:
            continue
        if kind == "scad" and (par - 1) * d <= 1:
            continue
        f = 0.5 * d * grid * grid - u * grid
        if kind == "lasso":
            f = f + lam * np.abs(grid)
        elif kind == "enet":
            f = f + par * lam * np.abs(grid) + 0.5 * (1 - par) * lam * grid * grid
        else:
            f = f + _pen_vec(kind, grid, lam, par)
        # the oracle's penalty value agrees with the Table 1 forms used here
        for b in (0.05, 1.234, -4.5):
            assert penalty_value(np.array([b]), lam, pen) == pytest.approx(
                _scalar_pen(kind, b, lam, par), rel=1e-12, abs=1e-15)
        b_star = grid[int(np.argmin(f))]
        got = _apply(kind, u, lam, par, d)
        assert abs(got - b_star) <= 1e-4, (kind, par, d, lam, u, got, b_star)


def _pen_vec(kind, b, lam, g):
    a = np.abs(b)
    if kind == "mcp":
        return np.where(a <= g * lam, lam * a - a * a / (2 * g), g * lam * lam / 2)
    if kind == "scad":
        return np.where(a <= lam, lam * a,
                        np.where(a <= g * lam, -(a * a - 2 * g * lam * a + lam * lam) / (2 * (g - 1)),
                                 (g + 1) * lam * lam / 2))
    raise ValueError(kind)


def _scalar_pen(kind, b, lam, par):
    if kind == "lasso":
        return lam * abs(b)
    if kind == "enet":
        return par * lam * abs(b) + 0.5 * (1 - par) * lam * b * b
    return float(_pen_vec(kind, np.array([b]), lam, par)[0])


def test_group_threshold_is_prox_radially():
    """Group update = argmin_b 1/2 d ||b||^2 - u^T b + c lambda ||b||; the
    minimiser is parallel to u, so a 1-D grid search over the radius pins it."""
    rng = np.random.default_rng(7)
    radii = np.linspace(0, 10, 200001)
    for _ in range(30):
        u = rng.normal(size=4) * rng.uniform(0.1, 3)
        d = float(rng.uniform(1, 3))
        cl = float(rng.uniform(0.1, 4))
        nu = np.linalg.norm(u)
        f = 0.5 * d * radii ** 2 - nu * radii + cl * radii
        r = radii[int(np.argmin(f))]
        exp = u / nu * r
        got = threshold_group_lasso(u, [np.arange(4)], np.array([cl]), d)
        np.testing.assert_allclose(got, exp, atol=1e-4)


def test_thresholds_monotone_in_u():
    u = np.linspace(-20, 20, 4001)
    for f in (lambda v: threshold_lasso(v, 1.0, 2.0), lambda v: threshold_enet(v, 1.0, 0.3, 2.0),
              lambda v: threshold_mcp(v, 1.0, 3.0, 2.0), lambda v: threshold_scad(v, 1.0, 3.7, 2.0)):
        assert np.all(np.diff(f(u)) >= -1e-15)
