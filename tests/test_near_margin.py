"""The near-set search decides most pairs in FP32 (leaf-relative positions) and falls back
to the FP64 test only inside an error-bounded band around the boundary.  This host test
replays that FP32 arithmetic in numpy float32 on random configurations, including pairs
placed within a few ulps of the boundary, and checks that every FP32 decision outside the
band agrees with the FP64 test |x_p - x_t| < c (rho_p + rho_t)."""
import numpy as np


def test_fp32_pretest_outside_the_band_agrees_with_fp64():
    rng = np.random.default_rng(3)
    m = 200000
    c = 2.0
    f32 = np.float32
    # molecule-scale coordinates, leaf centres nearby, patch radii 0.05 - 1 A
    xp = rng.uniform(-300, 300, (m, 3))
    leaf_c = xp + rng.uniform(-8, 8, (m, 3))
    rho_p = rng.uniform(0.05, 1.0, m)
    rho_t = rng.uniform(0.05, 1.0, m)
    R = c * (rho_p + rho_t)
    # sources: half random around the target, half on the boundary sphere (+/- 1e-9 rel)
    d = rng.standard_normal((m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    scale = np.where(rng.random(m) < 0.5, rng.uniform(0.2, 2.0, m), 1.0 + rng.uniform(-1e-9, 1e-9, m))
    xt = xp + d * (R * scale)[:, None]
    # FP64 decision (the defining test)
    exact = np.sqrt(((xp - xt) ** 2).sum(1)) < R
    # FP32 replay: target offset from the source leaf centre, leaf-relative source position
    o = (xp - leaf_c).astype(f32)
    q = (xt - leaf_c).astype(f32)
    dx = (o - q).astype(f32)
    fd2 = (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1] + dx[:, 2] * dx[:, 2]).astype(f32)
    fR = (f32(c) * rho_t.astype(f32) + (c * rho_p).astype(f32)).astype(f32)
    fR2 = (fR * fR).astype(f32)
    S = (np.abs(o).sum(1) + np.abs(q).sum(1)).astype(f32)
    margin = (f32(1e-6) * fR * S + f32(1e-5) * fR2).astype(f32)
    surely_in = fd2 < fR2 - margin
    surely_out = fd2 > fR2 + margin
    assert not np.any(surely_in & ~exact)
    assert not np.any(surely_out & exact)
    band = ~(surely_in | surely_out)
    # the band is narrow: the boundary-placed pairs land in it, almost no other pair does
    on_boundary = np.abs(scale - 1) < 1e-8
    assert band[on_boundary].mean() > 0.99
    assert band[np.abs(scale - 1) > 1e-3].mean() < 1e-3
