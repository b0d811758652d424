"""The strips of a disk that label the stated-size parametric family (host code of
learned_m0, no GPU work): the glued contours close counter-clockwise, their
nodes are the oracle's piecewise rule on the same pieces, the widened areas
match the circle-segment formula, and the filter of each strip keeps every
point the strip owns inside (|rho| well above 1/2) and every point far outside
out."""
import math

import numpy as np
import pytest

from helpers import lib
from oracle import contour as ct

C, R = 0.3 + 0.0j, 0.5
CUTS = (-0.4, 0.0, 0.4)


def _strips(delta=0.04, K=12):
    lib()
    from paper_1404_2891_gb300 import learned_m0 as lm
    return lm, lm.disk_strips(C, R, CUTS, delta, K=K)


def _seg_end(sg, t):
    return complex(ct.segment_point(sg, t))


def test_pieces_close_counter_clockwise():
    _, strips = _strips()
    assert len(strips) == len(CUTS) + 1
    for s in strips:
        segs = s["segments"]
        for a, b in zip(segs, segs[1:] + segs[:1]):
            assert abs(_seg_end(a, 1.0) - _seg_end(b, 0.0)) < 1e-14
        assert s["area"] > 0


def test_nodes_are_the_oracle_rule_on_the_pieces():
    _, strips = _strips(K=12)
    for s in strips:
        zr, wr = ct.piecewise_quadrature(s["segments"], 12, "gauss")
        con = s["contour"]
        assert con.q_custom == len(s["segments"]) * 12
        z = np.array([complex(con.nodes[k].re, con.nodes[k].im) for k in range(con.q_custom)])
        w = np.array([complex(con.weights[k].re, con.weights[k].im) for k in range(con.q_custom)])
        assert np.allclose(z, zr, atol=1e-15, rtol=0) and np.allclose(w, wr, atol=1e-15, rtol=0)


def _segment_area(R2, d):
    """Area of the part of the disk of radius R2 beyond a chord at distance d from
    its centre (d may be negative)."""
    return R2 * R2 * math.acos(d / R2) - d * math.sqrt(R2 * R2 - d * d)


def test_widened_areas_match_the_circle_segment_formula():
    delta = 0.04
    _, strips = _strips(delta=delta)
    R2 = R + delta
    x = [R * t for t in CUTS]  # cut abscissae relative to the centre
    full = math.pi * R2 * R2
    want = [_segment_area(R2, -(x[0] + delta)),
            full - _segment_area(R2, x[1] + delta) - _segment_area(R2, -(x[0] - delta)),
            full - _segment_area(R2, x[2] + delta) - _segment_area(R2, -(x[1] - delta)),
            _segment_area(R2, x[2] - delta)]
    got = [s["area"] for s in strips]
    assert np.allclose(got, want, rtol=1e-4, atol=0), (got, want)


def test_each_point_of_the_disk_has_one_owner_and_passes_its_filter():
    delta = 0.04
    _, strips = _strips(delta=delta)
    rng = np.random.default_rng(3)
    pts = C + R * np.sqrt(rng.uniform(0, 1, 4000)) * np.exp(2j * np.pi * rng.uniform(0, 1, 4000))
    owners = np.zeros(len(pts), dtype=int)
    for s in strips:
        own = (pts.real >= s["lo"]) & (pts.real < s["hi"])
        owners += own
        z, w = ct.piecewise_quadrature(s["segments"], 12, "gauss")
        r_own = np.abs(ct.rho(pts[own], z, w))
        assert r_own.min() > 0.7, r_own.min()
        # points 3 delta beyond the widened domain are filtered out
        far = C + 1.3 * np.sqrt(rng.uniform(0, 1, 4000)) * np.exp(2j * np.pi * rng.uniform(0, 1, 4000))
        keep = (far.real > s["lo"] - 4 * delta) & (far.real < s["hi"] + 4 * delta) & (np.abs(far - C) < R + 4 * delta)
        assert np.abs(ct.rho(far[~keep], z, w)).max() < 0.5
    assert np.all(owners == 1)


def test_strip_subspace_sizes():
    lm, strips = _strips()
    m0 = lm.strip_m0(strips, 1024 / math.pi)
    assert all(m % 8 == 0 and m <= 160 for m in m0)
    for m, s in zip(m0, strips):
        assert m >= 1.3 * s["area"] * 1024 / math.pi + 8
    assert lm.strip_m0(strips, 1e6) == [160] * len(strips)


def test_strips_reject_bad_cuts_and_bands():
    lm, _ = _strips()
    for cuts, delta in [((-1.0, 0.0), 0.04), ((0.2, 0.2), 0.04), ((0.0, 1.3), 0.04), ((0.0,), 0.0),
                        ((0.0,), -0.1)]:
        with pytest.raises(ValueError):
            lm.disk_strips(C, R, cuts, delta)
    whole = lm.disk_strips(C, R, (), 0.04)  # no cut: the whole widened disk
    assert len(whole) == 1 and abs(whole[0]["area"] - math.pi * (R + 0.04) ** 2) < 1e-4
