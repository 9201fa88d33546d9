"""Model of the error of an FP32 r^2 formed from FP32 frame coordinates (host side, no GPU).

The cell kernel's FP32 pre-test and the random-batch-list kernel's classification compare
such an r^2 with thresholds. Each coordinate is the integer offset from the group leader,
converted to FP32 and multiplied by the FP32 L / 2^32. The r^2 is
fma(dx, dx, fma(dy, dy, dz * dz)) after FP32 subtractions. The exact decision in FP64 takes
over inside a band around r^2. The library sizes that band from a bound on the error, given
the largest frame coordinate X_d a group can stage (the band is at least 1e-5):
    e_d = 4u X_d + 2u r (+ 2u L_d when the difference is folded into the box),
    |r^2_fp32 - r^2| / r^2 <= 2 |e| / r + |e|^2 / r^2 + 5u,   u = 2^-24.
This model repeats the kernels' FP32 arithmetic bit for bit and checks two things:
- the observed error stays within that bound at the group extents the library allows;
- a fixed 1e-5 band would be too narrow for a group spanning half of a large box.
"""
import numpy as np

TWO32 = 4294967296.0
U = 2.0 ** -24


def _round_f32(s, e):
    """Round the exact value s + e (s its float64 sum, e the exact error) to FP32, to
    nearest even."""
    r = s.astype(np.float32)
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(-np.inf))
    rd = r.astype(np.float64)
    tie_up = (s == (rd + up.astype(np.float64)) / 2) & (e > 0)
    tie_dn = (s == (rd + dn.astype(np.float64)) / 2) & (e < 0)
    return np.where(tie_up, up, np.where(tie_dn, dn, r))


def _fma_f32(a, b, c):
    """FP32 fma, rounded once (a * b is exact in float64; TwoSum gives the sum's error)."""
    p = a.astype(np.float64) * b.astype(np.float64)
    cd = c.astype(np.float64)
    s = p + cd
    bb = s - p
    e = (p - (s - bb)) + (cd - bb)
    return _round_f32(s, e)


def band_bound(X, r, L, wrap=False):
    """The bound the library's band is built from (before its factor 1.25 and floor)."""
    e = [4 * U * X[d] + 2 * U * r + (2 * U * L[d] if wrap else 0.0) for d in range(3)]
    s2 = sum(x * x for x in e)
    return 2 * np.sqrt(s2) / r + s2 / (r * r) + 5 * U


def observed_error(L, X, r, n=300000, seed=0):
    """Largest relative r^2 error over pairs at distance ~r with frame coordinates up to X."""
    rng = np.random.default_rng(seed)
    hd = L / TWO32
    h32 = np.float32(hd)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    rr = r * (1 + 0.002 * (rng.random(n) - 0.5))
    d = np.round(v * (rr / hd)[:, None]).astype(np.int64)
    lim = (np.asarray(X) / hd).astype(np.int64)
    di = np.stack([rng.integers(-lim[k], lim[k] + 1, n) for k in range(3)], 1)
    dj = di - d
    keep = (np.abs(dj) <= lim).all(1)
    di, dj = di[keep], dj[keep]
    xi = di.astype(np.float32) * h32  # FP32 conversion and product, round to nearest
    xj = dj.astype(np.float32) * h32
    dd = xi - xj                      # FP32 subtraction
    z2 = (dd[:, 2].astype(np.float64) ** 2).astype(np.float32)  # the exact square, rounded once
    r2 = _fma_f32(dd[:, 0], dd[:, 0], _fma_f32(dd[:, 1], dd[:, 1], z2)).astype(np.float64)
    ex = (di - dj) * hd
    return (np.abs(r2 - (ex * ex).sum(1)) / (r * r)).max()


CASES = [
    # (label, L, X per axis, r): the Coulomb pre-test of the 1,048,576- and 16,777,216-particle
    # boxes (cells of r_c / 2, R = 2, groups of up to 19 and 53 cells), the RBL core band of the
    # LJ electrolyte (cells of r_s = 8, groups of 5 and of the largest span, 14 cells)
    ("coulomb 1m", 218.877, (106.9, 15.3, 15.3), 10.0),
    ("coulomb 16m", 551.535, (275.8, 15.04, 15.04), 10.0),
    ("rbl core gs 5", 271.0, (49.3, 16.4, 16.4), 4.0),
    ("rbl core gs 14", 271.0, (123.2, 16.4, 16.4), 4.0),
    ("rbl shell gs 14", 271.0, (123.2, 16.4, 16.4), 8.0),
]


def test_frame_r2_error_within_band_bound():
    for label, L, X, r in CASES:
        obs = observed_error(L, X, r)
        assert obs <= band_bound(X, r, (L, L, L)), (label, obs)


def observed_error_corner(L, X, w, r, n=300000, seed=1):
    """As observed_error, with the cluster kernel's j coordinates: x converted from the
    particle's own integer offset, y and z as the FP32 frame coordinate of its cluster's box
    corner plus its FP32 offset from that corner (an integer within one cell width w),
    added in FP32."""
    rng = np.random.default_rng(seed)
    hd = L / TWO32
    h32 = np.float32(hd)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    rr = r * (1 + 0.002 * (rng.random(n) - 0.5))
    d = np.round(v * (rr / hd)[:, None]).astype(np.int64)
    lim = (np.asarray(X) / hd).astype(np.int64)
    di = np.stack([rng.integers(-lim[k], lim[k] + 1, n) for k in range(3)], 1)
    dj = di - d
    off = rng.integers(0, int(w / hd) + 1, size=(n, 3))
    off[:, 0] = 0
    corner = dj - off
    keep = (np.abs(dj) <= lim).all(1) & (np.abs(corner) <= lim).all(1)
    di, dj, off, corner = di[keep], dj[keep], off[keep], corner[keep]
    xi = di.astype(np.float32) * h32
    xj = dj.astype(np.float32) * h32
    yz = corner[:, 1:].astype(np.float32) * h32 + off[:, 1:].astype(np.float32) * h32
    xj[:, 1:] = yz                    # corner + offset, one more FP32 rounding
    dd = xi - xj
    z2 = (dd[:, 2].astype(np.float64) ** 2).astype(np.float32)
    r2 = _fma_f32(dd[:, 0], dd[:, 0], _fma_f32(dd[:, 1], dd[:, 1], z2)).astype(np.float64)
    ex = (di - dj) * hd
    return (np.abs(r2 - (ex * ex).sum(1)) / (r * r)).max()


def test_cluster_corner_offsets_within_widened_band():
    """The cluster kernel's band takes X = L/2 on every axis, raised by 2 r_c + 2 w in y and
    z for the corner-plus-offset j coordinates; the observed error stays within that bound,
    in the 1,048,576-particle box and in the tightest box the kernel takes (w + 2 r_c just
    below L)."""
    for L, w, r in ((218.877, 218.877 / 43, 10.0), (26.0, 5.2, 10.0), (551.535, 551.535 / 110, 10.0)):
        X = (L / 2, L / 2, L / 2)
        obs = observed_error_corner(L, X, w, r)
        Xb = (L / 2, L / 2 + 2 * r + 2 * w, L / 2 + 2 * r + 2 * w)
        assert obs <= band_bound(Xb, r, (L, L, L)), (L, obs)


def test_fixed_band_too_narrow_for_half_box_groups():
    """A group spanning half of a 1103 A box (the 2^27-particle system): the FP32 error
    exceeds a fixed 1e-5 band, so the band must follow the bound."""
    L, X, r = 1103.07, (551.5, 15.0, 15.0), 10.0
    obs = observed_error(L, X, r)
    assert obs > 1e-5
    assert obs <= band_bound(X, r, (L, L, L))


def test_f32_emulation_rounds_exactly():
    """The emulated FP32 fma equals exact rational arithmetic rounded once to nearest even,
    on random operands and a constructed tie."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    a = rng.uniform(-12, 12, 2000).astype(np.float32)
    b = rng.uniform(-12, 12, 2000).astype(np.float32)
    c = (rng.uniform(0, 200, 2000) * rng.choice([1.0, 1e-6, 1e-12], 2000)).astype(np.float32)
    # (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24, halfway between two FP32 values near 1; the
    # smallest positive c decides it upward
    t = np.float32(1 + 2 ** -12)
    a = np.r_[a, t, t]
    b = np.r_[b, t, t]
    c = np.r_[c, np.float32(0), np.float32(2 ** -60)]
    got = _fma_f32(a, b, c)
    for k in range(len(a)):
        x = Fraction(float(a[k])) * Fraction(float(b[k])) + Fraction(float(c[k]))
        r = np.float32(float(x))
        cands = [np.nextafter(r, np.float32(-np.inf)), r, np.nextafter(r, np.float32(np.inf))]
        want = min(cands, key=lambda v: (abs(Fraction(float(v)) - x),
                                         int(v.view(np.uint32)) & 1))
        assert got[k] == want, (a[k], b[k], c[k])
    assert got[-2] == np.float32(1 + 2 ** -11) and got[-1] > got[-2]


def test_library_band_is_the_bound():
    """The library's band (host code, no GPU) is 1.25 times this bound, never below 1e-5,
    and so covers the observed FP32 error at every extent above; invalid input is refused."""
    import pytest
    from paper_2609_02694_gb300 import binding, build
    build.build()
    for label, L, X, r in CASES + [("half box 134m", 1103.07, (551.5, 15.0, 15.0), 10.0)]:
        band = binding.decision_band(X, r, (L, L, L))
        assert band == pytest.approx(max(1e-5, 1.25 * band_bound(X, r, (L, L, L))), rel=1e-12)
        assert band >= observed_error(L, X, r, n=50000), label
    wrap = binding.decision_band((16.0, 16.0, 16.0), 10.0, (32.0, 32.0, 32.0), wrap=True)
    assert wrap == pytest.approx(max(1e-5, 1.25 * band_bound((16.0,) * 3, 10.0, (32.0,) * 3,
                                                            wrap=True)), rel=1e-12)
    assert binding.decision_band((0.0, 0.0, 0.0), 10.0, (100.0,) * 3) == 1e-5
    for bad in [((1.0, 1.0, 1.0), 0.0, (10.0,) * 3), ((-1.0, 1.0, 1.0), 1.0, (10.0,) * 3),
                ((1.0, 1.0, float("nan")), 1.0, (10.0,) * 3), ((1.0,) * 3, 1.0, (10.0, 0.0, 10.0))]:
        with pytest.raises(ValueError):
            binding.decision_band(*bad)
