"""Model of the cell-list pair kernel's half-precision candidate pre-test (host side, no GPU).

The kernel first tests candidates in FP16x2. Each coordinate is the exact integer frame
offset from the group leader, converted to FP32 and scaled by L / 2^32 (two FP32 roundings).
It is then scaled by 8 / r_c in FP32 and rounded to half. Per pair it computes
r^2 = fma(dx, dx, fma(dy, dy, dz * dz)) in half, after half subtractions, each operation
rounded once to nearest. A candidate passes when that r^2 is below 66.5, where a neighbour
at the cutoff is at 64.

Groups keep every staged frame coordinate below 8 r_c, i.e. below 64 after scaling. The
rounding analysis then bounds the half r^2 above the exact scaled r^2 by about one unit. So
no pair within r_c can fail the test, and the exact decision that follows sees every
neighbour. This model repeats the arithmetic bit for bit on pairs near the cutoff, spread
over the whole coordinate range. It checks three things:
- every neighbour passes;
- the excess stays within the bound of 1.06;
- without the margin (a threshold of 64), neighbours are lost.
"""
import numpy as np

TWO32 = 4294967296.0
THRESHOLD = 66.5


def _round_half(s, e):
    """Round the exact value s + e to half, to nearest even. s is the float64 sum and e its
    exact error (TwoSum). Where s sits exactly halfway between two halves, e decides."""
    r = s.astype(np.float16)
    up = np.nextafter(r, np.float16(np.inf))
    dn = np.nextafter(r, np.float16(-np.inf))
    rd = r.astype(np.float64)
    tie_up = (s == (rd + up.astype(np.float64)) / 2) & (e > 0)
    tie_dn = (s == (rd + dn.astype(np.float64)) / 2) & (e < 0)
    return np.where(tie_up, up, np.where(tie_dn, dn, r))


def _fma_half(a, b, c):
    """fma(a, b, c) in half, rounded once: a * b is exact in float64, the sum is exact as
    float64 sum plus TwoSum error."""
    p = a.astype(np.float64) * b.astype(np.float64)
    cd = c.astype(np.float64)
    s = p + cd
    bb = s - p
    e = (p - (s - bb)) + (cd - bb)
    return _round_half(s, e)


def _coord_half(d, h32, scale32):
    """Half test coordinate of an integer frame offset: FP32 conversion, FP32 products,
    conversion to half (all round to nearest)."""
    x = d.astype(np.float32) * h32
    return (x * scale32).astype(np.float16)


def half_r2(di, dj, L, rc):
    """The kernel's half r^2 for frame offsets di, dj (n x 3 int64, one axis per column)."""
    h32 = np.float32(L / TWO32)
    scale32 = np.float32(8.0 / rc)
    comp = []
    for k in range(3):
        a = _coord_half(di[:, k], h32, scale32)
        b = _coord_half(dj[:, k], h32, scale32)
        # the difference of two halves of these magnitudes is exact in float64
        comp.append(_round_half(a.astype(np.float64) - b.astype(np.float64), 0.0))
    dx, dy, dz = comp
    zz = _fma_half(dz, dz, np.zeros_like(dz))
    return _fma_half(dx, dx, _fma_half(dy, dy, zz))


def _pairs(rng, n, L, rc, span):
    """n pairs of integer frame offsets with both ends inside [-span, span] (Angstrom) and
    exact distance within r_c, most of them in the last percent below it."""
    hd = L / TWO32
    lim = int(span / hd)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = rc * np.where(rng.random(n) < 0.8, 1.0 - 0.01 * rng.random(n), rng.random(n) ** (1 / 3))
    d = np.round(v * (r / hd)[:, None]).astype(np.int64)
    di = rng.integers(-lim, lim + 1, size=(n, 3))
    dj = di - d
    keep = (np.abs(dj) <= lim).all(1)
    di, dj = di[keep], dj[keep]
    dd = (di - dj) * hd  # the oracle's displacement: integer difference times L / 2^32
    r2 = (dd * dd).sum(1)
    inside = r2 <= rc * rc
    return di[inside], dj[inside], r2[inside]


def _check(L, rc, n=400000, seed=0):
    rng = np.random.default_rng(seed)
    # frame offsets up to 8 r_c (the groups' bound), slightly inside it
    di, dj, r2 = _pairs(rng, n, L, rc, 8.0 * rc * (1 - 1e-6))
    t = half_r2(di, dj, L, rc).astype(np.float64)
    excess = t - 64.0 * r2 / (rc * rc)
    return t, excess


def test_half_pretest_keeps_every_neighbour():
    for L, rc in ((218.877, 10.0), (218.877, 11.0), (551.535, 10.0), (86.861, 10.0)):
        t, excess = _check(L, rc)
        assert len(t) > 300000
        assert (t < THRESHOLD).all(), (L, rc, t.max())
        assert excess.max() <= 1.06, (L, rc, excess.max())


def test_half_pretest_without_margin_loses_neighbours():
    """Planted mistake: a threshold of 64 (the exact cutoff, no room for rounding) must
    reject some pairs within r_c, or the model could not see a missing margin."""
    t, _ = _check(218.877, 10.0)
    assert (t >= 64.0).any()


def _exact_half(x):
    """Round a rational to half, to nearest even, by exact comparison."""
    from fractions import Fraction
    r = np.float16(float(x))
    cands = [np.nextafter(r, np.float16(-np.inf)), r, np.nextafter(r, np.float16(np.inf))]
    best = None
    for c in cands:
        dist = abs(Fraction(float(c)) - x)
        key = (dist, int(c.view(np.uint16)) & 1)  # ties: the even significand
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


def test_half_emulation_rounds_exactly():
    """The emulated fma and subtraction equal exact rational arithmetic rounded once,
    on random halves of the model's magnitudes and on constructed ties."""
    from fractions import Fraction
    rng = np.random.default_rng(3)
    n = 3000
    a = (rng.uniform(-16, 16, n)).astype(np.float16)
    b = (rng.uniform(-16, 16, n)).astype(np.float16)
    c = (rng.uniform(0, 128, n) * rng.choice([1.0, 1e-3, 1e-6], n)).astype(np.float16)
    # ties: 3/32 * 683 = 64.03125, halfway between the halves 64 and 64.0625; with c = 0 it
    # rounds to even (64), with the smallest subnormal it rounds up
    a = np.r_[a, np.float16(0.09375), np.float16(0.09375)]
    b = np.r_[b, np.float16(683.0), np.float16(683.0)]
    c = np.r_[c, np.float16(0.0), np.float16(2.0 ** -24)]
    got = _fma_half(a, b, c)
    for k in range(len(a)):
        want = _exact_half(Fraction(float(a[k])) * Fraction(float(b[k])) + Fraction(float(c[k])))
        assert got[k] == want, (a[k], b[k], c[k], got[k], want)
    assert got[-2] == np.float16(64.0) and got[-1] == np.float16(64.0625)
    d = _round_half(a.astype(np.float64) - b.astype(np.float64), 0.0)
    for k in range(0, len(a), 7):
        assert d[k] == _exact_half(Fraction(float(a[k])) - Fraction(float(b[k])))
