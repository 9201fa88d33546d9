"""Host model of the cluster kernel's reaction reduce-scatter (no GPU).

Per visit, the 8 lanes a = 0..7 that share a j-particle pair hold six FP32 partial sums each
(fx, fy, fz of particle h, then of particle h + 4). The kernel reduce-scatters them: slots
(the six values, then two zeros) are exchanged with lane a xor m for m = 1, 2, 4, each lane
keeping the slot whose bit m matches its own and adding its partner's copy; lane a ends
with slot a summed over the 8 lanes. This model repeats those steps in FP32 and checks,
bit for bit, that each lane's result equals what a full butterfly (every lane summing every
slot with the same xor exchanges) leaves in that lane for that slot, the reduction the
kernel used before: the same additions in the same tree, with a third of the shuffles.
"""
import numpy as np

F32 = np.float32


def butterfly(v):
    """v: (8 lanes, 6 slots) FP32. All-reduce per slot by exchanges xor 1, 2, 4, each lane
    adding its partner's value to its own (own + partner)."""
    v = v.copy()
    for m in (1, 2, 4):
        partner = v[[a ^ m for a in range(8)]]
        v = (v + partner).astype(F32)
    return v


def reduce_scatter(v):
    """The kernel's steps: returns the value lane a adds (slot a, for a < 6)."""
    out = np.zeros(8, F32)
    zero = F32(0)
    # slot order: fx0, fy0, fz0, fx1, fy1, fz1, 0, 0; round xor 1 pairs (0,1), (2,3), (4,5)
    s0 = [[v[a, 0], v[a, 2], v[a, 4]] for a in range(8)]
    s1 = [[v[a, 1], v[a, 3], v[a, 5]] for a in range(8)]
    w = np.zeros((8, 3), F32)
    for a in range(8):
        b0 = a & 1
        p = a ^ 1
        for k in range(3):
            keep = s1[a][k] if b0 else s0[a][k]
            recv = s0[p][k] if (p & 1) else s1[p][k]  # the partner sends the other slot
            w[a, k] = F32(keep + recv)
    u = np.zeros((8, 2), F32)
    for a in range(8):
        b1 = (a >> 1) & 1
        p = a ^ 2
        pb1 = (p >> 1) & 1
        keep0 = w[a, 1] if b1 else w[a, 0]
        send0 = w[p, 0] if pb1 else w[p, 1]
        u[a, 0] = F32(keep0 + send0)
        keep1 = zero if b1 else w[a, 2]
        send1 = w[p, 2] if pb1 else zero
        u[a, 1] = F32(keep1 + send1)
    for a in range(8):
        b2 = (a >> 2) & 1
        p = a ^ 4
        pb2 = (p >> 2) & 1
        keep = u[a, 1] if b2 else u[a, 0]
        send = u[p, 0] if pb2 else u[p, 1]
        out[a] = F32(keep + send)
    return out


def test_reduce_scatter_equals_butterfly_bit_for_bit():
    rng = np.random.default_rng(11)
    for trial in range(3000):
        scale = 10.0 ** rng.uniform(-6, 6, size=(8, 6))
        v = (rng.standard_normal((8, 6)) * scale).astype(F32)
        if trial % 5 == 0:  # zeros and sign patterns of masked pairs
            v[rng.random((8, 6)) < 0.3] = F32(0)
        full = butterfly(v)
        rs = reduce_scatter(v)
        for a in range(6):
            assert rs[a].view(np.uint32) == full[a, a].view(np.uint32), (trial, a)
        assert rs[6] == 0 and rs[7] == 0  # the padding slots


def test_model_sums_each_slot_over_the_lanes():
    """Independent of the tree: with small integers (exact in FP32) every lane's slot is the
    plain sum over the 8 lanes, so a wrong slot or partner in the model would show."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        v = rng.integers(-1000, 1000, size=(8, 6)).astype(F32)
        rs = reduce_scatter(v)
        assert np.array_equal(rs[:6], v.sum(0).astype(F32))


def test_sentinels_stay_finite():
    """An empty j slot's y (-3e18) against an empty i slot's y (3e18): r^2 stays finite in
    FP32 (no inf - inf), so its 1/r^2 is an exact zero through the cutoff test."""
    dy = F32(3e18) - F32(-3e18)
    r2 = F32(dy * dy) + F32(F32(1e4) * 3)
    assert np.isfinite(r2) and r2 > F32(1e37)
