"""Model of the cell-list pair kernel's hit-mask queue protocol (host side, no GPU).

The kernel stages candidates in a ring of four 32-candidate chunks. Each lane queues a
chunk's 32-bit hit mask, with its ring position, when the mask is not empty. Before a
chunk overwrites a ring position, the warp evaluates just enough iterations that no lane
has a hit pending there; each iteration takes the highest set bit of the lane's current
mask, or the next queued mask when that one is spent. This model runs the same integer
protocol: pending counts packed per ring position, a queue of kHitQ entries, and the
current mask. It uses adversarial hit patterns and checks four things:
- no queued mask is overwritten;
- no hit is read after its ring slot was restaged;
- nothing is pending at a position about to be restaged;
- every lane evaluates exactly its own hits, chunk by chunk, the highest candidate first.
The GPU parity tests check the kernel itself against the oracle.
"""
import numpy as np
import pytest

K_WIN = 4  # ring positions (chunks of 32 candidates)


def _field(q4, p):
    """Hits pending at ring position p (8-bit field p of the packed counts)."""
    return (q4 >> (8 * p)) & 0xFF


def run_protocol(h, qcap):
    """Run the kernel's protocol for one warp. h[l, c] says whether candidate c is a hit of
    lane l; qcap is the number of queue entries per lane. Asserts the four properties."""
    T = h.shape[1]
    nch = (T + 31) // 32
    queue = [[None] * qcap for _ in range(32)]  # entries (mask, ring slot base, chunk)
    hd = [0] * 32    # queue read count
    tl = [0] * 32    # queue write count
    cnt = [0] * 32   # hits pending
    q4 = [0] * 32    # hits per ring position, packed
    cm = [0] * 32    # mask being consumed
    cp = [0] * 32    # its ring slot base
    cch = [-1] * 32  # its chunk
    ring = [None] * K_WIN  # chunk staged at each ring position
    done = [[] for _ in range(32)]  # candidates evaluated, in order
    for ch in range(nch + 1):
        p = ch % K_WIN
        if ch >= K_WIN or ch == nch:
            # drain: enough iterations that no lane keeps a hit at position p
            need = []
            for l in range(32):
                nd = cnt[l]
                if ch < nch:
                    newer = sum(_field(q4[l], b) for b in range(K_WIN)) - _field(q4[l], p)
                    nd = max(0, cnt[l] - newer)
                need.append(nd)
            nit = max(need)
            pending = list(cnt)
            for k in range(nit):
                for l in range(32):
                    if k >= pending[l]:
                        continue
                    if cm[l] == 0:
                        e = queue[l][hd[l] % qcap]
                        assert e is not None, "empty entry"
                        queue[l][hd[l] % qcap] = None
                        cm[l], cp[l], cch[l] = e
                        hd[l] += 1
                    assert cm[l] != 0
                    b = cm[l].bit_length() - 1  # highest pending candidate first
                    assert ring[cp[l] // 32] == cch[l], "ring slot restaged before use"
                    done[l].append(cch[l] * 32 + b)
                    cm[l] &= ~(1 << b)
            for l in range(32):
                cnt[l] = max(0, cnt[l] - nit)
            if ch < nch:
                for l in range(32):
                    assert not (cm[l] and cp[l] // 32 == p), "current mask at p"
                    assert all(e is None or e[1] // 32 != p for e in queue[l]), "queued mask at p"
        if ch == nch:
            break
        # stage chunk ch at position p, test it and queue each lane's non-empty mask
        ring[p] = ch
        for l in range(32):
            mk = 0
            for t in range(32):
                c = ch * 32 + t
                if c < T and h[l, c]:
                    mk |= 1 << t
            if mk:
                assert queue[l][tl[l] % qcap] is None, "queue overflow"
                queue[l][tl[l] % qcap] = (mk, p * 32, ch)
                tl[l] += 1
            nh = bin(mk).count("1")
            cnt[l] += nh
            q4[l] = (q4[l] & ~(0xFF << (8 * p))) | (nh << (8 * p))
    for l in range(32):
        want = [j for c0 in range(0, T, 32)
                for j in sorted(np.nonzero(h[l, c0:c0 + 32])[0] + c0, reverse=True)]
        assert done[l] == want
        assert cnt[l] == 0 and cm[l] == 0

def _patterns(rng, n):
    for trial in range(n):
        T = int(rng.integers(0, 40 * 32))
        kind = trial % 5
        if kind == 0:
            yield rng.random((32, T)) < rng.random()
        elif kind == 1:
            yield np.ones((32, T), bool)  # every candidate a hit (cells of r_c)
        elif kind == 2:
            h = np.zeros((32, T), bool)  # one contiguous stretch per lane
            for l in range(32):
                a = int(rng.integers(0, max(1, T)))
                h[l, a:int(rng.integers(a, T + 1))] = True
            yield h
        elif kind == 3:
            yield rng.random((32, T)) < rng.random((32, 1))
        else:
            h = np.zeros((32, T), bool)  # one saturated lane, the others empty
            h[0] = True
            yield h


def test_hit_queue_protocol():
    """The kernel's queue of four entries suffices."""
    for h in _patterns(np.random.default_rng(1), 300):
        run_protocol(h, 4)


def test_hit_queue_model_rejects_a_short_queue():
    """Three entries are too few (the model must catch the overflow)."""
    with pytest.raises(AssertionError):
        for h in _patterns(np.random.default_rng(1), 300):
            run_protocol(h, 3)
