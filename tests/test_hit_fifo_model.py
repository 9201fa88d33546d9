"""Model of the cell-list pair kernel's per-lane hit FIFO protocol (host side, no GPU).

The kernel stages candidates in a ring of four 32-candidate chunks and appends each lane's
hits (ring slots) to a FIFO of 160 bytes. Before a chunk overwrites a ring position, the
warp evaluates just enough iterations that no lane has a hit pending there. This model
runs the same integer protocol: pending counts packed per ring position, the writer's wrap
at chunk starts, the reader's wrap point, and an explicit pending count. It uses
adversarial hit patterns and checks four things:
- indices stay in range;
- no append overwrites a pending entry;
- no entry is read after its ring slot was restaged;
- every lane evaluates exactly its own hits, in order.
The GPU parity tests check the kernel itself against the oracle.
"""
import numpy as np
import pytest

K_WIN, K_HITQ = 4, 160


def run_protocol(hitmat, explicit_count=True):
    """hitmat: 32 lanes x T candidates (bool). explicit_count=False derives "pending" from
    the read and write indices alone, the variant that confuses full with empty."""
    T = hitmat.shape[1]
    nch = (T + 31) // 32
    fifo = [[None] * K_HITQ for _ in range(32)]
    hd, tl = [0] * 32, [0] * 32
    wrap, cnt, q4 = [K_HITQ] * 32, [0] * 32, [0] * 32
    ring = [None] * K_WIN
    done = [[] for _ in range(32)]

    def pending(l):
        if explicit_count:
            return cnt[l]
        return tl[l] - hd[l] + (wrap[l] if hd[l] > tl[l] else 0)

    for ch in range(nch + 1):
        p = ch & (K_WIN - 1)
        if ch >= K_WIN or ch == nch:
            need = []
            for l in range(32):
                nd = pending(l)
                if ch < nch:
                    tot = sum((q4[l] >> (8 * b)) & 0xFF for b in range(4))
                    nd = max(0, nd - (tot - ((q4[l] >> (8 * p)) & 0xFF)))
                need.append(nd)
            nit = max(need)
            start = [pending(l) for l in range(32)]
            for k in range(nit):
                for l in range(32):
                    if k < start[l]:
                        assert 0 <= hd[l] < K_HITQ
                        e = fifo[l][hd[l]]
                        assert e is not None, "read of an empty entry"
                        pos, chunk, t = e
                        assert ring[pos] == chunk, "ring slot restaged before use"
                        done[l].append(chunk * 32 + t)
                        fifo[l][hd[l]] = None
                        hd[l] += 1
                    if hd[l] == wrap[l]:
                        hd[l] = 0
            for l in range(32):
                cnt[l] = max(0, cnt[l] - nit)
            if ch < nch:
                for l in range(32):
                    assert all(e is None or e[0] != p for e in fifo[l]), "hit pending at p"
        if ch == nch:
            break
        ring[p] = ch
        for l in range(32):
            if tl[l] >= K_HITQ - 32:
                empty = cnt[l] == 0 if explicit_count else hd[l] == tl[l]
                wrap[l] = K_HITQ if empty else tl[l]
                hd[l] = 0 if empty else hd[l]
                tl[l] = 0
            elif hd[l] <= tl[l]:
                wrap[l] = K_HITQ
            t0 = tl[l]
            for t in range(32):
                assert 0 <= tl[l] < K_HITQ
                old = fifo[l][tl[l]]
                # the branch-free append writes every candidate at the tail
                assert old is None or old[2] == -1, "append overwrites a pending hit"
                c = ch * 32 + t
                hit = c < T and bool(hitmat[l, c])
                fifo[l][tl[l]] = (p, ch, t if hit else -1)
                tl[l] += hit
            if tl[l] < K_HITQ and fifo[l][tl[l]] is not None and fifo[l][tl[l]][2] == -1:
                fifo[l][tl[l]] = None
            cnt[l] += tl[l] - t0
            q4[l] = (q4[l] & ~(0xFF << (8 * p))) | ((tl[l] - t0) << (8 * p))
    for l in range(32):
        assert done[l] == list(np.nonzero(hitmat[l])[0]), l
        assert cnt[l] == 0


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


def test_hit_fifo_protocol():
    for h in _patterns(np.random.default_rng(1), 300):
        run_protocol(h)


def test_hit_fifo_model_rejects_full_empty_confusion():
    with pytest.raises(AssertionError):
        for h in _patterns(np.random.default_rng(1), 300):
            run_protocol(h, explicit_count=False)
