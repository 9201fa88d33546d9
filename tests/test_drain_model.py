"""Performance model of the cell-list pair kernel's hit evaluation (host side, no GPU).

A warp evaluates one pair per lane and iteration, so its cost is the number of iterations:
at each evaluation point, the largest number of hits any lane has to take. The model
rebuilds, for sampled warp groups of a 262,144-particle box at the 1M workload's density,
cells and group limits, the candidate stream the kernel stages:
- the trimmed stencil row runs in the kernel's order;
- each lane's hits from the bit-exact half-precision pre-test.
It counts the iterations of three evaluation schedules:
- per chunk: every 32-candidate chunk evaluated before the next is staged;
- per window: four chunks staged, then evaluated together;
- the kernel's lazy drain: a ring of four chunks, where the oldest position is drained just
  enough before it is restaged, so that lanes light on one chunk work ahead on the next.
The lazy drain must need the fewest iterations and the per-chunk schedule the most.
"""
import math

import numpy as np

from paper_2609_02694_gb300 import synth

from test_half_pretest_model import THRESHOLD, half_r2
from test_trim_model import M32, _cells, _i32

K_WIN = 4


def group_streams(s, box, rc=10.0, sub=2, smax=10, n_warps=120, seed=0, width=32,
                  trim=True):
    """Yield (member rows of S, ordered candidate rows of S, S, leader coordinates) for the
    groups of n_warps random warps, with the kernel's rows, segments and trimming. Groups form
    within windows of `width` lanes (32: the kernel; 16: half-warp groups, a design option);
    trim=False keeps whole runs (the kernel's charged-subset Coulomb pass)."""
    n = [int(math.floor(box[d] * sub / rc)) for d in range(3)]
    a = [box[d] / n[d] for d in range(3)]
    R = [int(math.ceil(rc / a[d])) for d in range(3)]
    order, (cx, cy, cz), cs = _cells(s, n)
    S = s[order].astype(np.int64)
    N = len(S)
    hd = [box[d] / M32 for d in range(3)]
    ny, nrows = 2 * R[1] + 1, (2 * R[1] + 1) * (2 * R[2] + 1)
    rng = np.random.default_rng(seed)
    for w in rng.choice(N // 32, n_warps, replace=False):
        for h0 in range(32 * w, 32 * w + 32, width):
            remaining = list(range(h0, h0 + width))
            while remaining:
                ld = remaining[0]
                gy, gz, gx0 = cy[ld], cz[ld], cx[ld]
                ins = [l for l in remaining
                       if cy[l] == gy and cz[l] == gz and cx[l] - gx0 < smax]
                remaining = [l for l in remaining if l not in ins]
                cxlo, cxhi = min(cx[l] for l in ins), max(cx[l] for l in ins)
                o = [int(v) for v in S[ld]]
                fr = [[_i32(int(S[l, d]) - o[d]) for l in ins] for d in range(3)]
                gxlo, gxhi = min(fr[0]), max(fr[0])
                gylo, gyhi, gzlo, gzhi = min(fr[1]), max(fr[1]), min(fr[2]), max(fr[2])
                span = cxhi - cxlo + 2 * R[0] + 1
                runs = []
                for r in range(nrows):
                    dz, dy = r // ny - R[2], r % ny - R[1]
                    rowbase = n[0] * ((gy + dy) % n[1] + n[1] * ((gz + dz) % n[2]))
                    if span >= n[0]:
                        segs = [(0, n[0] - 1, 0)]
                    else:
                        lo, hi = cxlo - R[0], cxhi + R[0]
                        if lo < 0:
                            segs = [(lo + n[0], n[0] - 1, -M32), (0, hi, 0)]
                        elif hi >= n[0]:
                            segs = [(lo, n[0] - 1, 0), (0, hi - n[0], M32)]
                        else:
                            segs = [(lo, hi, 0)]
                    wy, wz = M32 / n[1], M32 / n[2]
                    ylo, yhi = (gy + dy) * wy - o[1] - 2.0, (gy + dy + 1) * wy - o[1] + 2.0
                    zlo, zhi = (gz + dz) * wz - o[2] - 2.0, (gz + dz + 1) * wz - o[2] + 2.0
                    ddy = max(0.0, ylo - gyhi, gylo - yhi)
                    ddz = max(0.0, zlo - gzhi, gzlo - zhi)
                    rx2 = rc * rc * (1 + 1e-9) - (ddy * hd[1]) ** 2 - (ddz * hd[2]) ** 2
                    for c0, c1, sh in segs:
                        b = int(cs[rowbase + c0])
                        ln = int(cs[rowbase + c1 + 1]) - b
                        if trim and span < n[0]:
                            if rx2 <= 0:
                                continue
                            rx = int(math.ceil(math.sqrt(rx2) / hd[0]) + 2.0)
                            xs = S[b:b + ln, 0] + sh - o[0]  # sorted: the unwrapped coordinate
                            u = int(np.searchsorted(xs, gxlo - rx, side="left"))
                            v = int(np.searchsorted(xs, gxhi + rx + 1, side="left"))
                            b, ln = b + u, v - u
                        runs.append(np.arange(b, b + ln))
                yield ins, np.concatenate(runs) if runs else np.zeros(0, np.int64), S, o


def lane_hits(ins, cand, S, o, L, rc):
    """(members x candidates) pre-test hits, each lane against every staged candidate."""
    fi = ((S[ins] - np.asarray(o) + 2 ** 31) % M32 - 2 ** 31)
    fj = ((S[cand] - np.asarray(o) + 2 ** 31) % M32 - 2 ** 31)
    m, T = len(ins), len(cand)
    t = half_r2(np.repeat(fi, T, axis=0), np.tile(fj, (m, 1)), L, rc)
    return (t.astype(np.float64) < THRESHOLD).reshape(m, T)


def trip_counts(hits):
    """Iterations of the three schedules for one group's hit matrix (lanes x candidates)."""
    T = hits.shape[1]
    nch = (T + 31) // 32
    pc = np.stack([hits[:, 32 * c:32 * c + 32].sum(1) for c in range(nch)], 1) if nch else \
        np.zeros((hits.shape[0], 0), np.int64)
    per_chunk = int(pc.max(0).sum()) if nch else 0
    window = sum(int(pc[:, w:w + K_WIN].sum(1).max()) for w in range(0, nch, K_WIN))
    cnt = np.zeros(hits.shape[0], np.int64)
    q = np.zeros((hits.shape[0], K_WIN), np.int64)
    lazy = 0
    for ch in range(nch + 1):
        p = ch % K_WIN
        if ch >= K_WIN or ch == nch:
            need = cnt if ch == nch else np.maximum(0, cnt - (q.sum(1) - q[:, p]))
            nit = int(need.max()) if len(need) else 0
            lazy += nit
            cnt = np.maximum(0, cnt - nit)
        if ch == nch:
            break
        q[:, p] = pc[:, ch]
        cnt += pc[:, ch]
    return per_chunk, window, lazy


def test_lazy_drain_needs_fewest_iterations():
    sy = synth.make_system(1 << 18, density=0.1, frac_charged=0.1, seed=2)  # L = 137.9
    L = float(sy.box[0])
    tot = np.zeros(3)
    hits_per_lane, groups = [], 0
    for ins, cand, S, o in group_streams(sy.s, sy.box):
        h = lane_hits(ins, cand, S, o, L, 10.0)
        tot += trip_counts(h)
        hits_per_lane.extend(h.sum(1))
        groups += 1
    per_chunk, window, lazy = tot / groups
    assert groups > 100 and 300 < np.mean(hits_per_lane) < 600
    assert lazy < 0.85 * window and window < 0.85 * per_chunk, (per_chunk, window, lazy)
