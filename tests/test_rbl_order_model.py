"""Model of the random-batch-list kernel's shell enumeration (host side, no GPU).

The draws index each particle's shell in its canonical order: the 27 neighbour cells in
(dz, dy, dx) order, each -1..1, and inside a cell ascending (s_x, id). The kernel produces
that order in these steps:
- A warp splits into groups: lanes in one cell row whose x cells lie within gs cells of the
  leader's.
- For each of the nine rows (dz, dy), the group walks one run of x cells, gx - 1 .. gx + gs
  (mod n_x). The run is split at the box edge into at most two parts, the left part first.
- Every candidate carries its offset in the run. A lane keeps the candidates of its own
  three x cells (offsets lo .. lo + 2), or all of them when gs = 1.
- The exact decision sorts them into core and shell.

This model repeats those steps on the oracle's cells. It checks that every particle's core
count and shell list, in order, equal the canonical enumeration, in three layouts:
- a box of three cells of r_s per axis (the wrapping variant, gs = 1);
- a dilute box with multi-cell groups;
- a wrapping box with multi-cell groups.
A run whose two parts are taken in the wrong order must fail it. The GPU parity tests
compare the kernel's draws with the oracle's.
"""
import math

import numpy as np

from paper_2609_02694_gb300 import synth

TWO32 = 4294967296.0
K_MAX_SPAN = 14  # the kernel's largest group span


def _shape(N, box, n, r_s, span=0):
    """Group span and wrapping flag, by the library's rule: gs = floor(32 / particles per
    cell), within [1, min(14, n_x - 2)], reduced until a group's frame is a valid minimum
    image unless the box wraps."""
    gs = span if span > 0 else max(1, int(math.floor(32.0 / (N / np.prod(n)))))
    gs = max(1, min(gs, K_MAX_SPAN, n[0] - 2))
    wrap = any(not (box[d] / n[d] + r_s < 0.5 * box[d] * (1 - 1e-9)) for d in range(3))
    if not wrap:
        while gs > 1 and not (gs * box[0] / n[0] + r_s < 0.5 * box[0] * (1 - 1e-9)):
            gs -= 1
    return gs, wrap


def _r2(s, i, js, box):
    """The exact decision's r^2: int32 differences times L / 2^32, squared and summed."""
    d = ((s[i].astype(np.int64) - s[js].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31)
    d = d * (np.asarray(box) / TWO32)
    return (d * d).sum(1)


def _classify(s, i, js, box, r_core, r_s):
    js = js[js != i]
    r2 = _r2(s, i, js, box)
    return int((r2 <= r_core * r_core).sum()), js[(r2 > r_core * r_core) & (r2 <= r_s * r_s)]


def canonical(orc, s, box, n, r_core, r_s):
    """Core counts and shell lists in the canonical order, from the oracle's cells."""
    cell_of, start, ids = orc.cells(s, n, within="x")
    N = len(s)
    core = np.zeros(N, np.int64)
    shell = []
    for i in range(N):
        c = int(cell_of[i])
        c3 = (c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1]))
        js = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    cc = ((c3[0] + dx) % n[0], (c3[1] + dy) % n[1], (c3[2] + dz) % n[2])
                    cj = cc[0] + n[0] * (cc[1] + n[1] * cc[2])
                    js.append(ids[start[cj]:start[cj + 1]])
        core[i], sh = _classify(s, i, np.concatenate(js), box, r_core, r_s)
        shell.append(sh)
    return core, shell


def kernel_order(orc, s, box, n, r_core, r_s, gs, swap_parts=False):
    """Core counts and shell lists as the kernel's groups, runs and offset filters give them."""
    cell_of, start, ids = orc.cells(s, n, within="x")
    N = len(s)
    cx = cell_of[ids] % n[0]
    cy = (cell_of[ids] // n[0]) % n[1]
    cz = cell_of[ids] // (n[0] * n[1])
    core = np.zeros(N, np.int64)
    shell = [None] * N
    for w0 in range(0, N, 32):
        remaining = list(range(w0, min(N, w0 + 32)))
        while remaining:
            ld = remaining[0]
            gx, gy, gz = cx[ld], cy[ld], cz[ld]
            members = [l for l in remaining
                       if cy[l] == gy and cz[l] == gz and 0 <= cx[l] - gx < gs]
            remaining = [l for l in remaining if l not in members]
            run, off = [], []
            for r in range(9):
                dz, dy = r // 3 - 1, r % 3 - 1
                rowbase = n[0] * ((gy + dy) % n[1] + n[1] * ((gz + dz) % n[2]))
                xlo, xhi = gx - 1, gx + gs
                if xlo < 0:
                    parts = [(n[0] - 1, n[0] - 1), (0, xhi)]
                elif xhi >= n[0]:
                    parts = [(xlo, n[0] - 1), (0, xhi - n[0])]
                else:
                    parts = [(xlo, xhi)]
                if swap_parts:
                    parts = parts[::-1]
                for c0, c1 in parts:
                    seg = ids[start[rowbase + c0]:start[rowbase + c1 + 1]]
                    run.append(seg)
                    # offset of each candidate's x cell in the run gx - 1 .. gx + gs (mod n_x)
                    off.append((cell_of[seg] % n[0] - gx + 1) % n[0])
            run = np.concatenate(run)
            off = np.concatenate(off)
            for l in members:
                i = int(ids[l])
                lo = cx[l] - gx
                keep = run if gs == 1 else run[(off >= lo) & (off <= lo + 2)]
                core[i], shell[i] = _classify(s, i, keep, box, r_core, r_s)
    return core, shell


def _compare(orc, s, box, r_core, r_s, span=0, swap_parts=False):
    n = [int(math.floor(box[d] / r_s)) for d in range(3)]
    gs, wrap = _shape(len(s), box, n, r_s, span)
    c0, s0 = canonical(orc, s, box, n, r_core, r_s)
    c1, s1 = kernel_order(orc, s, box, n, r_core, r_s, gs, swap_parts)
    same = np.array_equal(c0, c1) and all(np.array_equal(a, b) for a, b in zip(s0, s1))
    return same, gs, wrap, sum(len(x) for x in s0)


def test_wrapping_box_three_cells(orc):
    sy = synth.make_system(2000, density=0.1, frac_charged=0.1, seed=3)  # L = 27.1, r_s = 8
    same, gs, wrap, nshell = _compare(orc, sy.s, sy.box, 4.0, 8.0)
    assert wrap and gs == 1 and nshell > 2000 * 100
    assert same


def test_dilute_box_multi_cell_groups(orc):
    sy = synth.make_system(3000, density=0.01, frac_charged=0.1, seed=4)  # L = 66.9, r_s = 6
    for span in (0, 2, 3):
        same, gs, wrap, nshell = _compare(orc, sy.s, sy.box, 3.0, 6.0, span)
        assert not wrap and gs > 1 and nshell > 0
        assert same, span


def test_wrapping_box_multi_cell_groups(orc):
    """Three cells of r_s in y and z force the wrapping variant, while x holds ten cells and
    the system is dilute enough for groups of several cells."""
    # 5 a cell (gs = 6); a jitter of nearly half the lattice spacing spreads the x planes
    sy = synth.make_system(450, L=40.0, frac_charged=0.1, seed=5, jitter=2.4)
    box = np.array([60.0, 18.0, 18.0])  # the same fractional positions in another box
    same, gs, wrap, nshell = _compare(orc, sy.s, box, 3.0, 6.0)
    assert wrap and gs > 1 and nshell > 0
    assert same


def test_model_sees_parts_out_of_order(orc):
    """Planted mistake: taking the run's part across the box edge after the other part
    breaks the canonical order of the particles at the edge."""
    sy = synth.make_system(2000, density=0.1, frac_charged=0.1, seed=3)
    same, _, _, _ = _compare(orc, sy.s, sy.box, 4.0, 8.0, swap_parts=True)
    assert not same
