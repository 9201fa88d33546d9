"""Model of the cell-list pair kernel's stencil-row trimming (host side, no GPU).

Cells keep their members in (s_x, id) order, so each stencil row's run of cells is
sorted by x. The kernel works per warp group (lanes sharing a cell row, within a bounded
x extent). It cuts every row's run to [x_lo - reach, x_hi + reach]:
- x_lo and x_hi span the members' frame coordinates;
- reach = sqrt(r^2 - d^2), with d the row's y/z distance from the group's box, plus
  integer margins;
- the binary searches run on exact unwrapped coordinates (s_x plus the segment's wrap
  shift), because the minimum-image frame coordinate is not monotone along a run that
  crosses the periodic boundary.
This model repeats that integer arithmetic on small periodic boxes (runs that wrap, cells
of r_c and r_c/2, a dilute subset). It checks that no pair within the radius is cut. The
random-batch-list kernel trims its nine rows of cells of r_s the same way; a second model
repeats its runs. The GPU parity tests compare the kernels' exact neighbour counts and
shell orders with the oracle.
"""
import math

import numpy as np

from paper_2609_02694_gb300 import synth

M32 = 1 << 32


def _i32(v):
    v &= 0xFFFFFFFF
    return v - M32 if v >= 1 << 31 else v


def _cells(s, n):
    """Cell of each particle on the fixed-point grid, members ordered by (cell, s_x, id)."""
    c3 = [(s[:, d].astype(np.uint64) * np.uint64(n[d]) >> np.uint64(32)).astype(np.int64)
          for d in range(3)]
    cell = c3[0] + n[0] * (c3[1] + n[1] * c3[2])
    order = np.lexsort((np.arange(len(s)), s[:, 0].astype(np.int64), cell))
    start = np.zeros(int(np.prod(n)) + 1, np.int64)
    np.add.at(start, cell + 1, 1)
    return order, [c[order] for c in c3], np.cumsum(start)


def _check(s, box, sub, radius, smax, r_c=10.0):
    """Every pair within `radius` of a group member must survive its group's trimming.
    Cells are r_c / sub wide (the binning's grid); the stencil reaches `radius` (r_c, or the
    Verlet-list radius r_c + skin)."""
    n = [int(math.floor(box[d] * sub / r_c)) for d in range(3)]
    a = [box[d] / n[d] for d in range(3)]
    R = [int(math.ceil(radius / a[d])) for d in range(3)]
    assert all(n[d] >= 2 * R[d] + 1 for d in range(3))
    order, (cx, cy, cz), cs = _cells(s, n)
    S = s[order].astype(np.int64)
    N = len(S)
    hd = [box[d] / M32 for d in range(3)]
    ny, nrows = 2 * R[1] + 1, (2 * R[1] + 1) * (2 * R[2] + 1)
    pairs = missed = 0
    for w0 in range(0, N, 32):
        remaining = list(range(w0, min(N, w0 + 32)))
        while remaining:
            ld = remaining[0]
            gy, gz, gx0 = cy[ld], cz[ld], cx[ld]
            ins = [l for l in remaining if cy[l] == gy and cz[l] == gz and cx[l] - gx0 < smax]
            remaining = [l for l in remaining if l not in ins]
            cxlo, cxhi = min(cx[l] for l in ins), max(cx[l] for l in ins)
            ox, oy, oz = (int(v) for v in S[ld])
            fr = [[_i32(int(S[l, d]) - o) for l in ins] for d, o in enumerate((ox, oy, oz))]
            gxlo, gxhi = min(fr[0]), max(fr[0])
            gylo, gyhi, gzlo, gzhi = min(fr[1]), max(fr[1]), min(fr[2]), max(fr[2])
            span = cxhi - cxlo + 2 * R[0] + 1
            cand = set()
            for r in range(nrows):
                dz, dy = r // ny - R[2], r % ny - R[1]
                rowbase = n[0] * ((gy + dy) % n[1] + n[1] * ((gz + dz) % n[2]))
                segs = []  # (first cell, last cell, unwrapping shift)
                if span >= n[0]:
                    segs.append((0, n[0] - 1, 0))
                else:
                    lo, hi = cxlo - R[0], cxhi + R[0]
                    if lo < 0:
                        segs += [(lo + n[0], n[0] - 1, -M32), (0, hi, 0)]
                    elif hi >= n[0]:
                        segs += [(lo, n[0] - 1, 0), (0, hi - n[0], M32)]
                    else:
                        segs.append((lo, hi, 0))
                wy, wz = M32 / n[1], M32 / n[2]
                ylo, yhi = (gy + dy) * wy - oy - 2.0, (gy + dy + 1) * wy - oy + 2.0
                zlo, zhi = (gz + dz) * wz - oz - 2.0, (gz + dz + 1) * wz - oz + 2.0
                ddy = max(0.0, ylo - gyhi, gylo - yhi) * hd[1]
                ddz = max(0.0, zlo - gzhi, gzlo - zhi) * hd[2]
                rx2 = radius * radius * (1 + 1e-9) - ddy * ddy - ddz * ddz
                for c0, c1, sh in segs:
                    b, ln = int(cs[rowbase + c0]), int(cs[rowbase + c1 + 1] - cs[rowbase + c0])
                    if span < n[0]:  # trimmed (the kernel's trim condition)
                        if rx2 <= 0:
                            continue
                        rx = int(math.ceil(math.sqrt(rx2) / hd[0]) + 2.0)

                        def first_ge(key):
                            lo_, hi_ = 0, ln
                            while lo_ < hi_:
                                mid = (lo_ + hi_) >> 1
                                if int(S[b + mid, 0]) + sh - ox < key:
                                    lo_ = mid + 1
                                else:
                                    hi_ = mid
                            return lo_

                        u, v = first_ge(gxlo - rx), first_ge(gxhi + rx + 1)
                        b, ln = b + u, v - u
                    cand.update(range(b, b + ln))
            for l in ins:
                d = (S - S[l] + 2 ** 31) % M32 - 2 ** 31
                r2 = ((d * np.asarray(hd)) ** 2).sum(1)
                nb = np.nonzero(r2 <= radius * radius)[0]
                pairs += len(nb)
                missed += sum(1 for j in nb if int(j) not in cand)
    return pairs, missed


def test_trim_keeps_every_neighbour_small_box():
    sy = synth.make_system(4000, density=0.1, frac_charged=0.1, seed=7)  # L = 34.2, runs wrap
    pairs, missed = _check(sy.s, sy.box, 2, 10.0, 1)
    assert pairs > 4000 * 300 and missed == 0


def test_trim_keeps_every_neighbour_rc_cells():
    sy = synth.make_system(5000, density=0.1, frac_charged=0.1, seed=8)
    pairs, missed = _check(sy.s, sy.box, 1, 10.0, 1)  # cells of r_c, R = 1
    assert pairs > 0 and missed == 0


def test_trim_keeps_every_neighbour_dilute_list_build():
    """The charged subset's Verlet-list build: cells of r_c / 2, stencil R = 3 for the list
    radius 11, groups of two cells. Runs then cover nearly a whole row, and candidates beyond
    L/2 of the leader wrap in the minimum-image frame."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=12)
    q = sy.q != 0
    pairs, missed = _check(sy.s[q], sy.box, 2, 11.0, 2)
    assert pairs > 0 and missed == 0


def _check_rbl(s, box, r_s, gs):
    """The RBL kernel's runs: cells of r_s (one cell of stencil), groups of lanes in one cell
    row within gs cells of the leader, each row's run the cells gx - 1 .. gx + gs as at most
    two parts, cut like the cell kernel's runs. Every pair within r_s must survive.

    The kernel trims only where gs * a + r_s < L/2 (a >= r_s the cell width), so a run never
    reaches L/2 from the leader and its frame coordinates stay monotone as well. What this
    model pins is the unwrap shift of the part across x = 0 or x = L: a dropped or
    sign-swapped shift cuts whole cells of neighbours on these boxes."""
    n = [int(math.floor(box[d] / r_s)) for d in range(3)]
    a = [box[d] / n[d] for d in range(3)]
    assert all(a[d] + r_s < 0.5 * box[d] for d in range(3)) and gs * a[0] + r_s < 0.5 * box[0]
    order, (cx, cy, cz), cs = _cells(s, n)
    S = s[order].astype(np.int64)
    N = len(S)
    hd = [box[d] / M32 for d in range(3)]
    pairs = missed = 0
    for w0 in range(0, N, 32):
        remaining = list(range(w0, min(N, w0 + 32)))
        while remaining:
            ld = remaining[0]
            gx, gy, gz = cx[ld], cy[ld], cz[ld]
            ins = [l for l in remaining
                   if cy[l] == gy and cz[l] == gz and 0 <= cx[l] - gx < gs]
            remaining = [l for l in remaining if l not in ins]
            ox, oy, oz = (int(v) for v in S[ld])
            fr = [[_i32(int(S[l, d]) - o) for l in ins] for d, o in enumerate((ox, oy, oz))]
            gxlo, gxhi = min(fr[0]), max(fr[0])
            gylo, gyhi, gzlo, gzhi = min(fr[1]), max(fr[1]), min(fr[2]), max(fr[2])
            cand = set()
            for r in range(9):
                dz, dy = r // 3 - 1, r % 3 - 1
                rowbase = n[0] * ((gy + dy) % n[1] + n[1] * ((gz + dz) % n[2]))
                xlo, xhi = gx - 1, gx + gs
                for part in (0, 1):
                    if xlo < 0:
                        c0, c1 = (0, xhi) if part else (n[0] - 1, n[0] - 1)
                    elif xhi >= n[0]:
                        c0, c1 = (0, xhi - n[0]) if part else (xlo, n[0] - 1)
                    else:
                        c0, c1 = (xlo, xlo - 1) if part else (xlo, xhi)
                    if c1 < c0:
                        continue
                    b, ln = int(cs[rowbase + c0]), int(cs[rowbase + c1 + 1] - cs[rowbase + c0])
                    wy, wz = M32 / n[1], M32 / n[2]
                    ylo, yhi = (gy + dy) * wy - oy - 2.0, (gy + dy + 1) * wy - oy + 2.0
                    zlo, zhi = (gz + dz) * wz - oz - 2.0, (gz + dz + 1) * wz - oz + 2.0
                    ddy = max(0.0, ylo - gyhi, gylo - yhi) * hd[1]
                    ddz = max(0.0, zlo - gzhi, gzlo - zhi) * hd[2]
                    rx2 = r_s * r_s * (1 + 1e-9) - ddy * ddy - ddz * ddz
                    if rx2 <= 0:
                        continue
                    rx = int(math.ceil(math.sqrt(rx2) / hd[0]) + 2.0)
                    sh = -M32 if (xlo < 0 and not part) else (M32 if (xhi >= n[0] and part) else 0)

                    def first_ge(key):
                        lo_, hi_ = 0, ln
                        while lo_ < hi_:
                            mid = (lo_ + hi_) >> 1
                            if int(S[b + mid, 0]) + sh - ox < key:
                                lo_ = mid + 1
                            else:
                                hi_ = mid
                        return lo_

                    u, v = first_ge(gxlo - rx), first_ge(gxhi + rx + 1)
                    cand.update(range(b + u, b + v))
            for l in ins:
                d = (S - S[l] + 2 ** 31) % M32 - 2 ** 31
                r2 = ((d * np.asarray(hd)) ** 2).sum(1)
                nb = np.nonzero(r2 <= r_s * r_s)[0]
                pairs += len(nb)
                missed += sum(1 for j in nb if int(j) not in cand)
    return pairs, missed


def test_rbl_trim_keeps_every_shell_member_dense():
    sy = synth.make_system(12000, density=0.1, frac_charged=0.05, seed=5)  # 4 cells of 12.3 A
    pairs, missed = _check_rbl(sy.s, sy.box, 10.0, 1)
    assert pairs > 12000 * 300 and missed == 0


def test_rbl_trim_keeps_every_shell_member_multi_cell_groups():
    sy = synth.lj_electrolyte(20000)  # r_s = 8, about 6 ions a cell: groups span 5 cells
    pairs, missed = _check_rbl(sy.s, sy.box, synth.LJ_ELECTROLYTE["r_c"], 5)
    assert pairs > 0 and missed == 0
