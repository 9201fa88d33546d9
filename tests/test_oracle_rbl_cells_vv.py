"""Pins of the oracle's linked cells, random batch list (Eqs. Ci_Si, RBL, F_corr) and
velocity-Verlet integrator.

RBL is pinned by its exact limit (p >= #S_i gives the full cutoff sum), by set sizes
recounted by brute force, by the zero net force of Eq. F_corr, by the validity of every
drawn partner, by a brute-force re-derivation of the draws for a few particles, and by
unbiasedness over seeds. The integrator is pinned by the small-oscillation period of an
LJ dimer (closed form) and by energy conservation.
"""
import math

import numpy as np
import pytest

from paper_2609_02694_gb300 import synth

TWO32 = 2.0 ** 32


def test_cells_x_order_is_a_within_cell_sort(orc):
    """within="x": the same cells and cell_start, each cell's members ordered by (s_x, id),
    checked against one global sort by (cell, s_x, id)."""
    sy = synth.make_system(3000, density=0.1, seed=9)
    n = np.array([6, 5, 7], np.int32)
    c1, cs1, ids1 = orc.cells(sy.s, n)
    c2, cs2, ids2 = orc.cells(sy.s, n, within="x")
    assert np.array_equal(c1, c2) and np.array_equal(cs1, cs2)
    ref = np.lexsort((np.arange(3000), sy.s[:, 0].astype(np.int64), c1.astype(np.int64)))
    assert np.array_equal(ids2, ref)
    for c in range(int(np.prod(n))):  # a permutation inside every cell
        a, b = cs1[c], cs1[c + 1]
        assert np.array_equal(np.sort(ids1[a:b]), np.sort(ids2[a:b]))


def test_cells_contain_their_particles(orc):
    sy = synth.make_system(2000, density=0.1, seed=7)
    n = np.array([5, 6, 4], np.int32)
    cell_of, cell_start, ids = orc.cells(sy.s, n)
    r = sy.positions()
    a = sy.box / n
    c3 = np.stack([cell_of % n[0], (cell_of // n[0]) % n[1], cell_of // (n[0] * n[1])], 1)
    assert np.all(c3 * a <= r + 1e-12) and np.all(r < (c3 + 1) * a + 1e-12)
    # (cell, id) order and consistent cell_start
    assert np.array_equal(np.sort(ids), np.arange(2000))
    key = cell_of[ids].astype(np.int64) * 2000 + ids
    assert np.all(np.diff(key) > 0)
    assert cell_start[0] == 0 and cell_start[-1] == 2000
    counts = np.bincount(cell_of, minlength=int(np.prod(n)))
    assert np.array_equal(np.diff(cell_start), counts)


def _small(N=2000, seed=9, frac=0.1):
    return synth.make_system(N, density=0.1, frac_charged=frac, seed=seed)


def test_rbl_exact_limit(orc):
    """p >= #S_i: Eq. RBL is the plain cutoff sum at r_s and the correction vanishes."""
    sy = _small()
    r_s, r_core = 9.0, 4.5
    args = (sy.q, sy.types, sy.box, 0.09)
    ex = orc.real_space(sy.s, *args, r_s, synth.COULOMB_C, sy.eps, sy.sig)
    rb = orc.rbl(sy.s, *args, r_core, r_s, 100000, 1, 0, 0, synth.COULOMB_C, sy.eps, sy.sig)
    assert np.linalg.norm(rb["F"] - ex["F"]) < 1e-12 * np.linalg.norm(ex["F"])
    for k in ("U_real", "U_lj", "W_real", "W_lj"):
        assert rb[k] == pytest.approx(ex[k], rel=1e-12)
    assert np.array_equal(rb["n_core"] + rb["n_shell"], ex["nbr"])
    core = orc.real_space(sy.s, *args, r_core, synth.COULOMB_C, sy.eps, sy.sig)
    assert np.array_equal(rb["n_core"], core["nbr"])


def test_rbl_draws_valid_and_net_force_zero(orc):
    sy = _small()
    r_s, r_core, p = 9.0, 4.5, 10
    rb = orc.rbl(sy.s, sy.q, sy.types, sy.box, 0.09, r_core, r_s, p, 3, 5, 0,
                 synth.COULOMB_C, sy.eps, sy.sig)
    Fsum = rb["F"].sum(axis=0)
    assert np.abs(Fsum).max() < 1e-10 * np.abs(rb["F"]).sum()
    assert np.all(rb["n_shell"] > p)
    for i in range(0, sy.n, 97):
        for j in rb["partners"][i]:
            r2, _ = orc.min_image_r2(sy.s[i], sy.s[j], sy.box)
            assert r_core ** 2 < r2 <= r_s ** 2


def test_rbl_draws_match_brute_force_enumeration(orc):
    """Re-derive the shell order and the Philox draws for a few particles by brute force."""
    sy = _small(N=1500, seed=12)
    r_s, r_core, p, seed, step = 8.0, 4.0, 6, 77, 9
    rb = orc.rbl(sy.s, sy.q, sy.types, sy.box, 0.09, r_core, r_s, p, seed, step, 0,
                 synth.COULOMB_C, sy.eps, sy.sig)
    n = np.floor(sy.box / r_s).astype(np.int32)
    cell_of, cell_start, ids = orc.cells(sy.s, n, within="x")  # the RBL's canonical order
    for i in (0, 13, 700, 1499):
        ci = cell_of[i]
        c3 = (ci % n[0], (ci // n[0]) % n[1], ci // (n[0] * n[1]))
        shell = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    cc = [(c3[0] + dx) % n[0], (c3[1] + dy) % n[1], (c3[2] + dz) % n[2]]
                    cj = cc[0] + n[0] * (cc[1] + n[1] * cc[2])
                    for j in ids[cell_start[cj]:cell_start[cj + 1]]:
                        if j == i:
                            continue
                        d = ((sy.s[i].astype(np.int64) - sy.s[j].astype(np.int64) + 2 ** 31)
                             % 2 ** 32 - 2 ** 31) * (sy.box / TWO32)
                        r = math.sqrt((d * d).sum())
                        if r_core < r <= r_s:
                            shell.append(int(j))
        assert len(shell) == rb["n_shell"][i]
        want = []
        for t in range(p):
            w = orc.philox4x32_10([i, t // 4, step, 1], [seed & 0xFFFFFFFF, seed >> 32])[t % 4]
            want.append(shell[(int(w) * len(shell)) >> 32])
        assert list(rb["partners"][i]) == want



def test_rbl_rows_are_the_rows_of_the_full_list(orc):
    """The sampled-rows entry (used where the whole list is too large for the oracle): over
    every row it gives the full list's set sizes, draws, corrected forces (Eq. F_corr applied
    here) and energies; a sample of rows gives exactly those rows, whatever the sample."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.05, seed=5)
    args = (sy.s, sy.q, sy.types, sy.box, 0.09, 5.0, 10.0, 10, 3, 7, 0, synth.COULOMB_C,
            sy.eps, sy.sig)
    rb = orc.rbl(*args)
    al = orc.rbl_rows(*args, np.arange(sy.n))
    assert np.array_equal(al["n_core"], rb["n_core"])
    assert np.array_equal(al["n_shell"], rb["n_shell"])
    assert np.array_equal(al["partners"], rb["partners"])
    assert (rb["n_shell"] > 10).all()  # every row draws
    mean = al["Ft"].sum(0) / sy.n
    scale = np.abs(rb["F"]).max()
    assert np.abs(al["Ft"] - mean - rb["F"]).max() < 1e-12 * scale
    assert np.abs(mean).max() > 0.0  # the correction is not empty
    half = 0.5 * al["u"].sum(0)
    for k, key in enumerate(("U_real", "U_lj", "W_real", "W_lj")):
        assert half[k] == pytest.approx(rb[key], rel=1e-12, abs=1e-9)
    idx = np.array([sy.n - 1, 0, 4321, 17, 17, 9000])  # any order, repeats allowed
    sm = orc.rbl_rows(*args, idx)
    assert np.array_equal(sm["Ft"], al["Ft"][idx])
    assert np.array_equal(sm["partners"], al["partners"][idx])
    with pytest.raises(ValueError):
        orc.rbl_rows(*args, np.array([sy.n]))


@pytest.mark.slow
def test_rbl_unbiased_over_seeds(orc):
    """E[F_i] over RBL draws equals the exact cutoff force (Eq. RBL is unbiased; the mean
    correction of Eq. F_corr has zero expectation because the exact forces sum to 0)."""
    sy = synth.make_system(300, density=0.1, frac_charged=0.2, seed=21)
    r_s, r_core, p, n = 4.7, 2.5, 3, 3000
    ex = orc.real_space(sy.s, sy.q, sy.types, sy.box, 0.09, r_s, synth.COULOMB_C, sy.eps,
                        sy.sig)
    Fs = np.array([orc.rbl(sy.s, sy.q, sy.types, sy.box, 0.09, r_core, r_s, p, seed + 1, 0, 0,
                           synth.COULOMB_C, sy.eps, sy.sig)["F"] for seed in range(n)])
    z = np.abs(Fs.mean(0) - ex["F"]) / (Fs.std(0) / math.sqrt(n) + 1e-300)
    assert z.max() < 5.0, z.max()


def test_vv_dimer_period(orc):
    """LJ dimer near r_min = 2^(1/6) sigma oscillates with omega^2 = kappa U''(r_min) / mu,
    U''(r_min) = 144 eps / (2^(4/3) sigma^2)."""
    L, eps, sig, m = 40.0, 0.2, 3.0, 20.0
    rmin = 2 ** (1 / 6) * sig
    s = np.array([[0, 0, 0], [int((rmin + 0.01) / L * TWO32), 0, 0]], np.uint32)
    v = np.zeros((2, 3))
    mass = np.array([m, m])
    box = np.array([L, L, L])
    dt, kappa = 1.0, synth.ACCEL_KAPPA

    def forces(x):
        return orc.real_space(x, np.zeros(2), np.zeros(2, np.int32), box, 0.1, 12.0, 1.0,
                              [eps], [sig])["F"]

    F = forces(s)
    xs = []
    for _ in range(2600):
        orc.vv_drift(s, v, F, mass, box, dt, kappa)
        F = forces(s)
        orc.vv_kick(v, F, mass, dt, kappa)
        xs.append((int(s[1, 0]) - int(s[0, 0])) * L / TWO32 - rmin)
    xs = np.array(xs)
    cross = np.where((xs[:-1] > 0) & (xs[1:] <= 0))[0]
    # linear interpolation of downward zero crossings
    tc = cross + xs[cross] / (xs[cross] - xs[cross + 1])
    period = np.diff(tc).mean() * dt
    omega = math.sqrt(kappa * 144 * eps / (2 ** (4 / 3) * sig ** 2) / (m / 2))
    assert period == pytest.approx(2 * math.pi / omega, rel=2e-3)


def test_vv_energy_conservation(orc):
    sy = synth.make_system(216, density=0.03, frac_charged=0.0, seed=2, T=300.0)
    box, dt, kappa = sy.box, 1.0, synth.ACCEL_KAPPA
    s, v = sy.s.copy(), sy.v.copy()

    rc = 8.0
    u_rc = 4 * sy.eps[0] * ((sy.sig[0] / rc) ** 12 - (sy.sig[0] / rc) ** 6)

    def run_forces(x):
        # the truncated force is the gradient of the potential shifted by U(r_c) per pair
        r = orc.real_space(x, sy.q, sy.types, box, 0.09, rc, 1.0, sy.eps, sy.sig)
        return r["F"], r["U_lj"] - 0.5 * r["nbr"].sum() * u_rc

    def energy(U):
        return U + 0.5 * (sy.mass[:, None] * v * v).sum() / kappa

    F, U = run_forces(s)
    E0 = energy(U)
    Es = []
    for _ in range(300):
        orc.vv_drift(s, v, F, sy.mass, box, dt, kappa)
        F, U = run_forces(s)
        orc.vv_kick(v, F, sy.mass, dt, kappa)
        Es.append(energy(U))
    ke = 0.5 * (sy.mass[:, None] * v * v).sum() / kappa
    assert abs(np.array(Es) - E0).max() < 2e-4 * ke
    p = (sy.mass[:, None] * v).sum(0)
    assert np.abs(p).max() < 1e-9


def _nvt_run(orc, steps, tau, T0=300.0, dt=1.0):
    sy = synth.make_system(216, density=0.03, frac_charged=0.0, seed=2, T=150.0)
    box, kappa, kB = sy.box, synth.ACCEL_KAPPA, synth.BOLTZMANN_KB
    s, v = sy.s.copy(), sy.v.copy()
    rc = 8.0
    u_rc = 4 * sy.eps[0] * ((sy.sig[0] / rc) ** 12 - (sy.sig[0] / rc) ** 6)
    Nf = 3 * sy.n - 3
    Q = Nf * kB * T0 * tau ** 2
    xe = np.zeros(2)

    def forces(x):
        r = orc.real_space(x, sy.q, sy.types, box, 0.09, rc, 1.0, sy.eps, sy.sig)
        return r["F"], r["U_lj"] - 0.5 * r["nbr"].sum() * u_rc

    F, U = forces(s)
    H, T = [], []
    for _ in range(steps):
        orc.nh_half(v, sy.mass, kappa, Nf, kB * T0, Q, dt, xe)
        orc.vv_drift(s, v, F, sy.mass, box, dt, kappa)
        F, U = forces(s)
        orc.vv_kick(v, F, sy.mass, dt, kappa)
        orc.nh_half(v, sy.mass, kappa, Nf, kB * T0, Q, dt, xe)
        K = 0.5 * (sy.mass[:, None] * v * v).sum() / kappa
        H.append(U + K + 0.5 * Q * xe[0] ** 2 + Nf * kB * T0 * xe[1])
        T.append(2 * K / (Nf * kB))
    return np.array(H), np.array(T)


def test_nose_hoover_conserves_extended_energy_and_thermalises(orc):
    """With the Nose-Hoover half steps around Verlet, H = U + K + Q xi^2/2 + Nf kT eta is
    conserved, and the temperature is driven from 150 K towards the 300 K target."""
    H, T = _nvt_run(orc, 1500, tau=50.0)
    assert np.abs(H - H[0]).max() < 2e-3 * abs(H[0])
    assert abs(T[-500:].mean() - 300.0) < 45.0
    assert T[:20].mean() < 200.0


def test_nose_hoover_weak_coupling_limit_is_nve(orc):
    """tau -> infinity (Q -> infinity) leaves the velocities untouched."""
    sy = synth.make_system(64, density=0.03, frac_charged=0.0, seed=3)
    v = sy.v.copy()
    xe = np.zeros(2)
    orc.nh_half(v, sy.mass, synth.ACCEL_KAPPA, 189, synth.BOLTZMANN_KB * 300, 1e300, 1.0, xe)
    assert np.array_equal(v, sy.v) and abs(xe[0]) < 1e-290
