"""Pins of the oracle's Ewald, RBE and real-space parts (Sec. 2.1, Eqs. Ewald .. F_long_RBE).

Each test checks the oracle against something its code does not contain: the rock-salt
Madelung constant, brute-force image sums, alpha-invariance of the total Coulomb energy,
finite differences of each energy (positions and volume), exact identities of the RBE
estimator and its unbiasedness over 10^4 seeds.
"""
import math
import os

import numpy as np
import pytest

from paper_2609_02694_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TWO32 = 2.0 ** 32


def _madelung():
    with open(os.path.join(GOLDEN, "madelung_nacl.txt")) as f:
        return float([ln for ln in f if not ln.startswith("#") and ln.strip()][0])


def _random_system(N, box, seed, charges=None, min_sep=1.0):
    rng = np.random.default_rng(seed)
    box = np.asarray(box, np.float64)
    pts = []
    while len(pts) < N:
        r = rng.uniform(0, 1, 3) * box
        ok = True
        for p in pts:
            d = r - p
            d -= box * np.round(d / box)
            if np.linalg.norm(d) < min_sep:
                ok = False
                break
        if ok:
            pts.append(r)
    s = np.floor(np.array(pts) / box * TWO32).astype(np.uint64).astype(np.uint32)
    if charges is None:
        q = np.array([(1.0 if i % 2 == 0 else -1.0) for i in range(N)])
    else:
        q = np.asarray(charges, np.float64)
    return s, q


def _coulomb_total(orc, s, q, box, alpha, rc, C=1.0):
    N = len(q)
    Fk, Uk, Wk = orc.ewald_kspace(s, q, box, alpha, C)
    rs = orc.real_space(s, q, np.zeros(N, np.int32), box, alpha, rc, C, [0.0], [1.0])
    U = Uk + rs["U_real"] - orc.self_energy(q, alpha, C)
    return Fk + rs["F"], U, Wk + rs["W_real"]


def test_madelung_rock_salt(orc):
    """Ewald energy of rock salt = -N M C / (2a); every force vanishes by symmetry."""
    n, a, C = 4, 2.0, synth.COULOMB_C
    L = n * a
    idx = np.array([(x, y, z) for z in range(n) for y in range(n) for x in range(n)])
    s = (idx * (TWO32 / n)).astype(np.uint64).astype(np.uint32)
    q = np.where(idx.sum(axis=1) % 2 == 0, 1.0, -1.0)
    box = np.array([L, L, L])
    F, U, _ = _coulomb_total(orc, s, q, box, alpha=2.7, rc=0.4999 * L, C=C)
    want = -len(q) * _madelung() * C / (2.0 * a)
    assert U == pytest.approx(want, rel=1e-9)
    assert np.abs(F).max() < 1e-9 * abs(want)


@pytest.mark.parametrize("box,R,tol_u,tol_f", [
    ((10.0, 10.0, 10.0), 64, 1e-7, 1e-6),
    ((10.0, 11.0, 12.0), 64, 1e-4, 1e-4),
])
def test_brute_force_image_sum(orc, box, R, tol_u, tol_f):
    """Spherical image sum (tin-foil corrected) of Eq. Coul_potential = Ewald sum."""
    box = np.array(box)
    s, q = _random_system(8, box, seed=5, charges=[1, -1, 1, -1, 2, -2, 1, -1])
    F, U, _ = _coulomb_total(orc, s, q, box, alpha=0.6, rc=0.4999 * box.min())
    Fb, Ub = orc.brute_coulomb(s, q, box, 1.0, R)
    assert abs(Ub - U) < tol_u * abs(U)
    assert np.abs(Fb - F).max() < tol_f * np.abs(F).max()


def test_alpha_invariance(orc):
    """Total Coulomb energy and forces do not depend on the splitting parameter alpha."""
    box = np.array([15.0, 15.0, 15.0])
    s, q = _random_system(20, box, seed=11)
    res = [_coulomb_total(orc, s, q, box, alpha, rc=7.4) for alpha in (0.4, 0.8, 1.6)]
    F0, U0, _ = res[0]
    for F, U, _ in res[1:]:
        assert U == pytest.approx(U0, rel=1e-9)
        assert np.abs(F - F0).max() < 1e-8 * np.abs(F0).max()


def _fd_forces(energy, s, box, h=1e-5):
    """Central differences of energy(s) with respect to each coordinate, on the grid."""
    N = len(s)
    F = np.zeros((N, 3))
    for i in range(N):
        for d in range(3):
            ds = max(1, int(round(h / box[d] * TWO32)))
            he = ds * box[d] / TWO32
            sp = s.copy(); sp[i, d] = np.uint32((int(sp[i, d]) + ds) % (1 << 32))
            sm = s.copy(); sm[i, d] = np.uint32((int(sm[i, d]) - ds) % (1 << 32))
            F[i, d] = -(energy(sp) - energy(sm)) / (2 * he)
    return F


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_fd_ewald_kspace(orc):
    box = np.array([9.0, 10.0, 11.0])
    s, q = _random_system(6, box, seed=3)
    F, U, _ = orc.ewald_kspace(s, q, box, 0.5, 1.0)
    Ffd = _fd_forces(lambda x: orc.ewald_kspace(x, q, box, 0.5, 1.0)[1], s, box)
    assert _rel_l2(F, Ffd) < 1e-6


def _far_from_cutoff(orc, s, box, rc, margin=1e-3):
    for i in range(len(s)):
        for j in range(i + 1, len(s)):
            r2, _ = orc.min_image_r2(s[i], s[j], box)
            if abs(math.sqrt(r2) - rc) < margin:
                return False
    return True


def test_fd_real_space_coulomb_lj(orc):
    box = np.array([14.0, 15.0, 16.0])
    rc = 6.5
    s, q = _random_system(24, box, seed=21, min_sep=2.6)
    q[::3] = 0.0
    assert _far_from_cutoff(orc, s, box, rc)
    types = np.zeros(len(q), np.int32)
    args = (box, 0.3, rc, 332.06371, [0.1], [3.0])
    rs = orc.real_space(s, q, types, *args)
    Ffd = _fd_forces(lambda x: (lambda r: r["U_real"] + r["U_lj"])(
        orc.real_space(x, q, types, *args)), s, box)
    assert _rel_l2(rs["F"], Ffd) < 1e-6


def test_fd_real_space_two_types(orc):
    """Per-type-pair LJ table (eps_ij, sig_ij of Eq. LJ) through finite differences."""
    box = np.array([14.0, 14.0, 14.0])
    rc = 6.0
    s, q = _random_system(18, box, seed=8, min_sep=2.4)
    types = (np.arange(18) % 2).astype(np.int32)
    eps = [0.1, 0.2, 0.2, 0.05]
    sig = [3.0, 2.5, 2.5, 2.2]
    assert _far_from_cutoff(orc, s, box, rc)
    args = (box, 0.35, rc, 1.0, eps, sig)
    rs = orc.real_space(s, q, types, *args)
    Ffd = _fd_forces(lambda x: (lambda r: r["U_real"] + r["U_lj"])(
        orc.real_space(x, q, types, *args)), s, box)
    assert _rel_l2(rs["F"], Ffd) < 1e-6


def _scaled_energy(fn, box, lam):
    return fn(np.asarray(box) * lam)


@pytest.mark.parametrize("part", ["kspace", "real"])
def test_virial_is_volume_derivative(orc, part):
    """W = -dU/d ln(lambda) under uniform scaling of the box at fixed fractional positions."""
    box = np.array([12.0, 13.0, 14.0])
    s, q = _random_system(16, box, seed=4, min_sep=2.5)
    types = np.zeros(16, np.int32)
    eps_ = 1e-6
    if part == "kspace":
        def fn(b):
            return orc.ewald_kspace(s, q, b, 0.45, 1.0)
        W = fn(box)[2]
        Up, Um = fn(box * (1 + eps_))[1], fn(box * (1 - eps_))[1]
    else:
        assert _far_from_cutoff(orc, s, box, 5.9, margin=1e-4)

        def fn(b):
            r = orc.real_space(s, q, types, b, 0.45, 5.9, 1.0, [0.1], [3.0])
            return r["U_real"] + r["U_lj"], r["W_real"] + r["W_lj"]
        W = fn(box)[1]
        Up, Um = fn(box * (1 + eps_))[0], fn(box * (1 - eps_))[0]
    dUdl = (Up - Um) / (math.log(1 + eps_) - math.log(1 - eps_))
    assert W == pytest.approx(-dUdl, rel=1e-6, abs=1e-9)


def test_lj_force_vanishes_at_minimum(orc):
    """G_LJ = 0 at r = 2^(1/6) sigma (minimum of Eq. LJ), and U_LJ = -eps there."""
    L, sig, eps = 40.0, 3.0, 0.2
    rmin = 2 ** (1 / 6) * sig
    s = np.array([[0, 0, 0], [int(round(rmin / L * TWO32)), 0, 0]], np.uint32)
    r_eff = int(s[1, 0]) * L / TWO32
    rs = orc.real_space(s, np.zeros(2), np.zeros(2, np.int32), np.array([L] * 3), 0.1, 10.0,
                        1.0, [eps], [sig])
    # |F| <= U''(rmin) |r - rmin| with U'' = 144 eps / (2^(4/3) sig^2)
    bound = 144 * eps / (2 ** (4 / 3) * sig ** 2) * abs(r_eff - rmin) * 1.01 + 1e-12
    assert np.abs(rs["F"]).max() <= bound
    assert rs["U_lj"] == pytest.approx(-eps, rel=1e-9)


def test_small_alpha_gives_bare_coulomb(orc):
    """alpha -> 0: the erfc kernel of Eq. Ewald becomes bare minimum-image Coulomb."""
    L, d = 100.0, 3.0
    s = np.array([[0, 0, 0], [int(d / L * TWO32), 0, 0]], np.uint32)
    dd = int(s[1, 0]) * L / TWO32
    q = np.array([1.0, -1.0])
    rs = orc.real_space(s, q, np.zeros(2, np.int32), np.array([L] * 3), 1e-18, 40.0,
                        synth.COULOMB_C, [0.0], [1.0])
    want = synth.COULOMB_C / dd ** 2
    assert rs["F"][0, 0] == pytest.approx(want, rel=1e-8)     # pulled towards +x
    assert rs["F"][1, 0] == pytest.approx(-want, rel=1e-8)
    assert rs["U_real"] == pytest.approx(-synth.COULOMB_C / dd, rel=1e-8)


def test_isolated_pair_energy_approaches_minus_c_over_r(orc):
    """Two opposite charges far from their images: total Ewald energy -> -C/r."""
    L, d = 60.0, 2.0
    s = np.array([[0, 0, 0], [int(d / L * TWO32), 0, 0]], np.uint32)
    dd = int(s[1, 0]) * L / TWO32
    q = np.array([1.0, -1.0])
    F, U, _ = _coulomb_total(orc, s, q, np.array([L] * 3), alpha=0.1, rc=29.0, C=1.0)
    assert U == pytest.approx(-1.0 / dd, rel=1e-3)
    assert F[0, 0] == pytest.approx(1.0 / dd ** 2, rel=1e-3)


# ----------------------------------------------------------------------------------
# RBE estimator on a fixed mode set


def test_rbe_net_force_zero(orc):
    """sum_i q_i Im(exp(-ik.r_i) rho) = Im(conj(rho) rho) = 0 for every sampled mode."""
    sy = synth.make_system(3000, L=32.0, all_charged=True, seed=1)
    m, S = orc.sample_k(1, 0, 0, sy.box, 0.09, 100)
    F, U, W = orc.rbe_kspace(sy.s, sy.q, sy.box, 0.09, synth.COULOMB_C, m, S)
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).sum()


def test_rbe_fd_on_fixed_modes(orc):
    box = np.array([10.0, 11.0, 12.0])
    s, q = _random_system(8, box, seed=13)
    m, S = orc.sample_k(5, 2, 0, box, 0.3, 40)
    F, U, _ = orc.rbe_kspace(s, q, box, 0.3, 1.0, m, S)
    Ffd = _fd_forces(lambda x: orc.rbe_kspace(x, q, box, 0.3, 1.0, m, S)[1], s, box)
    assert _rel_l2(F, Ffd) < 1e-6


def test_rbe_matches_ewald_when_modes_enumerate(orc):
    """With the sampled set replaced by every mode, each weighted by exp(-k^2/4a) P/S, the
    estimator reduces to the full sum: check via a weighted mode list (P copies)."""
    box = np.array([7.0, 8.0, 9.0])
    s, q = _random_system(6, box, seed=31)
    alpha = 1.5
    Fe, Ue, We = orc.ewald_kspace(s, q, box, alpha, 1.0)
    # Build the full mode list and evaluate each mode as a P=1 estimator with S = weight.
    Ms = [orc.kdim_M(L, alpha) for L in box]
    F = np.zeros_like(Fe)
    U = W = 0.0
    for mz in range(-Ms[2], Ms[2] + 1):
        for my in range(-Ms[1], Ms[1] + 1):
            for mx in range(-Ms[0], Ms[0] + 1):
                if mx == my == mz == 0:
                    continue
                k2 = sum((2 * np.pi * v / Lb) ** 2 for v, Lb in zip((mx, my, mz), box))
                w = math.exp(-k2 / (4 * alpha))
                if w < 1e-18:
                    continue
                f, u, wv = orc.rbe_kspace(s, q, box, alpha, 1.0, np.array([[mx, my, mz]]), w)
                F += f
                U += u
                W += wv
    assert U == pytest.approx(Ue, rel=1e-10)
    assert W == pytest.approx(We, rel=1e-9, abs=1e-12)
    assert _rel_l2(F, Fe) < 1e-10


@pytest.mark.slow
def test_rbe_unbiased_over_seeds(orc):
    """Mean of the RBE force over 10^4 seeds equals the full Ewald force within 4 sigma."""
    box = np.array([10.0, 10.0, 10.0])
    s, q = _random_system(12, box, seed=17)
    alpha, P, n = 0.5, 8, 10000
    Fe, Ue, We = orc.ewald_kspace(s, q, box, alpha, 1.0)
    Fs = np.zeros((n, 12, 3))
    Us = np.zeros(n)
    Ws = np.zeros(n)
    for seed in range(n):
        m, S = orc.sample_k(seed + 1, 0, 0, box, alpha, P)
        Fs[seed], Us[seed], Ws[seed] = orc.rbe_kspace(s, q, box, alpha, 1.0, m, S)
    mean = Fs.mean(axis=0)
    sem = Fs.std(axis=0) / math.sqrt(n)
    z = np.abs(mean - Fe) / sem
    assert z.max() < 4.5, z.max()
    for est, exact in ((Us, Ue), (Ws, We)):
        assert abs(est.mean() - exact) < 4 * est.std() / math.sqrt(n)


def test_rbe_variance_scales_as_one_over_p(orc):
    box = np.array([10.0, 10.0, 10.0])
    s, q = _random_system(12, box, seed=17)
    alpha, n = 0.5, 1500
    var = {}
    for P in (4, 16):
        Fs = np.array([orc.rbe_kspace(s, q, box, alpha, 1.0,
                                      *orc.sample_k(seed + 7, 1, 0, box, alpha, P))[0]
                       for seed in range(n)])
        var[P] = Fs.var(axis=0).sum()
    assert var[4] / var[16] == pytest.approx(4.0, rel=0.2)


def test_truncated_ewald_rock_salt(orc):
    """Ewald sum truncated at mode weight 1e-10 still gives the rock-salt Madelung energy
    (to the accuracy the truncation allows) and zero forces by symmetry."""
    n, a, C = 4, 2.0, synth.COULOMB_C
    L = n * a
    idx = np.array([(x, y, z) for z in range(n) for y in range(n) for x in range(n)])
    s = (idx * (TWO32 / n)).astype(np.uint64).astype(np.uint32)
    q = np.where(idx.sum(axis=1) % 2 == 0, 1.0, -1.0)
    box = np.array([L, L, L])
    alpha, rc = 2.7, 0.4999 * L
    rs = orc.real_space(s, q, np.zeros(len(q), np.int32), box, alpha, rc, C, [0.0], [1.0])
    Fk, Uk, _ = orc.ewald_kspace_tol(s, q, box, alpha, C, 1e-10)
    U = rs["U_real"] + Uk - orc.self_energy(q, alpha, C)
    want = -len(q) * _madelung() * C / (2.0 * a)
    assert U == pytest.approx(want, rel=1e-8)
    assert np.abs(rs["F"] + Fk).max() < 1e-8 * abs(want)


def test_truncated_ewald_converges_to_full(orc):
    """The truncated sum is the full sum restricted to the sphere exp(-k^2/4 alpha) >= tol:
    a tolerance below every mode weight the full sum keeps reproduces it, and the error of a
    coarse tolerance falls with the tolerance and stays of its order."""
    box = np.array([15.0, 16.0, 17.0])
    s, q = _random_system(30, box, seed=21)
    alpha, C = 0.3, 1.0
    F0, U0, W0 = orc.ewald_kspace(s, q, box, alpha, C)
    F1, U1, W1 = orc.ewald_kspace_tol(s, q, box, alpha, C, 1e-17)
    assert np.abs(F1 - F0).max() < 1e-12 * np.abs(F0).max()
    assert U1 == pytest.approx(U0, rel=1e-12) and W1 == pytest.approx(W0, rel=1e-11)
    errs = []
    for tol in (1e-3, 1e-5, 1e-7):
        F, U, _ = orc.ewald_kspace_tol(s, q, box, alpha, C, tol)
        errs.append(np.linalg.norm(F - F0) / np.linalg.norm(F0))
        assert errs[-1] < 30 * tol
    assert errs[0] > errs[1] > errs[2]
    # invalid tolerances are refused
    with pytest.raises(ValueError):
        orc.ewald_kspace_tol(s, q, box, alpha, C, 0.0)
