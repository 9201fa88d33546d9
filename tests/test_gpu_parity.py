"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Integer results (mode sets, cells and their order, neighbour and RBL set sizes, RBL
draws) must match bit for bit. Forces must match within 1e-5 relative L2 in the FP32
forms on the same sampled mode set (FP64 form: 1e-10), and energies and virials within
the tolerances stated beside each check. Inputs come from the seeded generator; the
oracle never sees the GPU's output.
"""
import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build, synth

import sampled

pytestmark = pytest.mark.gpu

C = synth.COULOMB_C
ALPHA = synth.ALPHA
RC = synth.R_CUT
TOL_F32 = 1e-5
TOL_F64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def handle(sy, P, precision="fp32_comp", **kw):
    return binding.from_system(sy, P=P, alpha=kw.pop("alpha", ALPHA), r_c=kw.pop("r_c", RC),
                               precision=precision, coulomb_C=C, **kw)


def sample_ids(sy, n, seed=0):
    """n random particles, the first 16 charged ones, and the first and last id."""
    rng = np.random.default_rng(seed)
    charged = np.flatnonzero(sy.q != 0)
    return np.unique(np.concatenate([rng.choice(sy.n, n, replace=False), charged[:16],
                                     [0, sy.n - 1]]))


def oracle_all(orc, sy, m, S, alpha=ALPHA, rc=RC):
    return orc.total_forces(sy.s, sy.q, sy.types, sy.box, alpha, rc, C, sy.eps, sy.sig, m, S)


# -------------------------------------------------------------------------- sampler


@pytest.mark.parametrize("box,P,seed,step", [
    ((32.0, 32.0, 32.0), 100, 1, 0),
    ((32.0, 32.0, 32.0), 2000, 7, 123456),
    ((218.877, 218.877, 218.877), 1000, 2, 3),
    ((25.3, 31.0, 47.9), 333, 2 ** 40 + 5, 2 ** 32 + 9),
])
def test_kset_bit_exact(orc, box, P, seed, step):
    sy = synth.make_system(64, L=min(box), seed=5)
    sy.box = np.array(box)
    with handle(sy, P, seed=seed, r_c=min(10.0, min(box) / 3 - 0.1)) as h:
        m, S = h.sample_k(step)
    mo, So = orc.sample_k(seed, step, 0, np.array(box), ALPHA, P)
    assert np.array_equal(m, mo)
    assert S == So


# -------------------------------------------------------------------------- cells


@pytest.mark.parametrize("N,L,sub", [(3000, 32.0, 0), (20000, 58.48, 2), (20000, 58.48, 1),
                                     (5000, 40.0, 3)])
def test_cells_bit_exact(orc, N, L, sub):
    """Cell traversal: members ordered by (cell, s_x, id)."""
    sy = synth.make_system(N, L=L, frac_charged=0.1, seed=11)
    with handle(sy, 50, cell_sub=sub) as h:
        h.forces(0)
        n, cs, ids = h.cells()
    _, cso, idso = orc.cells(sy.s, n, within="x")
    assert np.array_equal(cs, cso)
    assert np.array_equal(ids, idso)


def test_cells_bit_exact_rbl_grid(orc):
    """Random batch list (cells of r_s): members ordered by (cell, s_x, id) as well, the
    order its shells enumerate."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=11)
    with handle(sy, 50, r_core=4.0, p_rbl=8) as h:
        h.forces(0)
        n, cs, ids = h.cells()
    _, cso, idso = orc.cells(sy.s, n, within="x")
    assert np.array_equal(cs, cso)
    assert np.array_equal(ids, idso)


# -------------------------------------------------------------------------- k-space


@pytest.mark.parametrize("precision,tol", [("fp32_comp", 2e-6), ("fp32", 2e-5), ("fp64", 1e-12)])
def test_structure_factor(orc, precision, tol):
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=12)
    with handle(sy, 200, precision=precision) as h:
        h.forces(0)
        rho, m = h.rho()
    mo, _ = orc.sample_k(1, 0, 0, sy.box, ALPHA, 200)
    assert np.array_equal(m, mo)
    ro = orc.rho(sy.s, sy.q, sy.box, mo)
    assert rel_l2(rho, ro) < tol


# -------------------------------------------------------------------------- forces


CASES = [
    # name, system kwargs, P, extra handle kwargs
    ("n3000_all_charged", dict(N=3000, L=32.0, all_charged=True, seed=1), 100, {}),
    ("n20k_10pct", dict(N=20000, density=0.1, frac_charged=0.1, seed=2), 200, {}),
    ("n20k_10pct_sub1", dict(N=20000, density=0.1, frac_charged=0.1, seed=2), 200,
     dict(cell_sub=1)),
    ("n7777_ragged", dict(N=7777, density=0.08, frac_charged=0.3, seed=9), 57, {}),
]


@pytest.mark.parametrize("name,skw,P,hkw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp32_comp", "fp64"])
def test_forces_match_oracle(orc, name, skw, P, hkw, precision):
    sy = synth.make_system(**skw)
    with handle(sy, P, precision=precision, **hkw) as h:
        F, E, W = h.forces_f64(0)
        m, S = sampled.oracle_modes(orc, h, sy, P, 0)
        nbr, _ = h.neighbor_counts()
    ref = oracle_all(orc, sy, m, S)
    tol = TOL_F64 if precision == "fp64" else TOL_F32
    assert rel_l2(F, ref["F"]) < tol
    assert np.array_equal(nbr, ref["nbr"])
    etol = 1e-10 if precision == "fp64" else 2e-6
    assert E["real"] == pytest.approx(ref["U_real"], rel=etol, abs=1e-6)
    assert E["lj"] == pytest.approx(ref["U_lj"], rel=etol)
    assert E["kspace"] == pytest.approx(ref["U_k"], rel=etol)
    assert E["self"] == pytest.approx(ref["U_self"], rel=1e-12)
    assert W["real"] == pytest.approx(ref["W_real"], rel=etol, abs=1e-6)
    assert W["lj"] == pytest.approx(ref["W_lj"], rel=etol)
    assert W["kspace"] == pytest.approx(ref["W_k"], rel=etol)


def test_orthorhombic_two_types(orc):
    rng = np.random.default_rng(4)
    sy = synth.make_system(6000, L=40.0, frac_charged=0.2, seed=4)
    sy.box = np.array([40.0, 45.0, 52.0])
    sy.types = (rng.uniform(size=sy.n) < 0.3).astype(np.int32)
    sy.eps = np.array([0.1, 0.15, 0.15, 0.2])
    sy.sig = np.array([3.0, 2.8, 2.8, 2.6])
    with handle(sy, 150) as h:
        F, E, W = h.forces_f64(4)
        m, S = sampled.oracle_modes(orc, h, sy, 150, 4)
        nbr, _ = h.neighbor_counts()
    ref = oracle_all(orc, sy, m, S)
    assert rel_l2(F, ref["F"]) < TOL_F32
    assert np.array_equal(nbr, ref["nbr"])
    assert E["lj"] == pytest.approx(ref["U_lj"], rel=2e-6)


def test_plain_fp32_is_worse_than_compensated(orc):
    sy = synth.make_system(40000, density=0.1, frac_charged=0.1, seed=21)
    errs = {}
    for prec in ("fp32", "fp32_comp"):
        with handle(sy, 400, precision=prec) as h:
            h.forces(0)
            rho, m = h.rho()
        errs[prec] = rel_l2(rho, orc.rho(sy.s, sy.q, sy.box, m))
    assert errs["fp32_comp"] < errs["fp32"]


def test_no_charges_and_single_mode(orc):
    sy = synth.make_system(3000, density=0.1, frac_charged=0.0, seed=3)
    with handle(sy, 1) as h:
        F, E, W = h.forces_f64(0)
    ref = orc.real_space(sy.s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig)
    assert rel_l2(F, ref["F"]) < TOL_F32
    assert E["kspace"] == 0.0 and E["real"] == 0.0


def test_tiny_box_edge(orc):
    """Smallest box the stencil allows (5 cells of r_c/2 per axis) with a few particles."""
    sy = synth.make_system(12, L=25.1, all_charged=True, seed=8)
    with handle(sy, 16) as h:
        F, E, W = h.forces_f64(2)
        m, S = sampled.oracle_modes(orc, h, sy, 16, 2)
        nbr, _ = h.neighbor_counts()
    ref = oracle_all(orc, sy, m, S)
    assert rel_l2(F, ref["F"]) < TOL_F32
    assert np.array_equal(nbr, ref["nbr"])


def test_deterministic_across_runs():
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=2)
    out = []
    for _ in range(2):
        with handle(sy, 200) as h:
            F, E, W = h.forces_f64(5)
            out.append((F, E["total"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_rbe_net_force_zero_on_gpu():
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=2)
    with handle(sy, 200, precision="fp64") as h:
        F, _, _ = h.forces_f64(0)
    # total force: real space obeys Newton 3, RBE k-space sums to zero (Eq. F_long_RBE)
    assert np.abs(F.sum(axis=0)).max() < 1e-9 * np.abs(F).sum()


def test_invalid_input_rejected():
    sy = synth.make_system(100, L=30.0, all_charged=True, seed=1)
    q = sy.q.copy()
    q[0] += 0.5
    with pytest.raises(binding.RBEError):
        binding.RBE(sy.box, sy.positions(), q, alpha=ALPHA, r_c=RC, P=10, eps=sy.eps,
                    sigma=sy.sig)
    with pytest.raises(binding.RBEError):
        binding.RBE(sy.box, sy.positions(), sy.q, alpha=ALPHA, r_c=15.5, P=10, eps=sy.eps,
                    sigma=sy.sig)


# -------------------------------------------------------------------------- RBL


@pytest.mark.parametrize("precision,tol", [("fp32_comp", TOL_F32), ("fp64", TOL_F64)])
def test_rbl_bit_exact_sets_and_draws(orc, precision, tol):
    sy = synth.make_system(12000, density=0.1, frac_charged=0.05, seed=5)
    p, r_core, seed, step = 10, 5.0, 3, 7
    with handle(sy, 100, precision=precision, r_core=r_core, p_rbl=p, seed=seed) as h:
        F, E, W = h.forces_f64(step)
        nc, ns = h.neighbor_counts()
        partners = h.rbl_partners()
        m, S = sampled.oracle_modes(orc, h, sy, 100, step, seed=seed)
    ref = orc.rbl(sy.s, sy.q, sy.types, sy.box, ALPHA, r_core, RC, p, seed, step, 0, C,
                  sy.eps, sy.sig)
    assert np.array_equal(nc, ref["n_core"])
    assert np.array_equal(ns, ref["n_shell"])
    assert np.array_equal(partners, ref["partners"])
    Fk, Uk, Wk = orc.rbe_kspace(sy.s, sy.q, sy.box, ALPHA, C, m, S)
    assert rel_l2(F, ref["F"] + Fk) < tol
    etol = 1e-10 if precision == "fp64" else 2e-6
    assert E["lj"] == pytest.approx(ref["U_lj"], rel=etol)
    assert E["real"] == pytest.approx(ref["U_real"], rel=etol, abs=1e-6)


@pytest.mark.parametrize("precision,tol", [("fp32_comp", TOL_F32), ("fp64", TOL_F64)])
@pytest.mark.parametrize("eager", [0, 1])
def test_rbl_wrapping_box_matches_oracle(orc, precision, tol, eager):
    """A box of three cells of r_s per axis (6,000 particles at density 0.1, L = 39.1 A):
    a cell plus r_s reaches past L/2, so the random batch list runs its wrapping variant,
    which folds every difference into the box. Core and shell sizes and the drawn partners
    (Eqs. Ci_Si, RBL) match the oracle bit for bit, and forces and energies (with the
    correction of Eq. F_corr) match it within the form's tolerance, with eager shell sums
    on and off."""
    sy = synth.make_system(6000, density=0.1, frac_charged=0.1, seed=17)
    p, r_core, seed, step, P = 10, 5.0, 4, 2, 64
    with handle(sy, P, precision=precision, r_core=r_core, p_rbl=p, seed=seed) as h:
        h.set_tuning("rbl_eager", eager)
        F, E, W = h.forces_f64(step)
        nc, ns = h.neighbor_counts()
        partners = h.rbl_partners()
        n, _, _ = h.cells()
        m, S = sampled.oracle_modes(orc, h, sy, P, step, seed=seed)
    assert tuple(n) == (3, 3, 3)
    assert RC + sy.box[0] / 3 >= sy.box[0] / 2  # the condition that selects the variant
    ref = orc.rbl(sy.s, sy.q, sy.types, sy.box, ALPHA, r_core, RC, p, seed, step, 0, C,
                  sy.eps, sy.sig)
    assert np.array_equal(nc, ref["n_core"])
    assert np.array_equal(ns, ref["n_shell"])
    assert np.array_equal(partners, ref["partners"])
    assert (ns > p).any()
    Fk, Uk, Wk = orc.rbe_kspace(sy.s, sy.q, sy.box, ALPHA, C, m, S)
    assert rel_l2(F, ref["F"] + Fk) < tol
    etol = 1e-10 if precision == "fp64" else 2e-6
    assert E["lj"] == pytest.approx(ref["U_lj"], rel=etol)
    assert E["real"] == pytest.approx(ref["U_real"], rel=etol, abs=1e-6)
    assert W["lj"] == pytest.approx(ref["W_lj"], rel=etol)


def test_rbl_small_shell_takes_all(orc):
    """p >= #S_i: every shell partner enters with weight 1 (exact cutoff sum)."""
    sy = synth.make_system(4000, density=0.1, frac_charged=0.1, seed=6)
    with handle(sy, 50, r_core=8.0, p_rbl=32, r_c=8.1) as h:
        F, E, W = h.forces_f64(0)
        m, S = sampled.oracle_modes(orc, h, sy, 50, 0)
    ex = oracle_all(orc, sy, m, S, rc=8.1)
    assert rel_l2(F, ex["F"]) < TOL_F32


def test_rbl_eager_shell_bit_identical(orc):
    """Shells of mean size ~p: the eager variant (shell pairs summed while classifying) and
    the draw pass give bit-identical forces, energies, counts and partners, and match the
    oracle's draws."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=8)
    p, r_core, r_c, seed, step = 30, 4.5, 5.2, 2, 3
    out = {}
    for eager in (0, 1):
        with handle(sy, 64, r_core=r_core, p_rbl=p, r_c=r_c, seed=seed) as h:
            h.set_tuning("rbl_eager", eager)
            assert h.get_tuning("rbl_eager") == eager
            F, E, W = h.forces_f64(step)
            out[eager] = (F, E, W, *h.neighbor_counts(), h.rbl_partners())
    F0, E0, W0, nc0, ns0, pa0 = out[0]
    F1, E1, W1, nc1, ns1, pa1 = out[1]
    assert np.array_equal(F0, F1)
    assert E0 == E1 and W0 == W1
    assert np.array_equal(nc0, nc1) and np.array_equal(ns0, ns1) and np.array_equal(pa0, pa1)
    assert (ns0 <= p).any() and (ns0 > p).any()  # both branches taken
    ref = orc.rbl(sy.s, sy.q, sy.types, sy.box, ALPHA, r_core, r_c, p, seed, step, 0, C,
                  sy.eps, sy.sig)
    assert np.array_equal(ns1, ref["n_shell"])
    assert np.array_equal(pa1, ref["partners"])


@pytest.mark.parametrize("density,eager", [(0.1, 0), (0.1, 1), (0.02, 1)])
def test_rbl_span_bit_identical(orc, density, eager):
    """Warp groups spanning several cells in x (the dilute-system layout) enumerate every
    particle's shell in the same canonical order: forces, energies, counts and draws are
    bit-identical for every span and match the oracle's sets and draws."""
    sy = synth.make_system(20000, density=density, frac_charged=0.1, seed=9)
    p, r_core, r_c, seed, step = 12, 4.5, 6.0, 4, 5
    out = {}
    for span in (1, 3, 6):
        with handle(sy, 32, r_core=r_core, p_rbl=p, r_c=r_c, seed=seed) as h:
            h.set_tuning("rbl_eager", eager)
            h.set_tuning("rbl_span", span)
            F, E, W = h.forces_f64(step)
            out[span] = (F, E, W, *h.neighbor_counts(), h.rbl_partners())
    F1, E1, W1, nc1, ns1, pa1 = out[1]
    for span in (3, 6):
        F, E, W, nc, ns, pa = out[span]
        assert np.array_equal(F, F1) and E == E1 and W == W1
        assert np.array_equal(nc, nc1) and np.array_equal(ns, ns1) and np.array_equal(pa, pa1)
    ref = orc.rbl(sy.s, sy.q, sy.types, sy.box, ALPHA, r_core, r_c, p, seed, step, 0, C,
                  sy.eps, sy.sig)
    assert np.array_equal(nc1, ref["n_core"]) and np.array_equal(ns1, ref["n_shell"])
    assert np.array_equal(pa1, ref["partners"])


def test_rbl_capacity_is_reported_not_faulted():
    """A 27-cell stencil with more candidates than the per-chunk counters hold (6,144) is
    skipped and reported as RBE_ERR_CAPACITY at the next synchronising call."""
    sy = synth.make_system(30000, density=1.5, frac_charged=0.0, seed=10)
    with handle(sy, 8, r_core=3.0, p_rbl=10, r_c=6.0) as h:
        with pytest.raises(binding.RBEError) as e:
            h.forces_f64(0)
        assert e.value.code == -10
        h.check_device()  # the flag was read and cleared: no error now


# -------------------------------------------------------------------------- Verlet


def test_verlet_one_step_matches_oracle(orc):
    sy = synth.make_system(3000, L=32.0, all_charged=True, seed=1)
    dt, kappa = 1.0, synth.ACCEL_KAPPA
    with handle(sy, 100, precision="fp64", dt=dt, kappa=kappa) as h:
        h.step(1)
        pos, vel, s1 = h.state()
    m0, S0 = orc.sample_k(1, 0, 0, sy.box, ALPHA, 100)
    m1, S1 = orc.sample_k(1, 1, 0, sy.box, ALPHA, 100)
    s, v = sy.s.copy(), sy.v.copy()
    F0 = oracle_all(orc, sy, m0, S0)["F"]
    orc.vv_drift(s, v, F0, sy.mass, sy.box, dt, kappa)
    F1 = orc.total_forces(s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig, m1, S1)["F"]
    orc.vv_kick(v, F1, sy.mass, dt, kappa)
    ds = (s1.astype(np.int64) - s.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
    assert np.abs(ds).max() <= 1
    # the FP64 form keeps 1/m in FP32 (relative 1.5e-8 for m = 20)
    assert rel_l2(vel, v) < 1e-7


def test_verlet_shadowing_fp32(orc):
    """After 20 graph-replayed steps, the GPU forces on the GPU's own state match the
    oracle's forces on that state (the trajectory itself is chaotic)."""
    sy = synth.make_system(3000, L=32.0, all_charged=True, seed=1)
    with handle(sy, 100, dt=1.0, kappa=synth.ACCEL_KAPPA) as h:
        h.step(20)
        assert h.step_count() == 20
        pos, vel, s = h.state()
        F, E, W = h.forces_f64(20)
        m, S = sampled.oracle_modes(orc, h, sy, 100, 20)
    sy2 = synth.System(box=sy.box, s=s, q=sy.q, types=sy.types, mass=sy.mass, v=vel,
                       eps=sy.eps, sig=sy.sig)
    ref = oracle_all(orc, sy2, m, S)
    assert rel_l2(F, ref["F"]) < TOL_F32
    assert np.isfinite(E["kinetic"]) and E["kinetic"] > 0


def test_graph_replay_equals_single_steps():
    sy = synth.make_system(5000, density=0.1, frac_charged=0.1, seed=2)
    with handle(sy, 64) as a, handle(sy, 64) as b:
        a.step(6)
        for _ in range(6):
            b.step(1)
        pa, va, _ = a.state()
        pb, vb, _ = b.state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)


# -------------------------------------------------------------------------- full size


@pytest.mark.slow
def test_full_size_one_million_sampled(orc):
    """1,048,576 particles (10% charged, density 0.1, P = 200), the launch configuration
    of the benchmark: forces and neighbour counts of sampled particles against the oracle's
    O(N) sums."""
    sy = synth.make_system(1 << 20, density=0.1, frac_charged=0.1, seed=2)
    with handle(sy, 200) as h:
        F, E, W = h.forces_f64(0)
        nbr, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, 200, 0)
        rho, _ = h.rho()
    idx = sample_ids(sy, 48)
    assert rel_l2(rho, sampled.charged_rho(orc, sy, m)) < 2e-6
    Fo, nbr_o = sampled.total_forces_sampled(orc, sy, idx, m, S)
    assert np.array_equal(nbr[idx], nbr_o)
    assert rel_l2(F[idx], Fo) < TOL_F32


@pytest.fixture(scope="module")
def sys16m():
    return synth.make_system(1 << 24, density=0.1, frac_charged=0.1, seed=3)


@pytest.mark.parametrize("precision,P,tol", [("fp32_comp", 2000, TOL_F32), ("fp32", 500, TOL_F32),
                                             ("fp64", 100, TOL_F64)])
def test_full_size_sixteen_million_sampled(orc, sys16m, precision, P, tol):
    """16,777,216 particles (10% charged, density 0.1) in the three forms of the precision
    sweep: forces and neighbour counts of sampled particles against the oracle's O(N) sums."""
    sy = sys16m
    with handle(sy, P, precision=precision) as h:
        F, E, W = h.forces_f64(0)
        nbr, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, P, 0)
    idx = sample_ids(sy, 32)
    Fo, nbr_o = sampled.total_forces_sampled(orc, sy, idx, m, S)
    assert np.array_equal(nbr[idx], nbr_o)
    assert rel_l2(F[idx], Fo) < tol

def test_full_size_rbl_134m_sampled(orc):
    """134,217,728 particles (5% charged, density 0.1, P = 500, random batch list with
    r_core = 5 A, r_s = 10 A, p = 10, seed 1), in the benchmark's launch configuration. On
    sampled particles: core and shell sizes bit for bit, and the force against the oracle's
    rows of the random batch list plus the k-space force from the oracle's structure factor.
    The mean-force correction (Eq. F_corr) sums all 2^27 rows, which the oracle cannot do in
    a test: it is the one offset common to the sample, and it must be small."""
    sy = synth.make_system(1 << 27, density=0.1, frac_charged=0.05, seed=5)
    p, r_core, seed, step = 10, 5.0, 1, 0
    with handle(sy, 500, r_core=r_core, p_rbl=p, seed=seed) as h:
        F, E, W = h.forces_f64(step)
        nc, ns = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, 500, step, seed=seed)
    idx = sample_ids(sy, 64)
    F, nc, ns = F[idx], nc[idx], ns[idx]
    rows = orc.rbl_rows(sy.s, sy.q, sy.types, sy.box, ALPHA, r_core, RC, p, seed, step, 0, C,
                        sy.eps, sy.sig, idx)
    assert np.array_equal(nc, rows["n_core"])
    assert np.array_equal(ns, rows["n_shell"])
    assert (rows["n_shell"] > p).all()  # every sampled row draws
    Fo = rows["Ft"] + sampled.kspace_force_sampled(sy, idx, m, S,
                                                   sampled.charged_rho(orc, sy, m))
    off = (F - Fo).mean(0)
    assert np.linalg.norm(off) < 1e-2 * np.sqrt((Fo * Fo).sum(1).mean())
    assert rel_l2(F - off, Fo) < TOL_F32


# -------------------------------------------------------------------------- tuning


@pytest.mark.parametrize("test16", [0, 1])
@pytest.mark.parametrize("skw", [dict(N=20000, density=0.1, frac_charged=0.1, seed=2),
                                 dict(N=30000, density=0.05, frac_charged=0.6, seed=4)])
def test_pair_pretest_variants_match_oracle(orc, test16, skw):
    """Both candidate pre-tests (FP32, packed FP16x2) give the oracle's neighbour sets."""
    sy = synth.make_system(**skw)
    with handle(sy, 100) as h:
        h.set_tuning("pair_test16", test16)
        assert h.get_tuning("pair_test16") == test16
        F, E, W = h.forces_f64(0)
        m, S = sampled.oracle_modes(orc, h, sy, 100, 0)
        nbr, _ = h.neighbor_counts()
    ref = oracle_all(orc, sy, m, S)
    assert np.array_equal(nbr, ref["nbr"])
    assert rel_l2(F, ref["F"]) < TOL_F32


def test_autotune_keeps_results(orc):
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=2)
    with handle(sy, 200) as h:
        chosen = h.autotune(2)
        assert chosen["pair_test16"] in (0, 1) and chosen["sf_tile"] % 32 == 0
        F, E, W = h.forces_f64(0)
        m, S = sampled.oracle_modes(orc, h, sy, 200, 0)
        h.step(3)
    ref = oracle_all(orc, sy, m, S)
    assert rel_l2(F, ref["F"]) < TOL_F32


# -------------------------------------------------------------------------- NVT


def test_nvt_one_step_matches_oracle(orc):
    """One Nose-Hoover velocity-Verlet step in the FP64 form against the oracle's half
    steps around its Verlet step (same modes at steps 0 and 1)."""
    sy = synth.make_system(3000, L=32.0, all_charged=True, seed=1, T=200.0)
    dt, kappa, kB, T0, tau = 1.0, synth.ACCEL_KAPPA, synth.BOLTZMANN_KB, 300.0, 20.0
    with handle(sy, 100, precision="fp64", dt=dt, kappa=kappa) as h:
        h.set_thermostat(T0, tau, kB)
        h.step(1)
        pos, vel, s1 = h.state()
        xi, eta, _ = h.thermostat()
    Nf = 3 * sy.n - 3
    Q = Nf * kB * T0 * tau ** 2
    xe = np.zeros(2)
    m0, S0 = orc.sample_k(1, 0, 0, sy.box, ALPHA, 100)
    m1, S1 = orc.sample_k(1, 1, 0, sy.box, ALPHA, 100)
    s, v = sy.s.copy(), sy.v.copy()
    F0 = oracle_all(orc, sy, m0, S0)["F"]
    orc.nh_half(v, sy.mass, kappa, Nf, kB * T0, Q, dt, xe)
    orc.vv_drift(s, v, F0, sy.mass, sy.box, dt, kappa)
    F1 = orc.total_forces(s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig, m1, S1)["F"]
    orc.vv_kick(v, F1, sy.mass, dt, kappa)
    orc.nh_half(v, sy.mass, kappa, Nf, kB * T0, Q, dt, xe)
    ds = (s1.astype(np.int64) - s.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
    assert np.abs(ds).max() <= 1
    assert rel_l2(vel, v) < 1e-7
    # thermostat state at the end of the step equals the oracle's. Each quarter update is
    # (dt/4)(2K - Nf kT)/Q, whose difference 2K - Nf kT cancels near the target, so the
    # comparison is on the scale of one update, dt / tau^2
    assert abs(xi - xe[0]) < 1e-7 * dt / tau ** 2
    assert abs(eta - xe[1]) < 1e-7 * dt * dt / tau ** 2


def test_nvt_thermalises_lj_system():
    """LJ fluid without charges (deterministic forces): the temperature is driven from
    150 K to the 300 K target and the extended energy stays constant."""
    sy = synth.make_system(4000, density=0.03, frac_charged=0.0, seed=2, T=150.0)
    kB = synth.BOLTZMANN_KB
    with handle(sy, 8, dt=1.0, kappa=synth.ACCEL_KAPPA, precision="fp64") as h:
        h.set_thermostat(300.0, 50.0, kB)
        Hs, Ts = [], []
        for _ in range(30):
            h.step(50)
            E, _ = h.energies()
            xi, eta, ext = h.thermostat()
            Nf = 3 * sy.n - 3
            Ts.append(2 * E["kinetic"] / (Nf * kB))
            Hs.append(E["total"] + E["kinetic"] + ext)
    Ts, Hs = np.array(Ts), np.array(Hs)
    assert abs(Ts[-10:].mean() - 300.0) < 30.0
    # plain truncation at r_c makes the extended energy jump by U(r_c) per crossing pair
    assert np.abs(Hs - Hs[0]).max() < 0.02 * abs(Hs[0])


def test_lj_electrolyte_reduced_units(orc):
    """LJ electrolyte settings in reduced units (all ions charged, r_s = 8, r_c = 4, p = 30):
    RBL + RBE forces against the oracle on the same modes and draws."""
    prm = synth.LJ_ELECTROLYTE
    sy = synth.lj_electrolyte(3000)
    with binding.from_system(sy, P=prm["P"], alpha=prm["alpha"], r_c=prm["r_c"],
                             r_core=prm["r_core"], p_rbl=prm["p_rbl"],
                             coulomb_C=prm["coulomb_C"], dt=prm["dt"], kappa=prm["kappa"],
                             seed=9) as h:
        F, E, W = h.forces_f64(3)
        m, S = sampled.oracle_modes(orc, h, sy, prm["P"], 3, seed=9, alpha=prm["alpha"])
        nc, ns = h.neighbor_counts()
    ref = orc.rbl(sy.s, sy.q, sy.types, sy.box, prm["alpha"], prm["r_core"], prm["r_c"],
                  prm["p_rbl"], 9, 3, 0, prm["coulomb_C"], sy.eps, sy.sig)
    Fk, Uk, Wk = orc.rbe_kspace(sy.s, sy.q, sy.box, prm["alpha"], prm["coulomb_C"], m, S)
    assert np.array_equal(nc, ref["n_core"]) and np.array_equal(ns, ref["n_shell"])
    assert rel_l2(F, ref["F"] + Fk) < TOL_F32
    assert E["kspace"] == pytest.approx(Uk, rel=2e-6)
