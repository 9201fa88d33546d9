"""GPU parity of the cluster-pair kernel (each pair once, over clusters of 8 particles) against
the FP64 oracle and against the per-particle kernel, through the C ABI.

Neighbour counts (the exact cutoff decision of Eqs. F_i, G_short, LJ) are bit-exact; forces
match the oracle within 1e-5 relative L2 in the FP32 forms and 1e-10 in the FP64 form, on the
oracle's own mode draw. The cases cover the LJ pass beside a separate Coulomb pass, the fused
LJ + Coulomb pass of mostly charged systems, two LJ types in an orthorhombic box whose
super-clusters must be split into narrower groups, ragged particle counts, and cells of r_c,
r_c / 2 and r_c / 3.
"""
import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build, synth

import sampled

pytestmark = pytest.mark.gpu

C, ALPHA, RC = synth.COULOMB_C, synth.ALPHA, synth.R_CUT
TOL = {"fp32_comp": 1e-5, "fp32": 1e-5, "fp64": 1e-10}
ETOL = {"fp32_comp": 2e-6, "fp32": 2e-6, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def two_type(sy, seed=4):
    rng = np.random.default_rng(seed)
    sy.types = (rng.uniform(size=sy.n) < 0.3).astype(np.int32)
    sy.eps = np.array([0.1, 0.15, 0.15, 0.2])
    sy.sig = np.array([3.0, 2.8, 2.8, 2.6])
    return sy


def orthorhombic():
    sy = synth.make_system(6000, L=40.0, frac_charged=0.2, seed=4)
    sy.box = np.array([40.0, 45.0, 52.0])
    return two_type(sy)


SYSTEMS = {
    "n20k_10pct": lambda: synth.make_system(20000, density=0.1, frac_charged=0.1, seed=2),
    "n8000_all_charged": lambda: synth.make_system(8000, L=45.0, all_charged=True, seed=11),
    "ortho_two_types": orthorhombic,
    "n7777_ragged": lambda: synth.make_system(7777, density=0.08, frac_charged=0.3, seed=9),
}


def run(sy, P, precision, cluster, step=0, **kw):
    with binding.from_system(sy, P=P, alpha=ALPHA, r_c=RC, precision=precision, coulomb_C=C,
                             **kw) as h:
        h.set_tuning("pair_cluster", cluster)
        assert h.get_tuning("pair_cluster") == cluster
        F, E, W = h.forces_f64(step)
        nbr, _ = h.neighbor_counts()
        return h, F, E, W, nbr


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("precision", ["fp32_comp", "fp64"])
def test_cluster_pair_matches_oracle(orc, name, precision):
    sy = SYSTEMS[name]()
    P, step = 96, 3
    with binding.from_system(sy, P=P, alpha=ALPHA, r_c=RC, precision=precision,
                             coulomb_C=C) as h:
        h.set_tuning("pair_cluster", 1)
        F, E, W = h.forces_f64(step)
        nbr, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, P, step)
    ref = orc.total_forces(sy.s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig, m, S)
    assert np.array_equal(nbr, ref["nbr"])
    assert rel_l2(F, ref["F"]) < TOL[precision]
    etol = ETOL[precision]
    assert E["lj"] == pytest.approx(ref["U_lj"], rel=etol)
    assert W["lj"] == pytest.approx(ref["W_lj"], rel=etol)
    assert E["real"] == pytest.approx(ref["U_real"], rel=max(etol, 1e-5), abs=1e-6)
    assert W["real"] == pytest.approx(ref["W_real"], rel=max(etol, 1e-5), abs=1e-6)
    assert E["kspace"] == pytest.approx(ref["U_k"], rel=etol)


@pytest.mark.parametrize("sub", [1, 2, 3])
def test_cluster_pair_cell_sizes(orc, sub):
    """Cells of r_c, r_c / 2 and r_c / 3 (stencils of 1, 2 and 3 cells): same neighbour sets."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=7)
    with binding.from_system(sy, P=32, alpha=ALPHA, r_c=RC, coulomb_C=C, cell_sub=sub) as h:
        h.set_tuning("pair_cluster", 1)
        F, E, W = h.forces_f64(0)
        nbr, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, 32, 0)
    ref = orc.total_forces(sy.s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig, m, S)
    assert np.array_equal(nbr, ref["nbr"])
    assert rel_l2(F, ref["F"]) < 1e-5


@pytest.mark.parametrize("precision", ["fp32_comp", "fp32", "fp64"])
def test_cluster_and_particle_kernels_agree(precision):
    """The two traversals of the same cutoff sum: identical neighbour counts, forces equal to
    rounding, and the cluster kernel's forces bit-identical from run to run (fixed-point sums
    do not depend on the order of the atomics)."""
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=5)
    out = {}
    for cl in (0, 1, 1):
        h, F, E, W, nbr = run(sy, 64, precision, cl)
        out.setdefault(cl, []).append((F, E, W, nbr))
    F0, E0, W0, n0 = out[0][0]
    F1, E1, W1, n1 = out[1][0]
    F2, E2, W2, n2 = out[1][1]
    assert np.array_equal(n0, n1) and np.array_equal(n1, n2)
    assert np.array_equal(F1, F2) and E1 == E2 and W1 == W2
    # FP32: the cluster kernel rounds frame coordinates of up to ~25 A from its super-cluster's
    # centre (about 1e-6 A each), the per-particle kernel converts exact integer displacements;
    # each is within 1e-5 of the oracle (test_cluster_pair_matches_oracle)
    tol = 1e-12 if precision == "fp64" else 5e-6
    assert rel_l2(F1, F0) < tol
    assert E1["lj"] == pytest.approx(E0["lj"], rel=tol)
    assert W1["lj"] == pytest.approx(W0["lj"], rel=tol)


def test_cluster_pair_verlet_steps_track_particle_kernel():
    """Ten graph-captured Verlet steps with each traversal stay together to FP32 rounding."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=14)
    vel = {}
    for cl in (0, 1):
        with binding.from_system(sy, P=64, alpha=ALPHA, r_c=RC, coulomb_C=C, dt=1.0,
                                 kappa=synth.ACCEL_KAPPA) as h:
            h.set_tuning("pair_cluster", cl)
            h.step(10)
            _, v, _ = h.state()
            vel[cl] = v
    assert rel_l2(vel[1], vel[0]) < 1e-4


def test_cluster_pair_wide_groups_split(orc):
    """A dilute orthorhombic box whose x edge leaves little room beside 2 r_c (14 A): a
    super-cluster spans far more, so it is split into groups narrow enough for a valid frame
    (down to single particles where one cluster is wider), and every neighbour is kept."""
    sy = synth.make_system(2200, L=34.0, frac_charged=0.2, seed=6)
    sy.box = np.array([34.0, 46.0, 46.0])
    with binding.from_system(sy, P=16, alpha=ALPHA, r_c=RC, coulomb_C=C) as h:
        h.set_tuning("pair_cluster", 1)
        F, E, W = h.forces_f64(1)
        nbr, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, 16, 1)
    ref = orc.total_forces(sy.s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig, m, S)
    assert np.array_equal(nbr, ref["nbr"])
    assert rel_l2(F, ref["F"]) < 1e-5


def test_switching_passes_keeps_energies(orc):
    """The energy totals sum every per-block partial slot of a pass. Switching one handle
    between the per-particle kernel, the cluster kernel and the Verlet list (whose grids write
    different numbers of slots) leaves the same energies as a fresh handle, and the oracle's."""
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=8)
    P = 64

    def fresh(cl):
        with binding.from_system(sy, P=P, alpha=ALPHA, r_c=RC, coulomb_C=C) as h:
            h.set_tuning("pair_cluster", cl)
            return h.forces_f64(2)[1:]

    E_cl, W_cl = fresh(1)
    E_pp, W_pp = fresh(0)
    with binding.from_system(sy, P=P, alpha=ALPHA, r_c=RC, coulomb_C=C) as h:
        h.set_tuning("pair_cluster", 0)
        h.forces_f64(2)
        h.set_tuning("pair_cluster", 1)
        _, E1, W1 = h.forces_f64(2)
        h.set_neighbor_list(1.0)
        h.forces_f64(2)
        h.set_neighbor_list(0.0)
        _, E2, W2 = h.forces_f64(2)
        h.set_tuning("pair_cluster", 0)
        _, E3, W3 = h.forces_f64(2)
        m, S = sampled.oracle_modes(orc, h, sy, P, 2)
    assert E1 == E_cl and W1 == W_cl
    assert E2 == E_cl and W2 == W_cl
    assert E3 == E_pp and W3 == W_pp
    ref = orc.total_forces(sy.s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig, m, S)
    assert E1["lj"] == pytest.approx(ref["U_lj"], rel=2e-6)
    assert E1["real"] == pytest.approx(ref["U_real"], rel=1e-5)


@pytest.mark.parametrize("precision,frac", [("fp32_comp", 0.1), ("fp64", 0.1), ("fp32_comp", 0.8)])
def test_two_branch_step_graph_equals_sequential(precision, frac):
    """With profiling off, a captured step of the cluster kernel runs the k-space chain and the
    charged subset's Coulomb pass as a second graph branch beside the pair pass, all adding to
    the same integer fixed-point sums; with profiling on, the phases run one after another.
    Both give the same state and energies bit for bit after several steps, and so do a
    captured and an uncaptured force evaluation (frac 0.8: the fused LJ + Coulomb pass, with
    only the k-space chain beside it)."""
    sy = synth.make_system(15000, density=0.1, frac_charged=frac, seed=43)
    out = []
    for prof in (False, True):
        with binding.from_system(sy, P=64, alpha=ALPHA, r_c=RC, coulomb_C=C, dt=1.0,
                                 kappa=synth.ACCEL_KAPPA, precision=precision, seed=9) as h:
            h.set_tuning("pair_cluster", 1)
            h.set_profiling(prof)
            F0, E0, W0 = h.forces(0)  # a force evaluation alone (a captured one, unprofiled)
            h.step(6)
            s, v, _ = h.state()
            out.append((s, v, h.energies(), F0, E0, W0))
            if prof:
                ph = h.profile()[0]
                assert ph["pair"] > 0 and ph["tail"] > 0  # (the tail holds the finish)
    (s0, v0, e0, F0, E0, W0), (s1, v1, e1, F1, E1, W1) = out
    assert np.array_equal(s0, s1) and np.array_equal(v0, v1)
    assert e0 == e1
    assert np.array_equal(F0, F1) and E0 == E1 and W0 == W1


def test_replayed_force_evaluations_follow_new_positions():
    """rbe_forces replays a captured evaluation (one graph per buffer parity). Fed a sequence
    of new positions through rbe_set_positions, it gives the same forces and energies bit for
    bit as the uncaptured evaluation (profiling on) on a second handle, at both parities."""
    sy = synth.make_system(15000, density=0.1, frac_charged=0.1, seed=47)
    rng = np.random.default_rng(5)
    x0 = sy.positions()
    moves = [x0 + rng.normal(scale=s, size=x0.shape) for s in (0.0, 0.02, 0.1, 0.05, 0.15)]
    res = []
    for prof in (False, True):
        with binding.from_system(sy, P=64, alpha=ALPHA, r_c=RC, coulomb_C=C, seed=3) as h:
            h.set_tuning("pair_cluster", 1)
            h.set_profiling(prof)
            out = []
            for k, x in enumerate(moves):
                h.set_positions(x)
                out.append(h.forces(10 + k))
            res.append(out)
    for (F0, E0, W0), (F1, E1, W1) in zip(*res):
        assert np.array_equal(F0, F1) and E0 == E1 and W0 == W1
    # and they are forces of those positions: the last evaluation against a fresh handle
    sy2 = synth.make_system(15000, density=0.1, frac_charged=0.1, seed=47)
    with binding.from_system(sy2, P=64, alpha=ALPHA, r_c=RC, coulomb_C=C, seed=3) as h:
        h.set_tuning("pair_cluster", 1)
        h.set_positions(moves[-1])
        F2, E2, _ = h.forces(10 + len(moves) - 1)
    assert np.array_equal(F2, res[0][-1][0]) and E2 == res[0][-1][1]
