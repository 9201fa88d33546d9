"""Verlet neighbour list with skin against the oracle and against the cell traversal.

The list is an alternative traversal of the same real-space sum: forces match the FP64
oracle to the FP32 tolerance, and neighbour counts (the exact cutoff decision) are
bit-exact. Rebuilds are decided on the device from the displacements since the last
build."""
import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build, synth

import sampled

pytestmark = pytest.mark.gpu

ALPHA, RC, C = synth.ALPHA, synth.R_CUT, synth.COULOMB_C
TOL_F32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def handle(sy, P, precision="fp32_comp", **kw):
    return binding.from_system(sy, P=P, alpha=kw.pop("alpha", ALPHA), r_c=kw.pop("r_c", RC),
                               precision=precision, coulomb_C=C, **kw)


def oracle_all(orc, sy, m, S):
    return orc.total_forces(sy.s, sy.q, sy.types, sy.box, ALPHA, RC, C, sy.eps, sy.sig, m, S)


@pytest.mark.parametrize("kind,precision,tol", [
    ("10pct", "fp32_comp", TOL_F32),
    ("10pct", "fp64", 1e-10),
    ("all_charged", "fp32_comp", TOL_F32),
    ("two_types", "fp32", TOL_F32),
])
def test_list_forces_match_oracle(orc, kind, precision, tol):
    if kind == "all_charged":
        sy = synth.make_system(8000, L=45.0, all_charged=True, seed=11)
    else:
        sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=12)
    if kind == "two_types":
        rng = np.random.default_rng(5)
        sy.types = (rng.uniform(size=sy.n) < 0.4).astype(np.int32)
        sy.eps = np.array([0.1, 0.15, 0.15, 0.2])
        sy.sig = np.array([3.0, 2.8, 2.8, 2.6])
    with handle(sy, 120, precision=precision) as h:
        h.set_neighbor_list(1.0)
        F, E, W = h.forces_f64(3)
        nbr, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, 120, 3)
        st = h.neighbor_list_stats()
    ref = oracle_all(orc, sy, m, S)
    assert rel_l2(F, ref["F"]) < tol
    assert np.array_equal(nbr, ref["nbr"])
    etol = 1e-10 if precision == "fp64" else 2e-6
    assert E["lj"] == pytest.approx(ref["U_lj"], rel=etol)
    assert E["real"] == pytest.approx(ref["U_real"], rel=max(etol, 1e-5), abs=1e-6)
    assert st["builds"] == 1 and st["evaluations"] == 1
    assert 0 < st["max_len"] <= st["capacity"]


def test_list_and_cells_agree_over_steps(orc):
    """A hot system with a thin skin: the list is rebuilt several times on the device; the
    state after the steps gives the same forces as the cell traversal and the oracle."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=13, T=3000.0)
    with handle(sy, 64, dt=1.0, kappa=synth.ACCEL_KAPPA) as h:
        h.set_neighbor_list(0.3)
        h.step(12)
        st = h.neighbor_list_stats()
        pos, vel, s = h.state()
        F_list, E_list, _ = h.forces_f64(12)
        nbr_list, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, 64, 12)
    assert st["evaluations"] == 13  # the first step's priming force evaluation + 12 steps
    assert 2 <= st["builds"] < st["evaluations"]
    sy2 = synth.System(box=sy.box, s=s, q=sy.q, types=sy.types, mass=sy.mass, v=vel,
                       eps=sy.eps, sig=sy.sig)
    with handle(sy2, 64) as hc:
        F_cell, E_cell, _ = hc.forces_f64(12)
        nbr_cell, _ = hc.neighbor_counts()
    assert np.array_equal(nbr_list, nbr_cell)
    # the list kernel converts exact integer displacements; the cell traversal's cluster kernel
    # rounds frame coordinates of up to ~25 A (about 1e-6 A each); both are within 1e-5 of the
    # oracle (below)
    assert rel_l2(F_list, F_cell) < 5e-6
    ref = oracle_all(orc, sy2, m, S)
    assert rel_l2(F_list, ref["F"]) < TOL_F32
    assert np.array_equal(nbr_list, ref["nbr"])


def test_list_trajectory_tracks_cells():
    """Ten graph-replayed steps with and without the list stay together to FP32 rounding."""
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=14)
    out = {}
    for skin in (0.0, 1.0):
        with handle(sy, 64, dt=1.0, kappa=synth.ACCEL_KAPPA) as h:
            h.set_neighbor_list(skin)
            h.step(10)
            pos, vel, s = h.state()
            E, _ = h.energies()
            out[skin] = (vel, E["total"])
    assert rel_l2(out[1.0][0], out[0.0][0]) < 1e-4
    assert out[1.0][1] == pytest.approx(out[0.0][1], rel=1e-5)


def test_set_positions_rebuilds_only_when_moved(orc):
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=15)
    other = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=16)
    rng = np.random.default_rng(3)
    with handle(sy, 64) as h:
        h.set_neighbor_list(1.0)
        h.forces_f64(0)
        h.forces_f64(0)
        assert h.neighbor_list_stats()["builds"] == 1   # nothing moved
        h.set_positions(sy.positions() + rng.uniform(-0.2, 0.2, size=(sy.n, 3)))
        h.forces_f64(0)
        assert h.neighbor_list_stats()["builds"] == 1   # every move < skin / 2
        h.set_positions(other.positions())
        F, E, W = h.forces_f64(0)
        nbr, _ = h.neighbor_counts()
        m, S = sampled.oracle_modes(orc, h, sy, 64, 0)
        assert h.neighbor_list_stats()["builds"] == 2
    sy3 = synth.System(box=sy.box, s=other.s, q=sy.q, types=sy.types, mass=sy.mass, v=sy.v,
                       eps=sy.eps, sig=sy.sig)
    ref = oracle_all(orc, sy3, m, S)
    assert rel_l2(F, ref["F"]) < TOL_F32
    assert np.array_equal(nbr, ref["nbr"])


def test_list_errors():
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=17)
    with handle(sy, 32) as h:
        with pytest.raises(binding.RBEError) as e:
            h.set_neighbor_list(-1.0)
        assert e.value.code == -1
        with pytest.raises(binding.RBEError) as e:
            h.set_neighbor_list(20.0)      # r_c + skin >= L / 2
        assert e.value.code == -3
        h.set_neighbor_list(1.0, capacity=16)
        with pytest.raises(binding.RBEError) as e:
            h.forces_f64(0)
        assert e.value.code == -10
        h.set_neighbor_list(0.0)           # back to cells: usable again
        h.forces_f64(0)
    with handle(sy, 32, r_core=5.0, p_rbl=10) as h:
        with pytest.raises(binding.RBEError) as e:
            h.set_neighbor_list(1.0)
        assert e.value.code == -9
    small = synth.make_system(3000, L=32.0, all_charged=True, seed=1)
    with handle(small, 32) as h:
        with pytest.raises(binding.RBEError) as e:
            h.set_neighbor_list(1.0)       # 6 cells per axis, stencil needs 7
        assert e.value.code == -4
