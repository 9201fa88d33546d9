"""Checkpoint and resume through the C ABI (rbe_save / rbe_load).

Every mode and random-batch draw is a pure function of (seed, replica, step) and the cell
order a pure function of the positions, so a run that is saved, torn down and resumed in a
new handle continues bit for bit as the uninterrupted run: positions, velocities, energies
and the thermostat state are compared exactly.
"""
import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def cell_handle(sy, precision):
    return binding.from_system(sy, P=64, alpha=synth.ALPHA, r_c=synth.R_CUT,
                               coulomb_C=synth.COULOMB_C, dt=1.0, kappa=synth.ACCEL_KAPPA,
                               precision=precision, seed=7)


def rbl_nvt_handle(sy):
    prm = synth.LJ_ELECTROLYTE
    h = binding.from_system(sy, P=prm["P"], alpha=prm["alpha"], r_c=prm["r_c"],
                            r_core=prm["r_core"], p_rbl=prm["p_rbl"],
                            coulomb_C=prm["coulomb_C"], dt=prm["dt"], kappa=prm["kappa"], seed=3)
    h.set_thermostat(prm["T"], prm["tau"], prm["kB"])
    return h


CASES = {
    "cells_fp32_comp": (lambda: synth.make_system(6000, density=0.1, frac_charged=0.1, seed=31),
                        lambda sy: cell_handle(sy, "fp32_comp")),
    "cells_fp64": (lambda: synth.make_system(3000, density=0.1, frac_charged=0.1, seed=32),
                   lambda sy: cell_handle(sy, "fp64")),
    "rbl_nvt_ljelec": (lambda: synth.lj_electrolyte(4000), rbl_nvt_handle),
}


@pytest.mark.parametrize("name", list(CASES))
def test_resume_is_bit_identical(tmp_path, name):
    make_sys, make_h = CASES[name]
    sy = make_sys()
    n1, n2 = 4, 5
    with make_h(sy) as a:
        a.step(n1 + n2)
        pa, va, sa = a.state()
        ea, wa = a.energies()
        ta = a.thermostat() if name.startswith("rbl") else None
    path = str(tmp_path / "state.ckpt")
    with make_h(sy) as b:
        b.step(n1)
        b.save(path)
    with make_h(sy) as c:  # a new handle from the initial system, then the saved state
        c.load(path)
        assert c.step_count() == n1
        c.step(n2)
        assert c.step_count() == n1 + n2
        pc, vc, sc = c.state()
        ec, wc = c.energies()
        tc = c.thermostat() if name.startswith("rbl") else None
    assert np.array_equal(sa, sc)
    assert np.array_equal(va, vc)
    assert ea == ec and wa == wc
    assert ta == tc


def test_load_refuses_other_systems(tmp_path):
    sy = synth.make_system(3000, density=0.1, frac_charged=0.1, seed=33)
    path = str(tmp_path / "state.ckpt")
    with cell_handle(sy, "fp32_comp") as h:
        h.step(1)
        h.save(path)
    with cell_handle(sy, "fp64") as h:  # another precision: another fingerprint
        with pytest.raises(binding.RBEError) as e:
            h.load(path)
        assert e.value.code == -9
    other = synth.make_system(3001, density=0.1, frac_charged=0.1, seed=33)
    with cell_handle(other, "fp32_comp") as h:  # another particle count
        with pytest.raises(binding.RBEError) as e:
            h.load(path)
        assert e.value.code == -9
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint")
    with cell_handle(sy, "fp32_comp") as h:
        with pytest.raises(binding.RBEError) as e:
            h.load(str(bad))
        assert e.value.code == -1
        with pytest.raises(binding.RBEError):
            h.load(str(tmp_path / "missing.ckpt"))
        h.step(1)  # the handle stays usable
