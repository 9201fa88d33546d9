"""The sampled-particle oracle forces used by the full-size parity tests are rows of the
oracle's all-particle forces (the real-space rows restricted by id, and Eq. F_long_RBE from
the structure factor of the charged particles alone)."""
import numpy as np

from paper_2609_02694_gb300 import synth

import sampled


def test_sampled_forces_are_rows_of_the_total(orc):
    sy = synth.make_system(12000, density=0.1, frac_charged=0.1, seed=2)
    m, S = orc.sample_k(1, 0, 0, sy.box, synth.ALPHA, 100)
    ref = orc.total_forces(sy.s, sy.q, sy.types, sy.box, synth.ALPHA, synth.R_CUT,
                           synth.COULOMB_C, sy.eps, sy.sig, m, S)
    idx = np.unique(np.r_[[0, 5, 17, 4000, 11999], np.flatnonzero(sy.q)[:8]])
    F, nbr = sampled.total_forces_sampled(orc, sy, idx, m, S)
    assert np.array_equal(nbr, ref["nbr"][idx])
    assert np.abs(F - ref["F"][idx]).max() < 1e-12 * np.abs(ref["F"][idx]).max()
    # the k-space part alone: a planted sign error or a dropped charge would show here
    Fk, _, _ = orc.rbe_kspace(sy.s, sy.q, sy.box, synth.ALPHA, synth.COULOMB_C, m, S)
    Fk_s = sampled.kspace_force_sampled(sy, idx, m, S, sampled.charged_rho(orc, sy, m))
    assert np.abs(Fk_s - Fk[idx]).max() < 1e-12 * np.abs(Fk[idx]).max()
