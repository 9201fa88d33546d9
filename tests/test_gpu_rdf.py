"""Ion-ion radial distribution functions of the LJ electrolyte under random batch Ewald with the
random batch list, against the oracle's deterministic reference (Sec. 3.2, Fig. rdf).

The GPU run uses Table 1's parameters (r_s = 8, r_c = 4, p = 30, P = 200; alpha = 0.15, C = 1 in
this build's reading) with a Nose-Hoover thermostat at T = 1. The reference
(tests/golden/rdf_ljelec_n2000.txt, written by tests/golden/make_rdf_ljelec.py from the
oracle alone) samples the same model, LJ truncated at 8 plus the full Coulomb sum, with no
random batches. The cation-cation, anion-anion and cation-anion RDFs must agree within
their combined statistical errors (block averages on both sides).
"""
import importlib.util
import os

import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
REF = os.path.join(HERE, "golden", "rdf_ljelec_n2000.txt")


def _ref_module():
    spec = importlib.util.spec_from_file_location(
        "make_rdf_ljelec", os.path.join(HERE, "golden", "make_rdf_ljelec.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def test_ljelec_rdfs_match_full_ewald_reference():
    mk = _ref_module()
    ref = np.loadtxt(REF)
    edges = np.r_[ref[:, 0], ref[-1, 1]]
    prm = synth.LJ_ELECTROLYTE
    sy = synth.lj_electrolyte(mk.N)
    npos, nneg = int((sy.q > 0).sum()), int((sy.q < 0).sum())
    V = float(np.prod(sy.box))
    n_eq, n_frames, every, n_blocks = 3000, 480, 50, 8
    with binding.from_system(sy, P=prm["P"], alpha=prm["alpha"], r_c=prm["r_c"],
                             r_core=prm["r_core"], p_rbl=prm["p_rbl"],
                             coulomb_C=prm["coulomb_C"], dt=mk.DT, kappa=prm["kappa"],
                             seed=11) as h:
        h.set_thermostat(mk.T0, mk.TAU, 1.0)
        h.step(n_eq)
        frames = []
        for _ in range(n_frames):
            h.step(every)
            _, _, s = h.state()
            frames.append(mk.pair_histograms(s, sy.q, sy.box, edges))
        E, _ = h.energies()
    T = 2 * E["kinetic"] / (3 * mk.N - 3)
    assert abs(T - mk.T0) < 0.1
    frames = np.array(frames)
    blocks = [mk.rdf_from_counts(list(fr.sum(0)), len(fr), npos, nneg, V, edges)
              for fr in np.array_split(frames, n_blocks)]
    g = np.array([np.mean([b[k] for b in blocks], axis=0) for k in range(3)])
    e = np.array([np.std([b[k] for b in blocks], axis=0, ddof=1) / np.sqrt(n_blocks)
                  for k in range(3)])
    gr = ref[:, [2, 4, 6]].T
    er = ref[:, [3, 5, 7]].T
    r = 0.5 * (edges[1:] + edges[:-1])
    # bins outside the excluded core (reference g above 0.2) up to r = 6
    use = (gr > 0.2) & (r[None, :] <= 6.0)
    z = (g - gr)[use] / np.sqrt(er[use] ** 2 + e[use] ** 2 + 1e-12)
    assert use.sum() > 200
    assert np.abs(z).max() < 5.0, f"largest deviation {np.abs(z).max():.2f} sigma"
    assert np.mean(z ** 2) < 2.5, f"chi2 per bin {np.mean(z ** 2):.2f}"
    # the contact peak of the cation-anion RDF and the depletion of like ions at contact
    pk = (r > 0.9) & (r < 1.4)
    assert abs(g[2][pk].max() - gr[2][pk].max()) < 5 * np.sqrt(
        e[2][pk][np.argmax(g[2][pk])] ** 2 + er[2][pk][np.argmax(gr[2][pk])] ** 2)
