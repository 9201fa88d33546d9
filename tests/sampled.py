"""Oracle forces of a sample of particles in a system too large for the oracle's all-pairs
and all-particle sums, for the full-size parity tests.

The real-space part is the oracle's cutoff sum restricted to the sampled rows (O(N) per
row). The k-space part is Eq. F_long_RBE for the sampled particles. It uses the oracle's
structure factor over the charged particles only: zero charges add exact zeros to rho, so
the sums are the same.
"""
import numpy as np

from paper_2609_02694_gb300 import synth


def kspace_force_sampled(sy, idx, m, S, rho, C=synth.COULOMB_C):
    """k-space force (Eq. F_long_RBE, with the minus sign of Eq. F_i) of the particles idx,
    from the mode set m, its normalisation S and a structure factor rho."""
    k = 2 * np.pi * np.asarray(m, np.float64) / sy.box
    k2 = (k * k).sum(1)
    V = np.prod(sy.box)
    r = sy.s[idx].astype(np.float64) * (sy.box / synth.TWO32)
    th = r @ k.T
    im = rho.imag[None, :] * np.cos(th) - rho.real[None, :] * np.sin(th)
    c = (S / len(m)) * 4 * np.pi * C / (V * k2)
    return -(sy.q[idx][:, None, None] * (c * im)[:, :, None] * k[None, :, :]).sum(1)


def charged_rho(orc, sy, m):
    """The oracle's structure factor, summed over the charged particles (ascending id)."""
    ch = np.flatnonzero(sy.q != 0)
    return orc.rho(sy.s[ch], sy.q[ch], sy.box, m)


def total_forces_sampled(orc, sy, idx, m, S, alpha=synth.ALPHA, rc=synth.R_CUT,
                         C=synth.COULOMB_C):
    """Real-space cutoff sum plus RBE k-space force of the particles idx, and their exact
    neighbour counts."""
    rs = orc.real_space(sy.s, sy.q, sy.types, sy.box, alpha, rc, C, sy.eps, sy.sig, i_list=idx)
    F = rs["F"][idx] + kspace_force_sampled(sy, idx, m, S, charged_rho(orc, sy, m), C)
    return F, rs["nbr"][idx]


def oracle_modes(orc, h, sy, P, step, seed=1, replica=0, alpha=synth.ALPHA):
    """The oracle's own draw of a step's modes (the sampling density of Eq. F_long_RBE),
    after checking that the GPU drew exactly the same set and normaliser. A force test
    then hands the oracle its own modes, so a sampler fault at any box, seed or step
    fails the test instead of being copied into the reference."""
    mo, So = orc.sample_k(seed, step, replica, np.asarray(sy.box, np.float64), alpha, P)
    m, S = h.sample_k(step)
    assert np.array_equal(m, mo), "GPU mode set differs from the oracle's draw"
    assert S == So, "GPU normaliser S differs from the oracle's"
    return mo, So
