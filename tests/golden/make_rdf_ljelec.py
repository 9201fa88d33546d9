"""Reference radial distribution functions of the LJ electrolyte from an oracle trajectory.

The paper checks its random batch Ewald and random batch list setup by the ion-ion RDFs of
the LJ electrolyte (Sec. 3.2, Fig. rdf; system of Sec. 3.1, parameters r_s = 8, r_c = 4,
p = 30, P = 200 of Table 1), compared with a reference run of a mesh solver at a 1e-4
tolerance. This script writes the reference side for this repository: a Nose-Hoover NVT
trajectory of the same model computed entirely by the FP64 oracle, with the Coulomb sum
evaluated deterministically (no sampling):

  - LJ (eps = sigma = 1) truncated at r_s = 8, as in the random batch list run;
  - Coulomb (C = 1, unit charges) by Ewald splitting at alpha = 0.0096 with a real-space
    cutoff of 28 (erfc(sqrt(alpha) 28) = 1.1e-4) and the Fourier sum over the modes of
    weight exp(-k^2/4 alpha) >= 1e-6 (oracle.ewald_kspace_tol). The total Coulomb force does
    not depend on alpha (pinned by the oracle's alpha-invariance test), so this splitting,
    chosen for the oracle's cost, samples the same model as the GPU's alpha = 0.15.

System: 2,000 ions (1,000 of each sign) at the density of 200,000 ions in L = 271 (L = 58.39),
mass 1, T = 1, from the seeded LJ-electrolyte generator. Integration: the library's NVT
splitting (a Nose-Hoover half step, velocity Verlet, a half step), dt = 0.005, tau = 0.1.
Equilibration 3,000 steps, then 16,000 steps with a frame every 20 steps; RDFs in bins of
0.05 up to r = 8, with standard errors from 8 blocks of 100 frames.

Run from the repository root:  python tests/golden/make_rdf_ljelec.py
(about 20 minutes on 8 cores). It calls only the oracle and the input generator.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2609_02694_gb300 import synth  # noqa: E402

N = 2000
DT, TAU, T0 = 0.005, 0.1, 1.0
R_LJ = 8.0
ALPHA_REF, RC_REF, TOL_REF = 0.0096, 28.0, 1e-6
N_EQ, N_PROD, EVERY, N_BLOCKS = 3000, 16000, 20, 8
DR, R_MAX = 0.05, 8.0
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rdf_ljelec_n2000.txt")


def forces(sy, s):
    """LJ truncated at r_s plus the full Coulomb force (Ewald splitting, truncated Fourier
    sum); C = 1, kappa = 1."""
    qz = np.zeros_like(sy.q)
    lj = oracle.real_space(s, qz, sy.types, sy.box, ALPHA_REF, R_LJ, 1.0, sy.eps, sy.sig)
    co = oracle.real_space(s, sy.q, sy.types, sy.box, ALPHA_REF, RC_REF, 1.0,
                           np.zeros_like(sy.eps), sy.sig)
    fk, _, _ = oracle.ewald_kspace_tol(s, sy.q, sy.box, ALPHA_REF, 1.0, TOL_REF)
    return lj["F"] + co["F"] + fk


def pair_histograms(s, q, box, edges):
    """Unordered pair counts per bin for (+,+), (-,-) and (+,-), minimum image."""
    r = s.astype(np.float64) * (box / 2.0 ** 32)
    out = []
    pos, neg = r[q > 0], r[q < 0]
    for a, b, same in ((pos, pos, True), (neg, neg, True), (pos, neg, False)):
        d = a[:, None, :] - b[None, :, :]
        d -= box * np.round(d / box)
        dist = np.sqrt((d * d).sum(-1))
        if same:
            dist = dist[np.triu_indices(len(a), 1)]
        else:
            dist = dist.ravel()
        out.append(np.histogram(dist, bins=edges)[0].astype(np.float64))
    return out


def rdf_from_counts(counts, n_frames, npos, nneg, V, edges):
    """g(r) = counts / (frames * pair density * shell volume)."""
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    norms = (npos * (npos - 1) / 2 / V, nneg * (nneg - 1) / 2 / V, npos * nneg / V)
    return [c / (n_frames * n * shell) for c, n in zip(counts, norms)]


def main(n_eq=N_EQ, n_prod=N_PROD, out=OUT):
    oracle.lib()
    sy = synth.lj_electrolyte(N)
    s, v = sy.s.copy(), sy.v.copy()
    box, V = sy.box, float(np.prod(sy.box))
    Nf = 3 * N - 3
    Q = Nf * T0 * TAU ** 2
    xe = np.zeros(2)
    edges = np.arange(0.0, R_MAX + 1e-9, DR)
    npos, nneg = int((sy.q > 0).sum()), int((sy.q < 0).sum())
    F = forces(sy, s)
    frames = []  # per-frame pair counts (3 x bins)
    t0 = time.time()
    for step in range(n_eq + n_prod):
        oracle.nh_half(v, sy.mass, 1.0, Nf, T0, Q, DT, xe)
        oracle.vv_drift(s, v, F, sy.mass, box, DT, 1.0)
        F = forces(sy, s)
        oracle.vv_kick(v, F, sy.mass, DT, 1.0)
        oracle.nh_half(v, sy.mass, 1.0, Nf, T0, Q, DT, xe)
        if step >= n_eq and (step - n_eq + 1) % EVERY == 0:
            frames.append(pair_histograms(s, sy.q, box, edges))
        if step % 1000 == 0:
            T = (sy.mass[:, None] * v * v).sum() / Nf
            print(f"step {step} T {T:.3f} ({time.time() - t0:.0f} s)", flush=True)
    frames = np.array(frames)  # (frames, 3, bins)
    blocks = [rdf_from_counts(list(fr.sum(0)), len(fr), npos, nneg, V, edges)
              for fr in np.array_split(frames, N_BLOCKS)]
    g = [np.mean([b[k] for b in blocks], axis=0) for k in range(3)]
    e = [np.std([b[k] for b in blocks], axis=0, ddof=1) / np.sqrt(len(blocks)) for k in range(3)]
    with open(out, "w") as f:
        f.write("# Ion-ion RDFs of the LJ electrolyte (Sec. 3.2, Fig. rdf; Sec. 3.1; Table 1 "
                "parameters on the GPU side), reference from the FP64 oracle.\n")
        f.write(f"# Written by tests/golden/make_rdf_ljelec.py: N = {N}, L = {box[0]:.6f}, "
                f"LJ eps = sigma = 1 truncated at {R_LJ}, C = 1, Ewald alpha = {ALPHA_REF}, "
                f"real-space cutoff {RC_REF}, Fourier modes of weight >= {TOL_REF}, NVT T = "
                f"{T0}, tau = {TAU}, dt = {DT}, {n_eq} + {n_prod} steps, frame every {EVERY}, "
                f"{len(blocks)} blocks.\n")
        f.write("# columns: r_lo r_hi g_pp err_pp g_mm err_mm g_pm err_pm\n")
        for b in range(len(edges) - 1):
            f.write(f"{edges[b]:.3f} {edges[b + 1]:.3f} " +
                    " ".join(f"{g[k][b]:.6f} {e[k][b]:.6f}" for k in range(3)) + "\n")
    print("wrote", out, f"({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "--quick":  # a short trial run into another file
        main(n_eq=20, n_prod=160, out=sys.argv[2])
    else:
        main()
