"""Seeded synthetic inputs for the RBE force path (charged Lennard-Jones systems).

This module only draws inputs -- positions, charges, types, masses, velocities and the
size mix of batched replicas. It holds none of the method's arithmetic. The GPU library
and the FP64 oracle both take their inputs from here.

Positions come out on the 2^-32 fractional grid: s = uint32 with r = s * L / 2^32
exactly, so both sides see bit-identical coordinates.

The paper's benchmark systems (LJ electrolyte, SPC/E water, PEO-LiTFSI; Sec. 3.1) need
topologies and force-field files that are not available here. Seeded charged-LJ systems
of the same density and charge mix stand in for them.

Recipe (jittered simple-cubic lattice): a lattice of n^3 >= N sites of spacing L/n is
laid in the box. N sites are chosen by a random permutation, and each coordinate is
displaced by a uniform jitter in [-j, j]. floor(f N / 2) particles of each sign get
+/-1 e. The rest are neutral. Every particle has a single LJ type. Velocities are
Maxwell-Boltzmann at temperature T, with the centre-of-mass drift removed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Real units: Angstrom, fs, amu, kcal/mol, e.
COULOMB_C = 332.06371          # kcal Angstrom / (mol e^2)
BOLTZMANN_KB = 0.0019872067    # kcal / (mol K)
ACCEL_KAPPA = 4.184e-4         # (kcal/mol/Angstrom)/amu -> Angstrom/fs^2
TWO32 = 4294967296.0


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.uint64(seed) ^ np.uint64(stream << 32)))


@dataclass
class System:
    """One periodic box of point particles; positions on the 2^-32 fractional grid."""
    box: np.ndarray            # (3,) float64, Angstrom
    s: np.ndarray              # (N, 3) uint32 fractional coordinates
    q: np.ndarray              # (N,) float64 charges (e)
    types: np.ndarray          # (N,) int32 LJ type index
    mass: np.ndarray           # (N,) float64 amu
    v: np.ndarray              # (N, 3) float64 Angstrom/fs
    eps: np.ndarray            # (ntypes*ntypes,) kcal/mol
    sig: np.ndarray            # (ntypes*ntypes,) Angstrom
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.s.shape[0])

    @property
    def ntypes(self) -> int:
        return int(round(math.sqrt(self.eps.size)))

    def positions(self) -> np.ndarray:
        """Positions in Angstrom (exact on the grid)."""
        return self.s.astype(np.float64) * (self.box / TWO32)


def jittered_lattice(N: int, box, rng: np.random.Generator, jitter: float) -> np.ndarray:
    """N distinct sites of an n^3 simple-cubic lattice, each jittered by U[-j, j] per axis,
    returned as uint32 fractional coordinates."""
    box = np.asarray(box, np.float64)
    n = int(math.ceil(N ** (1.0 / 3.0) - 1e-9))
    while n ** 3 < N:
        n += 1
    sites = rng.permutation(n ** 3)[:N]
    idx = np.stack([sites % n, (sites // n) % n, sites // (n * n)], axis=1).astype(np.float64)
    r = (idx + 0.5) * (box / n) + rng.uniform(-jitter, jitter, size=(N, 3))
    frac = np.mod(r / box, 1.0)
    s = np.floor(frac * TWO32)
    s = np.where(s >= TWO32, 0.0, s)
    return s.astype(np.uint32)


def maxwell_velocities(mass: np.ndarray, T: float, rng: np.random.Generator,
                       kB: float = BOLTZMANN_KB, kappa: float = ACCEL_KAPPA) -> np.ndarray:
    """Maxwell-Boltzmann velocities at temperature T (kB, kappa give the unit system; the
    defaults are real units, Angstrom/fs), zero total momentum."""
    sd = np.sqrt(kB * T * kappa / mass)
    v = rng.standard_normal((mass.size, 3)) * sd[:, None]
    p = (v * mass[:, None]).sum(axis=0) / mass.sum()
    return v - p[None, :]


def make_system(N: int, *, density: float | None = None, L: float | None = None,
                frac_charged: float = 0.1, all_charged: bool = False, seed: int = 1,
                T: float = 300.0, mass: float = 20.0, eps: float = 0.1, sigma: float = 3.0,
                jitter: float = 0.1, kB: float = BOLTZMANN_KB,
                kappa: float = ACCEL_KAPPA) -> System:
    """A cubic box of N particles at the given number density (or side L)."""
    if L is None:
        if density is None:
            raise ValueError("give density or L")
        L = (N / density) ** (1.0 / 3.0)
    box = np.array([L, L, L], np.float64)
    rng = _rng(seed, 0)
    s = jittered_lattice(N, box, rng, jitter)
    q = np.zeros(N, np.float64)
    if all_charged:
        nq = N // 2
    else:
        nq = int(math.floor(frac_charged * N / 2.0))
    charged = rng.permutation(N)[: 2 * nq]
    q[charged[:nq]] = 1.0
    q[charged[nq:]] = -1.0
    types = np.zeros(N, np.int32)
    m = np.full(N, mass, np.float64)
    v = maxwell_velocities(m, T, _rng(seed, 1), kB, kappa)
    return System(box=box, s=s, q=q, types=types, mass=m, v=v,
                  eps=np.array([eps], np.float64), sig=np.array([sigma], np.float64),
                  meta=dict(N=N, L=L, density=N / L ** 3, n_plus=nq, n_minus=nq, seed=seed,
                            T=T, jitter=jitter))


def sub_box(N: int = 65536, density: float = 0.1, frac_charged: float = 0.1,
            seed: int = 3) -> System:
    """The 65,536-particle box of the same composition used for precision-sweep errors."""
    return make_system(N, density=density, frac_charged=frac_charged, seed=seed)


def lj_electrolyte(N: int = 200000, density: float = 200000 / 271.0 ** 3, seed: int = 6) -> System:
    """Implicit-solvent LJ electrolyte in LJ reduced units (Sec. 3.1): N monovalent ions, half
    of each sign, eps = sigma = m = kB = 1, T = 1, at the density of 200,000 ions in L = 271."""
    return make_system(N, density=density, all_charged=True, seed=seed, T=1.0, mass=1.0,
                       eps=1.0, sigma=1.0, jitter=0.1, kB=1.0, kappa=1.0)


# Reduced-unit parameters of the LJ electrolyte (Table 1: r_s = 8, r_c = 4, p = 30, P = 200).
# The paper gives no Coulomb strength or splitting parameter for it: C = 1 (unit charges in
# reduced units) and alpha = 0.15 (erfc(sqrt(alpha) r_s) = 1.2e-5) are this build's reading.
LJ_ELECTROLYTE = dict(coulomb_C=1.0, alpha=0.15, r_c=8.0, r_core=4.0, p_rbl=30, P=200,
                      dt=0.001, kappa=1.0, kB=1.0, T=1.0, tau=0.1)


def replica_sizes(n_rep: int = 96, lo: int = 2000, hi: int = 250000, seed: int = 4) -> list[int]:
    """Box sizes drawn log-uniformly from [lo, hi] (one draw per replica seed)."""
    out = []
    for b in range(n_rep):
        u = _rng(seed * 1000003 + b, 2).uniform()
        out.append(int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))))
    return out


# Workload presets (alpha in length^-2: sqrt(alpha) = 0.3 / Angstrom; r_c = 10 Angstrom).
PRESETS = {
    "n3000_all_charged": dict(N=3000, L=32.0, all_charged=True, P=100, seed=1),
    "n1m_10pct": dict(N=1 << 20, density=0.1, frac_charged=0.1, P=200, seed=2),
    "n16m_10pct": dict(N=1 << 24, density=0.1, frac_charged=0.1, P=500, seed=3),
    "n134m_5pct_rbl": dict(N=1 << 27, density=0.1, frac_charged=0.05, P=500, seed=5,
                           r_core=5.0, p_rbl=10),
}
ALPHA = 0.09
R_CUT = 10.0
