"""Batched replicas (independent boxes of uneven size advanced by one graph launch per
step) must give exactly the state that stepping each replica alone gives."""
import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.lib()


def _replicas(sizes):
    out = []
    for r, n in enumerate(sizes):
        sy = synth.make_system(n, density=0.1, frac_charged=0.1, seed=100 + r)
        out.append((r, sy))
    return out


def _handle(r, sy, precision="fp32_comp"):
    return binding.from_system(sy, P=64, alpha=synth.ALPHA, r_c=synth.R_CUT,
                               coulomb_C=synth.COULOMB_C, dt=1.0, kappa=synth.ACCEL_KAPPA,
                               replica=r, precision=precision)


@pytest.mark.parametrize("precision,order", [("fp32_comp", 1), ("fp64", 1), ("fp64", -1)])
def test_batch_equals_individual_steps(precision, order):
    """Uneven sizes, in either order: boxes whose pair kernels differ (half-precision
    pre-test or not, cluster pairs or per-particle) fall into different classes."""
    import torch
    reps = _replicas([2000, 5100, 3000, 9000, 2400][::order])
    hb = [_handle(r, sy, precision) for r, sy in reps]
    hi = [_handle(r, sy, precision) for r, sy in reps]
    with binding.Batch(hb) as b:
        b.step(3)
        b.step(2)
        torch.cuda.synchronize()
        for h in hi:
            h.step(5)
        for a, c in zip(hb, hi):
            pa, va, sa = a.state()
            pc, vc, sc = c.state()
            assert np.array_equal(sa, sc) and np.array_equal(va, vc)
            ea, _ = a.energies()
            ec, _ = c.energies()
            assert ea["total"] == ec["total"]
            assert a.step_count() == c.step_count() == 5
    for h in hb + hi:
        h.close()


@pytest.mark.parametrize("precision,nvt", [("fp32_comp", False), ("fp32", True),
                                           ("fp64", False)])
def test_batch_classes_equal_individual_steps(precision, nvt):
    """Replicas of one configuration (uneven sizes) form one class: every kernel of the step
    runs once over all of them, and the result is bit for bit what each replica's own steps
    give (with the Nose-Hoover thermostat in one case)."""
    import torch
    reps = _replicas([20000, 31000, 26000, 40000])
    hb = [_handle(r, sy, precision) for r, sy in reps]
    hi = [_handle(r, sy, precision) for r, sy in reps]
    if nvt:
        for h in hb + hi:
            h.set_thermostat(300.0, 50.0)
    with binding.Batch(hb) as b:
        ncls, nbat, kern = b.info()
        # the FP32 forms share every kernel; the FP64 form's per-particle pair kernel has a
        # half-precision pre-test variant that depends on the box
        assert nbat == 4 and ncls == 1 if precision != "fp64" else nbat == 4 and ncls <= 2, \
            (ncls, nbat, kern)
        # one launch per kernel of the step and class, the pair kernels one per replica
        assert 0 < kern < 30 * ncls + 3 * nbat
        b.step(3)
        torch.cuda.synchronize()
        for h in hi:
            h.step(3)
        for a, c in zip(hb, hi):
            _, va, sa = a.state()
            _, vc, sc = c.state()
            assert np.array_equal(sa, sc) and np.array_equal(va, vc)
            ea, wa = a.energies()
            ec, wc = c.energies()
            assert ea == ec and wa == wc
            if nvt:
                assert a.thermostat() == c.thermostat()
    for h in hb + hi:
        h.close()


def test_replica_key_gives_independent_modes():
    reps = _replicas([2000, 2000])
    h0 = _handle(0, reps[0][1])
    h1 = _handle(1, reps[0][1])
    m0, _ = h0.sample_k(0)
    m1, _ = h1.sample_k(0)
    assert not np.array_equal(m0, m1)
    import oracle
    mo, _ = oracle.sample_k(1, 0, 1, reps[0][1].box, synth.ALPHA, 64)
    assert np.array_equal(m1, mo)


def test_batch_mixed_traversals_equal_individual_steps():
    """A batch mixing a random-batch-list replica, a Verlet-list replica and a cell-list
    replica replays exactly what each replica's own steps give (list rebuilds, RBL draws
    and the RBL scratch pool included)."""
    import torch
    reps = _replicas([6000, 7000, 2500])

    def make(r, sy):
        if r == 0:
            return binding.from_system(sy, P=64, alpha=synth.ALPHA, r_c=synth.R_CUT,
                                       coulomb_C=synth.COULOMB_C, dt=1.0,
                                       kappa=synth.ACCEL_KAPPA, replica=r, r_core=5.0,
                                       p_rbl=10)
        h = _handle(r, sy)
        if r == 1:
            h.set_neighbor_list(0.5)
        return h

    hb = [make(r, sy) for r, sy in reps]
    hi = [make(r, sy) for r, sy in reps]
    with binding.Batch(hb) as b:
        assert b.info()[:2] == (0, 0)  # list and RBL replicas, and a lone cell replica
        b.step(4)
        torch.cuda.synchronize()
        for h in hi:
            h.step(4)
        for a, c in zip(hb, hi):
            _, va, sa = a.state()
            _, vc, sc = c.state()
            assert np.array_equal(sa, sc) and np.array_equal(va, vc)
            assert a.energies()[0]["total"] == c.energies()[0]["total"]
    assert hb[1].neighbor_list_stats()["builds"] == hi[1].neighbor_list_stats()["builds"] >= 1
    for h in hb + hi:
        h.close()


def test_full_size_batch96(orc):
    """The benchmark's 96 replicas (log-uniform 2,000..250,000 particles, 10% charged, seeds
    1000 + r, replica keys r, P = 200). Step-0 forces and neighbour counts of sampled
    particles of every replica match the oracle; then two batched steps (one graph launch
    each) leave every replica exactly where its own two steps leave it."""
    import torch
    import sampled
    sizes = synth.replica_sizes(96)
    systems = [synth.make_system(n, density=0.1, frac_charged=0.1, seed=1000 + r)
               for r, n in enumerate(sizes)]

    def make(r, sy):
        return binding.from_system(sy, P=200, alpha=synth.ALPHA, r_c=synth.R_CUT,
                                   coulomb_C=synth.COULOMB_C, dt=1.0, kappa=synth.ACCEL_KAPPA,
                                   replica=r)

    Fg, Fo = [], []
    for r, sy in enumerate(systems):
        with make(r, sy) as h:
            F, _, _ = h.forces_f64(0)
            nbr, _ = h.neighbor_counts()
            m, S = sampled.oracle_modes(orc, h, sy, 200, 0, replica=r)
        rng = np.random.default_rng(r)
        idx = np.unique(np.r_[rng.choice(sy.n, 4, replace=False), np.flatnonzero(sy.q)[:1]])
        Fo_r, nbr_o = sampled.total_forces_sampled(orc, sy, idx, m, S)
        assert np.array_equal(nbr[idx], nbr_o)
        Fg.append(F[idx])
        Fo.append(Fo_r)
    Fg, Fo = np.concatenate(Fg), np.concatenate(Fo)
    assert np.linalg.norm(Fg - Fo) / np.linalg.norm(Fo) < 1e-5
    hb = [make(r, sy) for r, sy in enumerate(systems)]
    hi = [make(r, sy) for r, sy in enumerate(systems)]
    with binding.Batch(hb) as b:
        ncls, nbat, _ = b.info()
        assert nbat >= 80 and ncls <= 6
        b.step(2)
        torch.cuda.synchronize()
        for h in hi:
            h.step(2)
        for a, c in zip(hb, hi):
            _, va, sa = a.state()
            _, vc, sc = c.state()
            assert np.array_equal(sa, sc) and np.array_equal(va, vc)
    for h in hb + hi:
        h.close()
