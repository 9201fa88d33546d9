"""GPU test of rbe_structure_factor_noalloc, the structure-factor entry point that
allocates no device memory. It serves callers that must not allocate: a host application
that owns one fixed device pool, or a latency-bound loop that cannot afford the
synchronisation of cudaMalloc.

The entry point is called twice in a row through the C ABI (all modes, then a shorter
mode list that reuses the shared scratch with another layout). Each result is compared
with the structure factor of the existing path (rbe_forces + rbe_get_rho) and with the
oracle's, at the tolerance of the other structure-factor tests; two more cases (four
mode blocks, and the largest mode count the scratch holds) are checked against the
oracle alone. This file is collected last so that a run
that stops at its first failure has already run every other test."""
import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu

TOL = 2e-6  # the FP32-compensated structure-factor tolerance of test_gpu_parity


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_structure_factor_matches_handle_path():
    import torch
    build.build()
    L = binding.lib()
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=12)
    P = 200
    with binding.from_system(sy, P=P, alpha=synth.ALPHA, r_c=synth.R_CUT,
                             coulomb_C=synth.COULOMB_C) as h:
        h.forces(0)
        rho_ref, m = h.rho()
    import oracle
    mo, _ = oracle.sample_k(1, 0, 0, sy.box, synth.ALPHA, P)
    assert np.array_equal(m, mo)
    rho_orc = oracle.rho(sy.s, sy.q, sy.box, mo)
    # caller-owned device inputs and output, in the layout the entry point documents
    s_dev = torch.from_numpy(np.ascontiguousarray(sy.s.T).view(np.int32)).cuda()
    q_dev = torch.from_numpy(sy.q.astype(np.float32)).cuda()
    m_dev = torch.from_numpy(np.ascontiguousarray(m, np.int32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for Pc in (P, 150):
        rho_dev = torch.full((Pc, 2), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.rbe_structure_factor_noalloc(s_dev.data_ptr(), q_dev.data_ptr(), sy.n,
                                            m_dev.data_ptr(), Pc, rho_dev.data_ptr(), stream)
        assert rc == 0, binding.lib().rbe_error_string(rc)
        torch.cuda.synchronize()
        got = rho_dev.cpu().numpy()
        assert rel_l2(got[:, 0] + 1j * got[:, 1], rho_ref[:Pc]) < TOL
        assert rel_l2(got[:, 0] + 1j * got[:, 1], rho_orc[:Pc]) < TOL


@pytest.mark.parametrize("N,P", [(20000, 1000), (2500, 65536)])
def test_noalloc_structure_factor_matches_oracle(orc, N, P):
    """Against the oracle's structure factor on the oracle's own mode draw, twice in a row:
    P = 1000 spans four mode blocks, whose last one masks the modes past P; P = 65536 (the
    largest the scratch holds) cuts the particle blocks to the eight whose partial sums fit
    in the array."""
    import torch
    build.build()
    L = binding.lib()
    sy = synth.make_system(N, density=0.1, frac_charged=0.1, seed=13)
    m, _ = orc.sample_k(3, 1, 0, sy.box, synth.ALPHA, P)
    ref = orc.rho(sy.s, sy.q, sy.box, m)
    s_dev = torch.from_numpy(np.ascontiguousarray(sy.s.T).view(np.int32)).cuda()
    q_dev = torch.from_numpy(sy.q.astype(np.float32)).cuda()
    m_dev = torch.from_numpy(np.ascontiguousarray(m, np.int32)).cuda()
    for _ in range(2):
        rho_dev = torch.full((P, 2), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.rbe_structure_factor_noalloc(s_dev.data_ptr(), q_dev.data_ptr(), sy.n,
                                            m_dev.data_ptr(), P, rho_dev.data_ptr(), None)
        assert rc == 0, binding.lib().rbe_error_string(rc)
        torch.cuda.synchronize()
        got = rho_dev.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got[:, 0] + 1j * got[:, 1], ref) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    build.build()
    L = binding.lib()
    s_dev = torch.zeros((3, 8), dtype=torch.int32, device="cuda")
    q_dev = torch.zeros(8, dtype=torch.float32, device="cuda")
    m_dev = torch.ones((65537, 3), dtype=torch.int32, device="cuda")
    rho_dev = torch.zeros((65537, 2), dtype=torch.float64, device="cuda")
    # P above the fixed maximum is refused before anything is launched
    assert L.rbe_structure_factor_noalloc(s_dev.data_ptr(), q_dev.data_ptr(), 8,
                                          m_dev.data_ptr(), 65537, rho_dev.data_ptr(),
                                          None) == -1
    # missing inputs are refused as well
    assert L.rbe_structure_factor_noalloc(None, None, 8, m_dev.data_ptr(), 4,
                                          rho_dev.data_ptr(), None) == -1
    torch.cuda.synchronize()
    assert torch.all(rho_dev == 0).item()
