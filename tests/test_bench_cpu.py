"""CPU checks of bench.py's host-side pieces that need no GPU: the oracle baseline record
(all threads and one thread) has the fields the benchmark line reports, and the oracle's
thread count is restored afterwards."""
import oracle

import bench
from paper_2609_02694_gb300 import synth


def test_cpu_baseline_record_fields():
    oracle.lib()
    before = oracle.num_threads()
    sy = synth.make_system(20000, density=0.1, frac_charged=0.1, seed=2)
    rec = bench.cpu_baseline_record(oracle, sy, 50, n_sample=32, n_sample_1=16)
    assert oracle.num_threads() == before
    assert rec["kind"] == "oracle" and rec["unit"] == bench.UNIT and rec["cores"] == before
    assert rec["value"] > 0 and "32 random particles" in rec["sample"]
    one = rec["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and "16 random particles" in one["sample"]
