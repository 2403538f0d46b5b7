"""Host-side logic of bench.py (no GPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_launch_count_claim_matches_the_profiled_launch_list():
    # the ncu launch list of the 256^3 p = 6 bench counts per solve of the
    # headline form: mean 2, P2M 1, M2M 3, M2L 8 (level 2 double-float +
    # range sum, level 3 split table + range sum, levels 4-5 BF16 split +
    # tensor core), L2L 3, near zone by FFT 4 (forward, sums, L2P, inverse):
    # 21; the direct near zone is 1 kernel, and the plain form replaces each
    # tensor-core pair by one FP32 kernel
    import bench
    assert bench.launches_per_solve(5, True, 6, near_fft=True) == 21
    assert bench.launches_per_solve(5, True, 6) == 18
    assert bench.launches_per_solve(5, False, 6) == 16
