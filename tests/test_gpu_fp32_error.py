"""The FP32 form's error against the plain FP64 oracle on the benchmark's
4096-instance workload (full size, autotuned, graph-replayed), on six sampled
instances over 200 steps (tests/fp32_error.py describes the measure).  The
two forms draw identical random numbers, so the error is the FP32
arithmetic's; it stays at rounding size for the fields the conservation step
fixes (U, temperatures) and for stress and heat fluxes, and grows in q_vib
only where a rounding difference turns a level decision the other way.  The
bars are about ten times the measured values (DESIGN, section 5)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import fp32_error as E  # noqa: E402

pytestmark = pytest.mark.gpu

# (time-averaged L2, max) per field over the first 20 and 200 steps
BARS = {
    20: {"U": (2e-7, 5e-7), "T_tr": (1e-6, 2e-6), "T_rot": (1e-6, 2e-6), "T_vib": (1e-12, 1e-12),
         "sigma": (2e-7, 1e-6), "q_tr": (2e-6, 5e-6), "q_rot": (2e-7, 1e-6), "q_vib": (1e-7, 1e-6)},
    200: {"U": (2e-7, 5e-7), "T_tr": (1e-6, 2e-6), "T_rot": (1e-6, 2e-6), "T_vib": (1e-12, 1e-12),
          "sigma": (2e-7, 1e-6), "q_tr": (2e-6, 5e-6), "q_rot": (2e-7, 1e-6), "q_vib": (5e-4, 5e-3)},
}


def test_fp32_form_error_against_fp64_oracle_is_bounded():
    table, flags, sample, sizes = E.measure(200, windows=(20, 200))
    assert flags == 0
    for K, bars in BARS.items():
        for g, (l2_bar, max_bar) in bars.items():
            l2, mx = table[K][g]
            assert l2 < l2_bar and mx < max_bar, (K, g, l2, mx)
