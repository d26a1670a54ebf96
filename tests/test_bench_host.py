"""Host-side pieces of bench.py that need no GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2601_21407_gb300 import inputs as inp  # noqa: E402


def test_sfu_work_per_neuron_step():
    """Classic HH: 6 rate exponentials + 3 gate and 1 membrane relaxation
    factors = 10; 2 linoid + 1 sigmoid rate divisions + 3 p_inf + 1 V_inf = 7.
    Multi-channel: the bell-shaped time constants of KA (offsets 0.37 and 19
    ms) take one division each and that of Ih (no offset) none; KCa's
    constant time constant none."""
    assert bench.mufu_ops_per_neuron_step(inp.CLASSIC_HH) == (10, 7)
    assert bench.mufu_ops_per_neuron_step(inp.MULTI_CHANNEL) == (26, 16)
