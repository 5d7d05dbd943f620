"""Failure detection without a GPU fault: device waits that nothing
satisfies give up after their limit, report CLOAK_E_TIMEOUT through the
status word, and the context keeps working afterwards."""
import time

import pytest
import torch

from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device

pytestmark = pytest.mark.gpu


def test_bounded_waits_time_out_and_the_context_stays_usable(cloak_lib):
    m = synth.small_decoder(1, synth.DT_BF16)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x99, twin=False)
    x = x_device(m, synth.activations_host(4, m.tensors[0].k, seed=1))
    y0 = cm.linear(0, x, out_dtype=cloak_lib.OUT_F32).cpu()
    t0 = time.perf_counter()
    cm.check_waits()                       # both waits gave up and said so
    assert 1.5 < time.perf_counter() - t0 < 30.0
    assert cm.device_status() == 0         # the self-test cleared what it read
    y1 = cm.linear(0, x, out_dtype=cloak_lib.OUT_F32).cpu()
    assert torch.equal(y0, y1)
    cm.close()
