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


def test_concurrent_rekey_interrupted_by_the_host(cloak_lib):
    """The host stops advancing a concurrent re-key after two waves and shuts
    the context down mid-job: every step until then computes what it did
    before the re-key, the destroy returns (it synchronises the device, no
    wait is left hanging), and a new context on the device works."""
    m = synth.llama7b_layer(1)  # 193 pages through 8 staging pages: many waves
    key = 0x51
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=key, twin=False)
    x = x_device(m, synth.activations_host(2, m.tensors[4].k, seed=3))
    y0 = cm.linear(4, x, out_dtype=cloak_lib.OUT_F32).cpu()
    serve, side = torch.cuda.Stream(), torch.cuda.Stream()
    cm.rekey_begin(key, 1, side)
    done = False
    for _ in range(2):
        side.synchronize()
        with torch.cuda.stream(serve):
            y = cm.linear(4, x, out_dtype=cloak_lib.OUT_F32)
        done = cm.rekey_advance(serve, side)
        serve.synchronize()
        assert torch.equal(y.cpu(), y0)
    assert not done                         # interrupted mid-job
    t0 = time.perf_counter()
    cm.close()
    assert time.perf_counter() - t0 < 10.0
    cm2, om2, tb2, arena2, scales2, Ws2 = place_both(cloak_lib, synth.small_decoder(1, synth.DT_BF16), key=7,
                                                     twin=False)
    x2 = x_device(cm2.model, synth.activations_host(1, cm2.model.tensors[0].k, seed=1))
    y2 = cm2.linear(0, x2, out_dtype=cloak_lib.OUT_F32).cpu().numpy()
    import oracle as O
    ref = O.cloaked_linear(om2, tb2, 0, arena2, synth.activations_host(1, cm2.model.tensors[0].k, seed=1))
    assert O.relative_error(y2, ref) <= 1e-2
    assert cm2.device_status() == 0
    cm2.close()
