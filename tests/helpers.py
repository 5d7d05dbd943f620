"""Shared test helpers: run a model through the CUDA library and the oracle
on the same seeded inputs."""
import numpy as np

import oracle as O
from paper_2606_18400_gb300 import synth


def torch_bf16_bits(t):
    import torch
    return t.contiguous().view(torch.int16).cpu().numpy().view(np.uint16)


def place_both(cloak, model, key, epoch=0, seed=0, twin=True, weights=None, vmm=False):
    """Keygen + shuffle on the GPU and in the oracle with the same inputs.
    Returns (gpu model, oracle model, oracle tables, oracle arena, scales, Ws)."""
    import torch
    cm = cloak.CloakModel(model, twin=twin, vmm=vmm)
    cm.keygen(key, epoch)
    Ws = weights if weights is not None else synth.weights_host(model, seed=seed)
    for t, W in enumerate(Ws):
        cm.shuffle(t, torch.from_numpy(np.ascontiguousarray(W)).cuda())
    torch.cuda.synchronize()
    om = O.OracleModel(model)
    tb = O.keygen(om, key, epoch)
    arena, scales = O.shuffle_model(om, tb, Ws)
    return cm, om, tb, arena, scales, Ws


def x_device(model, x_f32):
    """Activations as the CUDA path takes them: FP32 for FP32 weights, else
    BF16 (rounded by torch)."""
    import torch
    x = torch.from_numpy(np.ascontiguousarray(x_f32)).cuda()
    return x if model.dtype == synth.DT_F32 else x.to(torch.bfloat16)
