"""GPU cloaked linear against the FP64 oracle (normwise relative error:
1e-5 FP32, 1e-2 BF16, 5e-2 E4M3) and bit-exact against the uncloaked
kernel with the same reduction order."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device, torch_bf16_bits

pytestmark = pytest.mark.gpu

TOL = {synth.DT_F32: 1e-5, synth.DT_BF16: 1e-2, synth.DT_E4M3: 5e-2}


def run_linear(cloak, cm, t, x, out_f32=True, uncloaked=False, relu=False):
    y = cm.linear(t, x, out_dtype=cloak.OUT_F32 if out_f32 else cloak.OUT_BF16,
                  uncloaked=uncloaked, relu=relu)
    torch.cuda.synchronize()
    return y


def check_tensor(cloak, cm, om, tb, arena, scales, t, M, seed):
    m = om.model
    tt = m.tensors[t]
    x = synth.activations_host(M, tt.k, seed=seed)
    xd = x_device(m, x)
    if m.dtype != synth.DT_F32:
        assert np.array_equal(torch_bf16_bits(xd), O.bf16_bits(x))  # same operand both sides
    ref = O.cloaked_linear(om, tb, t, arena, x, scales[t] if scales else None)
    y = run_linear(cloak, cm, t, xd).cpu().numpy()
    err = O.relative_error(y, ref)
    assert err <= TOL[m.dtype], (t, M, err)
    if cm.model is not None and getattr(cm, "_twin", True):
        yu = run_linear(cloak, cm, t, xd, uncloaked=True).cpu().numpy()
        assert np.array_equal(y.view(np.uint32), yu.view(np.uint32)), (t, M)
    yb = run_linear(cloak, cm, t, xd, out_f32=False)
    yb = yb.view(torch.int16).cpu().numpy().view(np.uint16)
    assert np.array_equal(yb, O.bf16_bits(y)), "BF16 output is the rounded FP32 result"
    return err


@pytest.mark.parametrize("M", [1, 3, 8, 17, 32, 64, 100, 256, 300])
def test_small_bf16_decoder_all_tensors(cloak_lib, M):
    m = synth.small_decoder(2, synth.DT_BF16, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200,
                            spare_pages=5)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234)
    for t in range(len(m.tensors)):
        check_tensor(cloak_lib, cm, om, tb, arena, scales, t, M, seed=M * 31 + t)
    cm.close()


@pytest.mark.parametrize("M", [1, 4, 16, 64, 200, 300])
def test_small_fp8_decoder_all_tensors(cloak_lib, M):
    m = synth.small_decoder(2, synth.DT_E4M3, page_bytes=2 * 128 * 128, d_model=384, n_heads=6,
                            n_kv_heads=2, d_ff=256)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=5)
    for t in range(len(m.tensors)):
        check_tensor(cloak_lib, cm, om, tb, arena, scales, t, M, seed=M * 7 + t)
    cm.close()


@pytest.mark.parametrize("M", [1, 3, 16, 260])
def test_fp8_quantised_operands_are_near_exact(cloak_lib, M):
    """With the oracle's quantised activations the only difference left is
    FP32 accumulation order: far below the 5e-2 bound (M <= 4 quantises inside
    the linear, M = 16 in the separate quantiser)."""
    m = synth.small_decoder(1, synth.DT_E4M3, page_bytes=2 * 128 * 128, d_model=512, d_ff=512,
                            n_heads=4, n_kv_heads=4, head_dim=128)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=9)
    for t in range(len(m.tensors)):
        err = check_tensor(cloak_lib, cm, om, tb, arena, scales, t, M, seed=t)
        assert err < 1e-5
    cm.close()


@pytest.mark.parametrize("grouped", [False, True])
def test_fp8_fused_quantisation_equals_separate(cloak_lib, grouped):
    """Decode batches (M <= 4) quantise their activations inside the linear;
    wider batches run the separate quantiser. A row's result depends only on
    its own token's codes and scale, and M = 4 and M = 5 share the tile shape
    and the split over CTAs, so the first four rows must agree bit for bit."""
    m = synth.small_decoder(2, synth.DT_E4M3, page_bytes=2 * 128 * 128, d_model=384, n_heads=6,
                            n_kv_heads=2, d_ff=256)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x3C)
    ts = [i for i, t in enumerate(m.tensors) if t.layer == 1]
    xs = [x_device(m, synth.activations_host(5, m.tensors[t].k, seed=90 + t)) for t in ts]
    if grouped:
        y5 = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32)
        y4 = cm.linear_batch(ts, [x[:4].contiguous() for x in xs], out_dtype=cloak_lib.OUT_F32)
    else:
        y5 = [cm.linear(t, x, out_dtype=cloak_lib.OUT_F32) for t, x in zip(ts, xs)]
        y4 = [cm.linear(t, x[:4].contiguous(), out_dtype=cloak_lib.OUT_F32) for t, x in zip(ts, xs)]
    torch.cuda.synchronize()
    for a, b in zip(y4, y5):
        assert torch.equal(a, b[:4])
    assert cm.device_status() == 0
    cm.close()


def test_mlp2_fp32_matches_fp64_oracle(cloak_lib):
    """Two-layer FP32 MLP (d 256, d_ff 1024, batch 4, key 0x1234): the
    cloaked W1 (rows permuted) and W2 (columns compensated) compute the plain
    MLP within 1e-5 normwise; the shuffle round trip is bit-exact."""
    m = synth.mlp2()
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234)
    x = synth.activations_host(4, 256, seed=1)
    xd = x_device(m, x)
    h = cm.linear(0, xd, out_dtype=cloak_lib.OUT_F32, relu=True)
    y = cm.linear(1, h, out_dtype=cloak_lib.OUT_F32)
    torch.cuda.synchronize()
    ref = O.mlp2_f64(x.astype(np.float64), Ws[0], Ws[1])
    assert O.relative_error(y.cpu().numpy(), ref) <= 1e-5
    for t in range(2):
        assert np.array_equal(cm.unshuffle(t).cpu().numpy(), Ws[t])
    # the hidden activations are permuted exactly as the oracle permutes W1's rows
    rmap, _ = O.axis_maps(om, tb, 0)
    hp = np.maximum(x.astype(np.float64) @ Ws[0].astype(np.float64).T, 0)[:, rmap]
    assert O.relative_error(h.cpu().numpy(), hp) <= 1e-5
    cm.close()


@pytest.mark.parametrize("M", [1, 8, 32, 64])
def test_llama7b_layer_decode(cloak_lib, M):
    """One 7B-class BF16 layer (Wq, Wk, Wv, Wo, Wgate, Wup, Wdown) at decode
    batch M: each cloaked linear within 1e-2 of the FP64 oracle and
    bit-identical to the uncloaked kernel."""
    m = synth.llama7b_layer(1)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234)
    for t in range(len(m.tensors)):
        check_tensor(cloak_lib, cm, om, tb, arena, scales, t, M, seed=100 + t)
    cm.close()


def test_integer_mlp_cloaked_equals_plain_exactly(cloak_lib):
    """Integer-valued weights and inputs keep every FP32 sum exact, so the
    cloaked, permuted and compensated MLP equals the plain one bit for bit,
    for several keys."""
    m = synth.mlp2()
    Ws = synth.int_weights_host(m, seed=3, lo=-1, hi=1)
    x = np.random.default_rng(4).integers(-2, 3, size=(4, 256)).astype(np.float32)
    ref = O.mlp2_f64(x.astype(np.float64), Ws[0], Ws[1])
    for key in (1, 2, 0x1234):
        cm, om, tb, arena, scales, _ = place_both(cloak_lib, m, key=key, weights=Ws)
        h = cm.linear(0, torch.from_numpy(x).cuda(), out_dtype=cloak_lib.OUT_F32, relu=True)
        y = cm.linear(1, h, out_dtype=cloak_lib.OUT_F32)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy().astype(np.float64), ref)
        cm.close()


def test_linear_host_entry_point(cloak_lib):
    m = synth.small_decoder(1, synth.DT_BF16)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=3)
    x = synth.activations_host(5, m.tensors[0].k, seed=2)
    xb = torch.from_numpy(x).to(torch.bfloat16).pin_memory()
    yh = torch.empty((5, m.tensors[0].n), dtype=torch.float32).pin_memory()
    cloak_lib.cloak_linear_host(cm.ctx, 0, xb.data_ptr(), yh.data_ptr(), 5, cloak_lib.OUT_F32)
    yd = cm.linear(0, xb.cuda(), out_dtype=cloak_lib.OUT_F32).cpu()
    assert torch.equal(yh, yd)
    cm.close()


@pytest.mark.parametrize("layout", ["packed", "separate", "pageable", "unaligned"])
def test_batch_host_entry_point(cloak_lib, layout):
    """The grouped launch from host buffers equals the same launch on device
    buffers bit for bit, whether the host vectors lie back to back (one copy
    each way), apart, in pageable memory, or in pinned memory at 2-byte
    offsets."""
    m = synth.small_decoder(1, synth.DT_BF16, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x5A)
    M = 3
    ts = list(range(len(m.tensors)))
    xs = [torch.from_numpy(synth.activations_host(M, m.tensors[t].k, seed=70 + t)).to(torch.bfloat16)
          for t in ts]
    pin = layout != "pageable"
    if layout in ("packed", "unaligned"):
        sh = 1 if layout == "unaligned" else 0
        xbuf = torch.cat([torch.zeros(sh, dtype=torch.bfloat16)] + [x.reshape(-1) for x in xs]).pin_memory()
        ybuf = torch.empty(sum(M * m.tensors[t].n for t in ts) + sh, dtype=torch.float32).pin_memory()
        xh, yh, o, q = [], [], sh, sh
        for t, x in zip(ts, xs):
            xh.append(xbuf[o:o + x.numel()].view(M, -1))
            o += x.numel()
            yh.append(ybuf[q:q + M * m.tensors[t].n].view(M, -1))
            q += M * m.tensors[t].n
    else:
        xh = [x.pin_memory() if pin else x.clone() for x in xs]
        yh = [torch.empty((M, m.tensors[t].n), dtype=torch.float32) for t in ts]
        if pin:
            yh = [y.pin_memory() for y in yh]
    cloak_lib.cloak_linear_batch_host(cm.ctx, ts, [x.data_ptr() for x in xh], [y.data_ptr() for y in yh],
                                      M, cloak_lib.OUT_F32)
    yd = cm.linear_batch(ts, [x.cuda() for x in xs], out_dtype=cloak_lib.OUT_F32)
    torch.cuda.synchronize()
    for y, d in zip(yh, yd):
        assert torch.equal(y, d.cpu())
    assert cm.device_status() == 0
    cm.close()


def test_bad_calls_return_errors(cloak_lib):
    m = synth.small_decoder(1, synth.DT_BF16)
    cm = cloak_lib.CloakModel(m)
    x = torch.zeros((2, m.tensors[0].k), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(cloak_lib.CloakError) as e:
        cm.linear(0, x)  # before keygen
    assert e.value.status == cloak_lib.E_STATE
    cm.keygen(1, 0)
    with pytest.raises(cloak_lib.CloakError):
        cm.linear(0, x, uncloaked=True)  # no twin
    with pytest.raises(cloak_lib.CloakError):
        cloak_lib.cloak_linear(cm.ctx, 99, x.data_ptr(), x.data_ptr(), 2, 0)
    assert cm.device_status() == 0
    cm.close()


@pytest.mark.parametrize("M", [1, 8, 64, 300])
def test_batched_layer_launch(cloak_lib, M):
    """All seven linears of a decoder layer in one launch (one split over
    their concatenated tiles): each output within tolerance of the oracle,
    cloaked and uncloaked batches bit-identical."""
    m = synth.small_decoder(2, synth.DT_BF16, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200,
                            spare_pages=5)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x77)
    for layer in range(2):
        ts = [i for i, t in enumerate(m.tensors) if t.layer == layer]
        xs_h = [synth.activations_host(M, m.tensors[t].k, seed=50 + t) for t in ts]
        xs = [x_device(m, x) for x in xs_h]
        ys = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32)
        yu = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
        torch.cuda.synchronize()
        for t, x, y, u in zip(ts, xs_h, ys, yu):
            ref = O.cloaked_linear(om, tb, t, arena, x)
            assert O.relative_error(y.cpu().numpy(), ref) <= 1e-2
            assert torch.equal(y, u)
    cm.close()


def test_batched_fp8_launch(cloak_lib):
    m = synth.small_decoder(1, synth.DT_E4M3, page_bytes=2 * 128 * 128, d_model=384, n_heads=6,
                            n_kv_heads=2, d_ff=256)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x78)
    ts = list(range(len(m.tensors)))
    xs_h = [synth.activations_host(5, m.tensors[t].k, seed=t) for t in ts]
    ys = cm.linear_batch(ts, [x_device(m, x) for x in xs_h], out_dtype=cloak_lib.OUT_F32)
    torch.cuda.synchronize()
    for t, x, y in zip(ts, xs_h, ys):
        ref = O.cloaked_linear(om, tb, t, arena, x, scales[t])
        assert O.relative_error(y.cpu().numpy(), ref) <= 1e-5
    cm.close()


def test_batched_full_layer(cloak_lib):
    m = synth.llama7b_layer(1)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234)
    ts = list(range(7))
    xs_h = [synth.activations_host(8, m.tensors[t].k, seed=200 + t) for t in ts]
    xs = [x_device(m, x) for x in xs_h]
    ys = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32)
    yu = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
    torch.cuda.synchronize()
    for t, x, y, u in zip(ts, xs_h, ys, yu):
        assert O.relative_error(y.cpu().numpy(), O.cloaked_linear(om, tb, t, arena, x)) <= 1e-2
        assert torch.equal(y, u)
    cm.close()


@pytest.mark.parametrize("M", [512])
def test_full_layer_prefill_sampled(cloak_lib, M):
    """Prefill of the full 7B-class layer in one grouped launch (whole 256x256
    output tiles per CTA): a keyed sample of 48 output features of every
    tensor, all tokens, against the FP64 product on the stored weights; the
    cloaked and uncloaked launches agree bit for bit on the whole output."""
    m = synth.llama7b_layer(1)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234)
    ts = list(range(7))
    xs_h = [synth.activations_host(M, m.tensors[t].k, seed=300 + t) for t in ts]
    xs = [x_device(m, x) for x in xs_h]
    ys = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32)
    yu = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0x5EED)
    for t, x, y, u in zip(ts, xs_h, ys, yu):
        assert torch.equal(y, u)
        rows = np.sort(rng.choice(m.tensors[t].n, 48, replace=False))
        W64 = O.stored_f64(om, tb, t, arena)[rows]
        ref = O.linear_f64(O.x_operand(om, x), W64)
        err = O.relative_error(y.cpu().numpy()[:, rows], ref)
        assert err <= 1e-2, (t, err)
    cm.close()


@pytest.mark.parametrize("M", [1, 2048])
def test_full_fp8_gqa_layer_sampled(cloak_lib, M):
    """The E4M3 GQA layer (d 3584, 28/4 heads, MLP 18944; 233 MB) in the
    launch the benchmark times (one grouped launch, tuned shape): decode
    M = 1 (activations quantised inside the launch) and prefill M = 2048 (the
    prefill GEMM). A keyed sample of 48 stored rows per tensor against the
    FP64 product of the dequantised operands (rows quantised per R12 from the
    logical weights, drawn again on the device from their seeds); cloaked and
    uncloaked agree bit for bit."""
    m = synth.gqa28_fp8(1)
    cm = cloak_lib.CloakModel(m, twin=True)
    key = 0x1234
    cm.keygen(key, 0)
    for t in range(len(m.tensors)):
        cm.shuffle(t, synth.weights_device(m, t, seed=7))
    om = O.OracleModel(m)
    tb = O.keygen(om, key, 0)
    ts = list(range(len(m.tensors)))
    xs_h = [synth.activations_host(M, m.tensors[t].k, seed=700 + t) for t in ts]
    xs = [x_device(m, x) for x in xs_h]
    cm.autotune(ts, xs)
    ys = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32)
    yu = cm.linear_batch(ts, xs, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0xF8)
    for t, x, y, u in zip(ts, xs_h, ys, yu):
        assert torch.equal(y, u), t
        tt = m.tensors[t]
        rows = np.sort(rng.choice(tt.n, 48, replace=False))
        rmap, cmap = O.axis_maps(om, tb, t)
        W = synth.weights_device(m, t, seed=7).cpu().numpy()
        Ws = W[rmap[rows]][:, cmap]                     # the stored rows, logical values
        q, s = O.quant_rows_e4m3(Ws)                    # per stored row: amax/448, E4M3
        Wdq = O.e4m3_value(q) * s.astype(np.float64)[:, None]
        ref = O.linear_f64(O.x_operand(om, x), Wdq)
        err = O.relative_error(y.cpu().numpy()[:, rows], ref)
        assert err <= 5e-2, (t, err)
        # the second figure: against the unquantised operands (the FP32 master
        # weights and the BF16 activations the call receives). E4M3 keeps 3
        # mantissa bits: about 3.6 % RMS relative rounding per operand, so
        # about 5 % for the product of two quantised operands
        ref_u = O.linear_f64(O.bf16_value(O.bf16_bits(x)), Ws.astype(np.float64))
        err_u = O.relative_error(y.cpu().numpy()[:, rows], ref_u)
        print(f"E4M3 layer M={M} tensor {t}: {err:.2e} vs dequantised operands, "
              f"{err_u:.2e} vs unquantised operands")
        assert err < err_u <= 0.1, (t, err, err_u)
        sc = cm.scales(t).cpu().numpy()[rows]
        assert np.array_equal(sc.view(np.uint32), s.view(np.uint32)), t  # the same row scales
    assert cm.device_status() == 0
    cm.close()


@pytest.mark.parametrize("fp8,M", [(False, 1), (False, 16), (True, 1), (True, 16)])
def test_chained_launches_equal_plain_ones(cloak_lib, fp8, M):
    """A chain of 24 dependent linears (Wq, then Wo on its output, then Wq
    on that, ...; BF16 outputs feeding the next call) launched as chained
    launches -- each one's CTAs stream weights while the previous one runs and
    read x after it completes -- gives the plain chain's result bit for bit,
    eagerly and replayed from a CUDA graph. E4M3 at M = 1 quantises inside the
    launch, at M = 16 in a separate kernel before it."""
    m = synth.gqa28_fp8(1) if fp8 else synth.llama7b_layer(1)
    cm = cloak_lib.CloakModel(m)
    cm.keygen(0x77, 0)
    for t in range(len(m.tensors)):
        cm.shuffle(t, synth.weights_device(m, t, seed=4))
    kinds = {tt.kind: i for i, tt in enumerate(m.tensors)}
    tq, to = kinds[synth.K_Q], kinds[synth.K_O]
    assert m.tensors[tq].n == m.tensors[to].k and m.tensors[to].n == m.tensors[tq].k
    x0 = x_device(m, synth.activations_host(M, m.tensors[tq].k, seed=3))
    s = torch.cuda.Stream()
    bufs = [torch.empty((M, m.tensors[tq if i % 2 == 0 else to].n), dtype=torch.bfloat16, device="cuda")
            for i in range(24)]

    def chain(chained):
        x = x0
        for i in range(24):
            t = tq if i % 2 == 0 else to
            y = bufs[i]
            cm.linear(t, x, y, out_dtype=cloak_lib.OUT_BF16, stream=s.cuda_stream, chained=chained)
            x = y
        return x

    with torch.cuda.stream(s):
        ref = torch_bf16_bits(chain(False))
        torch.cuda.synchronize()
        for b in bufs:
            b.zero_()
        got = torch_bf16_bits(chain(True))
        torch.cuda.synchronize()
    assert np.array_equal(ref, got)
    for b in bufs:
        b.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        out = chain(True)
    for _ in range(3):
        for b in bufs:
            b.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(ref, torch_bf16_bits(out))
    assert torch.isfinite(out.float()).all()
    assert cm.device_status() == 0
    cm.close()
