"""GPU serving step and loop: logits against the FP64 full-model oracle
(normwise 1e-2), a request's results identical alone and in a mixed batch,
and the continuous-batching loop serving a workload to completion with
re-keys in between."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import cloak, serve, synth

pytestmark = pytest.mark.gpu


def small_served(layers=2, page_bytes=None):
    m = synth.small_decoder(layers, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2, d_ff=384,
                            head_dim=128, spare_pages=3, page_bytes=page_bytes)
    return synth.with_lm_head(m, 1000)


@pytest.fixture(scope="module")
def served(cloak_lib):
    m = small_served()
    Ws = synth.weights_host(m, seed=0, std=0.05)
    sm = serve.ServedModel(m, kv_blocks=256, max_blocks=32, twin=True, weights=Ws)
    yield m, Ws, sm
    sm.close()


def run_steps(sm, seqs, uncloaked=False, tiled=False, decode_first=False, tile=64):
    """Prefill each (slot, tokens) fully in one step, then decode 3 steps
    feeding back greedy tokens; returns per slot the list of logits. With
    `tiled`, prefill tokens use query tiles (`tile` tokens, at most 64) and
    decode tokens single rows."""
    dev = "cuda"
    bt = torch.zeros((8, sm.max_blocks), dtype=torch.int32, device=dev)
    for slot, toks in seqs:
        bt[slot] = torch.arange(slot * sm.max_blocks, (slot + 1) * sm.max_blocks, dtype=torch.int32)
    state = {slot: list(toks) for slot, toks in seqs}
    logits = {slot: [] for slot, _ in seqs}
    first = True
    for step in range(4):
        ids, pos, req, samp, tiles, single = [], [], [], [], [], []
        for slot, toks in seqs:
            seq = state[slot]
            if first:
                for t0 in range(0, len(seq), tile):
                    tiles += [len(ids) + t0, min(tile, len(seq) - t0), 0]
                for i, t in enumerate(seq):
                    ids.append(t); pos.append(i); req.append(slot)
            else:
                single.append(len(ids))
                ids.append(seq[-1]); pos.append(len(seq) - 1); req.append(slot)
            samp.append(len(ids) - 1)
        first = False
        T = lambda a: torch.tensor(a, dtype=torch.int32, device=dev)
        out = torch.zeros(len(samp), dtype=torch.int32, device=dev)
        lg = torch.zeros((len(samp), sm.model.vocab), dtype=torch.float32, device=dev)
        if tiled:
            qt = T(tiles).view(-1, 3) if tiles else T([]).view(0, 3)
            sm.step(T(ids), T(pos), T(req), bt, T(samp), out, lg, uncloaked=uncloaked, qtiles=qt,
                    single_rows=T(single), decode_first=decode_first)
        else:
            sm.step(T(ids), T(pos), T(req), bt, T(samp), out, lg, uncloaked=uncloaked)
        torch.cuda.synchronize()
        for k, (slot, _) in enumerate(seqs):
            logits[slot].append(lg[k].cpu().numpy())
            state[slot].append(int(out[k]))
    return logits, state


@pytest.mark.parametrize("tiled,decode_first,tile", [(False, False, 64), (True, False, 64), (True, True, 64),
                                                    (True, True, 48)])
def test_serve_step_matches_full_model_oracle(served, tiled, decode_first, tile):
    """decode_first: the prompt rows take the prefill GEMM, decode rows the
    split-K kernel. Query tiles of 64 or 48 tokens (not aligned to the
    64-key tiles)."""
    m, Ws, sm = served
    toks = list(np.random.default_rng(1).integers(0, 1000, 23 if tile == 64 else 200))
    logits, state = run_steps(sm, [(0, toks)], tiled=tiled, decode_first=decode_first, tile=tile)
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    emb64 = O.bf16_value(O.bf16_bits(synth.embedding_host(1000, 512)))
    seq = state[0]
    ref = O.transformer_logits_f64(m, W64, emb64, seq[:-1])
    L = len(toks)
    for step, lg in enumerate(logits[0]):
        p = L - 1 + step  # position whose next token was sampled
        assert O.relative_error(lg, ref[p]) <= 1e-2, (step, O.relative_error(lg, ref[p]))
        top = np.sort(ref[p])[-2:]
        if top[1] - top[0] > 0.05 * np.std(ref[p]):
            assert seq[L + step] == int(np.argmax(ref[p]))


def test_decode_attention_over_a_long_context(cloak_lib):
    """A prompt of 2,200 tokens: each decode token attends over 18 key
    splits of 128, more than the blocks of one (token, head), so blocks take
    several splits and the last to finish merges them. Logits against the
    FP64 model; the request alone equals the request next to a short one."""
    m = small_served()
    Ws = synth.weights_host(m, seed=0, std=0.05)
    sm = serve.ServedModel(m, kv_blocks=400, max_blocks=160, twin=True, weights=Ws)
    long = list(np.random.default_rng(11).integers(0, 1000, 2200))
    short = list(np.random.default_rng(12).integers(0, 1000, 40))
    la, sa = run_steps(sm, [(0, long)], tiled=True)
    lm, _ = run_steps(sm, [(1, short), (0, long)], tiled=True)
    for x, y in zip(la[0], lm[0]):
        assert np.array_equal(x, y)
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    emb64 = O.bf16_value(O.bf16_bits(synth.embedding_host(1000, 512)))
    seq = sa[0]
    ref = O.transformer_logits_f64(m, W64, emb64, seq[:-1])
    for step, lg in enumerate(la[0]):
        p = 2199 + step
        assert O.relative_error(lg, ref[p]) <= 1e-2, (step, O.relative_error(lg, ref[p]))
    sm.close()


@pytest.mark.parametrize("tiled", [False, True])
def test_request_alone_equals_request_in_a_mix(served, tiled):
    m, Ws, sm = served
    rng = np.random.default_rng(2)
    a = list(rng.integers(0, 1000, 77))
    b = list(rng.integers(0, 1000, 140))
    c = list(rng.integers(0, 1000, 5))
    alone, sa = run_steps(sm, [(0, a)], tiled=tiled)
    mixed, sm_ = run_steps(sm, [(1, b), (0, a), (2, c)], tiled=tiled)
    for x, y in zip(alone[0], mixed[0]):
        assert np.array_equal(x, y)
    assert sa[0] == sm_[0]
    unc, su = run_steps(sm, [(0, a)], uncloaked=True, tiled=tiled)
    for x, y in zip(alone[0], unc[0]):
        assert np.array_equal(x, y)


def test_request_alone_equals_request_in_a_wide_mix(served):
    """A mix of over 256 tokens (the size where standalone linears switch to
    the prefill GEMM) still gives the request the numbers it gets alone."""
    m, Ws, sm = served
    rng = np.random.default_rng(3)
    a = list(rng.integers(0, 1000, 61))
    b = list(rng.integers(0, 1000, 230))
    alone, sa = run_steps(sm, [(0, a)], tiled=True)
    mixed, sm_ = run_steps(sm, [(1, b), (0, a)], tiled=True)
    for x, y in zip(alone[0], mixed[0]):
        assert np.array_equal(x, y)
    assert sa[0] == sm_[0]


def test_decode_rows_and_prompt_rows_in_one_step(served):
    """With decode tokens first (prompt rows through the prefill GEMM, decode
    rows through the split-K kernel), a request's numbers do not depend on
    the other requests of the step: request 0 decoding while request 1's
    prompt is in the same step gets the logits it gets alone, and so does
    request 1."""
    m, Ws, sm = served
    dev = "cuda"
    rng = np.random.default_rng(4)
    a = list(rng.integers(0, 1000, 37))
    b = list(rng.integers(0, 1000, 290))
    bt = torch.zeros((8, sm.max_blocks), dtype=torch.int32, device=dev)
    for slot in range(3):
        bt[slot] = torch.arange(slot * sm.max_blocks, (slot + 1) * sm.max_blocks, dtype=torch.int32)
    T = lambda v: torch.tensor(v, dtype=torch.int32, device=dev)

    def step(decodes, prompts):
        """decodes: [(slot, token, position)]; prompts: [(slot, tokens)] whole
        prompts from position 0. Returns the logits of every sampled row."""
        ids, pos, req, samp, tiles, single = [], [], [], [], [], []
        for slot, tok, p in decodes:
            single.append(len(ids))
            ids.append(tok); pos.append(p); req.append(slot); samp.append(len(ids) - 1)
        for slot, toks in prompts:
            for t0 in range(0, len(toks), 64):
                tiles += [len(ids) + t0, min(64, len(toks) - t0), 0]
            for i, t in enumerate(toks):
                ids.append(t); pos.append(i); req.append(slot)
            samp.append(len(ids) - 1)
        out = torch.zeros(len(samp), dtype=torch.int32, device=dev)
        lg = torch.zeros((len(samp), sm.model.vocab), dtype=torch.float32, device=dev)
        qt = T(tiles).view(-1, 3) if tiles else T([]).view(0, 3)
        sm.step(T(ids), T(pos), T(req), bt, T(samp), out, lg, qtiles=qt, single_rows=T(single),
                decode_first=True)
        torch.cuda.synchronize()
        return lg.cpu().numpy(), out.cpu().numpy()

    # alone: request 0 (slot 0) prefills, then decodes one token; request 1
    # (slot 1) prefills
    la0, oa0 = step([], [(0, a)])
    la1, _ = step([(0, int(oa0[0]), len(a))], [])
    lb, _ = step([], [(2, b)])
    # mixed: request 0 prefills (slot 1), then its decode token shares a
    # step with request 1's prompt (slot 2 again)
    lm0, om0 = step([], [(1, a)])
    lm1, _ = step([(1, int(om0[0]), len(a))], [(2, b)])
    assert np.array_equal(la0[0], lm0[0])
    assert np.array_equal(la1[0], lm1[0])  # decode row next to a prompt
    assert np.array_equal(lb[0], lm1[1])   # prompt next to a decode row


def test_server_serves_a_workload_with_rekeys(cloak_lib):
    m = small_served()
    Ws = synth.weights_host(m, seed=0, std=0.05)
    work = [(0.01 * i, np.random.default_rng(10 + i).integers(0, 1000, 20 + 7 * i).astype(np.int32), 4 + i % 5)
            for i in range(10)]
    outs = []
    for period, conc in ((None, True), (0.02, True), (0.02, False)):
        sm = serve.ServedModel(m, kv_blocks=128, max_blocks=16, weights=Ws)
        srv = serve.Server(sm, max_running=4, token_budget=64, rekey_period=period,
                           rekey_concurrent=conc)
        done, wall = srv.run(work)
        assert len(done) == 10 and all(len(r.out) == r.max_new for r in done)
        st = serve.latency_stats(done, wall)
        assert st["tokens"] == sum(w[2] for w in work) and st["ttft_p50_s"] is not None
        outs.append({r.rid: r.out for r in done})
        if period:
            assert len(srv.rekeys) >= 1
            assert all(r["mode"] == ("concurrent" if conc else "between_steps") for r in srv.rekeys)
            # every re-key ran to its end: the tables are those of the last epoch
            tb = O.keygen(O.OracleModel(m), sm.key, sm.epoch)
            assert np.array_equal(sm.cm.table(cloak.TAB_TILE_SLOT), tb.tile_slot)
        assert sm.cm.device_status() == 0
        sm.close()
    # continuous batching and re-keys (between steps or concurrent) do not change results
    assert outs[0] == outs[1] == outs[2]


def test_server_on_the_vmm_view(cloak_lib):
    """Served through the virtual view of a page-chunked arena (Section 4.2
    physical page remapping), with re-keys between steps and concurrent ones
    (the steps read the arena while pages move, the view again once it is
    remapped): the same tokens as the arena read."""
    m = small_served(page_bytes=2 << 20)
    Ws = synth.weights_host(m, seed=0, std=0.05)
    work = [(0.01 * i, np.random.default_rng(30 + i).integers(0, 1000, 25 + 9 * i).astype(np.int32), 3 + i % 4)
            for i in range(8)]
    outs = []
    for vmm, conc in ((False, True), (True, True), (True, False)):
        sm = serve.ServedModel(m, kv_blocks=128, max_blocks=16, weights=Ws, vmm=vmm)
        srv = serve.Server(sm, max_running=4, token_budget=64, rekey_period=0.02, rekey_concurrent=conc)
        done, wall = srv.run(work)
        assert len(done) == 8 and len(srv.rekeys) >= 1
        outs.append({r.rid: r.out for r in done})
        if vmm:
            assert sm.cm.vmm_stats()["remaps"] == 1 + len(srv.rekeys)
            assert not sm._rekeying
        assert sm.cm.device_status() == 0
        sm.close()
    assert outs[0] == outs[1] == outs[2]


@pytest.mark.parametrize("vmm", [False, True])
def test_cloaked_embedding(cloak_lib, vmm):
    """The embedding table as a cloaked tensor (looked up through the gather
    table): the same logits as the plain BF16 table, bit for bit, through the
    arena, the uncloaked twin and (page-chunked arena) the VMM view; and the
    full-model oracle's logits within 1e-2."""
    pb = (2 << 20) if vmm else None
    plain = small_served(page_bytes=pb)
    m = synth.small_decoder(2, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2, d_ff=384,
                            head_dim=128, spare_pages=3, page_bytes=pb)
    m = synth.with_lm_head(m, 1000, cloaked_embedding=True)
    assert m.tensors[-1].kind == synth.K_EMBED and m.tensors[-1].layer == m.tensors[-2].layer + 1
    Ws = synth.weights_host(plain, seed=0, std=0.05)
    toks = list(np.random.default_rng(5).integers(0, 1000, 30))
    a = serve.ServedModel(plain, kv_blocks=256, max_blocks=32, twin=not vmm, weights=Ws, vmm=vmm)
    b = serve.ServedModel(m, kv_blocks=256, max_blocks=32, twin=not vmm, weights=Ws + [None], vmm=vmm)
    assert b.embed_tensor == len(m.tensors) - 1 and b.embedding is None
    la, sa = run_steps(a, [(0, toks)], tiled=True)
    lb, sb = run_steps(b, [(0, toks)], tiled=True)
    for x, y in zip(la[0], lb[0]):
        assert np.array_equal(x, y)
    assert sa == sb
    if not vmm:
        lu, su = run_steps(b, [(0, toks)], tiled=True, uncloaked=True)
        for x, y in zip(la[0], lu[0]):
            assert np.array_equal(x, y)
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    emb64 = O.bf16_value(O.bf16_bits(synth.embedding_host(1000, 512)))
    ref = O.transformer_logits_f64(plain, W64, emb64, sb[0][:-1])
    assert O.relative_error(lb[0][0], ref[29]) <= 1e-2
    assert a.cm.device_status() == 0 and b.cm.device_status() == 0
    a.close()
    b.close()


def test_server_request_alone_equals_request_in_a_poisson_mix(cloak_lib):
    """Continuous batching end to end: eight requests with Poisson arrivals
    served through Server.run with at most three running at once (later ones
    admitted mid-flight as earlier ones finish, prompts split into prefill
    chunks that share steps with other requests' decode tokens), then each
    request served alone. Every request's greedy tokens are the same in both,
    and they are the FP64 full-model oracle's argmax wherever its top two
    logits are clearly apart."""
    m = small_served()
    Ws = synth.weights_host(m, seed=0, std=0.05)
    arr = synth.requests_poisson(80.0, 0.2, 1000, seed=7, prompt_median=60, prompt_sigma=0.6,
                                 prompt_min=9, prompt_max=150)
    work = [(a, np.asarray(p, np.int32), 3 + i % 6) for i, (a, p, _) in enumerate(arr[:8])]
    assert len(work) == 8
    sm = serve.ServedModel(m, kv_blocks=256, max_blocks=16, weights=Ws)
    srv = serve.Server(sm, max_running=3, token_budget=48, rekey_period=None)
    done, _ = srv.run(work)
    assert len(done) == 8 and all(len(r.out) == r.max_new for r in done)
    mixed = {r.rid: list(r.out) for r in done}
    solo_steps = 0
    for rid, (a, p, n) in enumerate(work):
        solo = serve.Server(sm, max_running=3, token_budget=48, rekey_period=None)
        d, _ = solo.run([(0.0, p, n)])
        assert d[0].out == mixed[rid], rid
        solo_steps += solo.steps
    # the mix really mixed: requests shared steps
    assert srv.steps < solo_steps, (srv.steps, solo_steps)
    assert sm.cm.device_status() == 0
    sm.close()
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    emb64 = O.bf16_value(O.bf16_bits(synth.embedding_host(1000, 512)))
    checked = 0
    for rid, (a, p, n) in enumerate(work):
        seq = list(p) + mixed[rid]
        ref = O.transformer_logits_f64(m, W64, emb64, seq[:-1])
        for j in range(n):
            row = ref[len(p) - 1 + j]
            top = np.sort(row)[-2:]
            if top[1] - top[0] > 0.05 * np.std(row):
                assert mixed[rid][j] == int(np.argmax(row)), (rid, j)
                checked += 1
    assert checked >= 20
