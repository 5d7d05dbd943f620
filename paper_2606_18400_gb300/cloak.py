"""Python binding of libcloak (include/cloak.h): argument marshalling only.

Every entry point of the C ABI is exposed under its own name and takes the
same arguments (device pointers as ints, streams as ints). ``CloakModel`` is
a thin convenience wrapper that accepts torch tensors; all computation runs
in the CUDA library. If the library is missing or fails to load, every call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcloak.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_STATE, E_UNSUPPORTED, E_DRAWS = 0, -1, -2, -3, -4, -5, -6, -7
F32, BF16, E4M3 = 0, 1, 2
MODEL_TWIN, MODEL_VMM, MODEL_TILE_REKEY = 1, 2, 4
TAB_LAYER_PERM, TAB_GROUP_PERM, TAB_TENSOR_BASE, TAB_TILE_PERM, TAB_PAGE_ALLOC, TAB_TILE_SLOT = range(6)
LINEAR_UNCLOAKED, LINEAR_RELU, LINEAR_VMM, LINEAR_CHAINED = 1, 2, 8, 16
SERVE_DECODE_FIRST = 4
OUT_F32, OUT_BF16 = 0, 1

_STATUS = {0: "CLOAK_OK", -1: "CLOAK_E_INVAL", -2: "CLOAK_E_NOMEM", -3: "CLOAK_E_CUDA",
           -4: "CLOAK_E_TIMEOUT", -5: "CLOAK_E_STATE", -6: "CLOAK_E_UNSUPPORTED", -7: "CLOAK_E_DRAWS"}


class CloakError(RuntimeError):
    def __init__(self, fn, status, msg=""):
        super().__init__(f"{fn} -> {_STATUS.get(status, status)} {msg}".strip())
        self.status = status


class TensorDesc(C.Structure):
    _fields_ = [(f, C.c_int32) for f in ("n", "k", "layer", "kind", "perm_group", "perm_axis", "perm_group2")]


class GroupDesc(C.Structure):
    _fields_ = [(f, C.c_int32) for f in ("n_units", "unit", "parent", "ratio")]


class ModelDesc(C.Structure):
    _fields_ = [("num_tensors", C.c_int32), ("num_groups", C.c_int32),
                ("tensors", C.POINTER(TensorDesc)), ("groups", C.POINTER(GroupDesc)),
                ("dtype", C.c_int32), ("tile_r", C.c_int32), ("tile_c", C.c_int32),
                ("spare_pages", C.c_int32), ("tile_scope", C.c_int32), ("flags", C.c_int32),
                ("page_bytes", C.c_int64)]


class StackDesc(C.Structure):
    _fields_ = [("num_layers", C.c_int32), ("layer_tensors", C.POINTER(C.c_int32)),
                ("d_model", C.c_int32), ("n_heads", C.c_int32), ("n_kv_heads", C.c_int32),
                ("head_dim", C.c_int32), ("d_ff", C.c_int32), ("rms_eps", C.c_float)]


class ServeDesc(C.Structure):
    _fields_ = [("stack", StackDesc), ("lm_head", C.c_int32), ("vocab", C.c_int32),
                ("embedding", C.c_void_p), ("k_cache", C.c_void_p), ("v_cache", C.c_void_p),
                ("num_blocks", C.c_int32), ("max_blocks", C.c_int32), ("rope_theta", C.c_float),
                ("embed_tensor", C.c_int32)]


class MoeDesc(C.Structure):
    _fields_ = [("n_experts", C.c_int32), ("top_k", C.c_int32), ("d_model", C.c_int32), ("d_ff", C.c_int32),
                ("router", C.c_int32), ("expert_group", C.c_int32),
                ("expert_tensors", C.POINTER(C.c_int32))]


class TuneResult(C.Structure):
    _fields_ = [("chunk", C.c_int32), ("stages", C.c_int32), ("grid", C.c_int32), ("us", C.c_float),
                ("default_us", C.c_float), ("candidates", C.c_int32), ("l2_prefetch", C.c_int32)]


class ServeBatch(C.Structure):
    _fields_ = [("num_tokens", C.c_int32), ("num_sample", C.c_int32), ("flags", C.c_int32),
                ("token_ids", C.c_void_p), ("positions", C.c_void_p), ("req_slots", C.c_void_p),
                ("block_tables", C.c_void_p), ("sample_rows", C.c_void_p),
                ("out_tokens", C.c_void_p), ("out_logits", C.c_void_p),
                ("num_qtiles", C.c_int32), ("num_single", C.c_int32),
                ("qtiles", C.c_void_p), ("single_rows", C.c_void_p)]


# (name, restype, argtypes); the list is the ABI this binding expects
_vp, _i32, _i64, _u32, _u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
SIGNATURES = [
    ("cloak_create", _i32, [C.POINTER(ModelDesc), _i32, C.POINTER(_vp)]),
    ("cloak_destroy", _i32, [_vp]),
    ("cloak_geometry", _i32, [_vp, C.POINTER(_i64)]),
    ("cloak_keygen", _i32, [_vp, _u64, _u32, _vp]),
    ("cloak_export_table", _i32, [_vp, _i32, C.POINTER(_u32), C.c_size_t]),
    ("cloak_shuffle", _i32, [_vp, _i32, _vp, _vp]),
    ("cloak_unshuffle", _i32, [_vp, _i32, _vp, _i32, _vp]),
    ("cloak_scales", _i32, [_vp, _i32, C.POINTER(_vp)]),
    ("cloak_arena", _i32, [_vp, _i32, C.POINTER(_vp), C.POINTER(_i64)]),
    ("cloak_linear", _i32, [_vp, _i32, _vp, _vp, _i32, _i32, _i32, _vp]),
    ("cloak_linear_batch", _i32, [_vp, _i32, C.POINTER(_i32), C.POINTER(_vp), C.POINTER(_vp), _i32,
                                  _i32, _i32, _vp]),
    ("cloak_linear_host", _i32, [_vp, _i32, _vp, _vp, _i32, _i32, _i32, _vp]),
    ("cloak_linear_batch_host", _i32, [_vp, _i32, C.POINTER(_i32), C.POINTER(_vp), C.POINTER(_vp), _i32,
                                       _i32, _i32, _vp]),
    ("cloak_linear_noalloc", _i32, [_vp, _i32, _vp, _vp, _i32, _i32, _i32, _vp]),
    ("cloak_stack_decode", _i32, [_vp, C.POINTER(StackDesc), _vp, _i32, _i32, _vp]),
    ("cloak_serve_step", _i32, [_vp, C.POINTER(ServeDesc), C.POINTER(ServeBatch), _vp]),
    ("cloak_rekey", _i32, [_vp, _u64, _u32, _vp]),
    ("cloak_rekey_begin", _i32, [_vp, _u64, _u32, _vp]),
    ("cloak_autotune", _i32, [_vp, _i32, C.POINTER(_i32), C.POINTER(_vp), C.POINTER(_vp), _i32, _i32, _vp,
                              C.POINTER(TuneResult)]),
    ("cloak_autotune_stack", _i32, [_vp, C.POINTER(StackDesc), _vp, _i32, _vp, C.POINTER(TuneResult)]),
    ("cloak_tune_save", _i32, [_vp, C.c_char_p]),
    ("cloak_tune_load", _i32, [_vp, C.c_char_p, C.POINTER(_i32)]),
    ("cloak_tune_clear", _i32, [_vp]),
    ("cloak_rekey_advance", _i32, [_vp, _vp, _vp, C.POINTER(_i32)]),
    ("cloak_device_status", _i32, [_vp]),
    ("cloak_check_waits", _i32, [_vp, _vp]),
    ("cloak_vmm_stats", _i32, [_vp, C.POINTER(_i64)]),
    ("cloak_upload", _i32, [_vp, C.POINTER(_vp), _i32, _vp]),
    ("cloak_moe_ffn", _i32, [_vp, C.POINTER(MoeDesc), _vp, _vp, _i32, _i32, _vp, _vp, _vp]),
    ("cloak_last_error", C.c_char_p, [_vp]),
    ("cloak_launch_count", _i64, [_vp]),
    ("cloak_version", C.c_char_p, []),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libcloak.so (raises if it is missing: build it with
    ``paper_2606_18400_gb300.build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libcloak.so not found at {path}; build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(name, rc, ctx=None):
    if rc != OK:
        msg = ""
        if ctx:
            msg = (load().cloak_last_error(ctx) or b"").decode()
        raise CloakError(name, rc, msg)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream


# ---------------------------------------------------------------- thin C names

def cloak_create(desc: ModelDesc, device: int = 0):
    ctx = C.c_void_p()
    _check("cloak_create", load().cloak_create(C.byref(desc), device, C.byref(ctx)))
    return ctx


def cloak_destroy(ctx):
    _check("cloak_destroy", load().cloak_destroy(ctx))


def cloak_geometry(ctx):
    out = (C.c_int64 * 8)()
    _check("cloak_geometry", load().cloak_geometry(ctx, out), ctx)
    return list(out)


def cloak_keygen(ctx, key: int, epoch: int, stream=None):
    _check("cloak_keygen", load().cloak_keygen(ctx, key & (2**64 - 1), epoch, _stream(stream)), ctx)


def cloak_export_table(ctx, which: int, count: int):
    import numpy as np
    out = np.zeros(max(count, 1), np.uint32)
    _check("cloak_export_table", load().cloak_export_table(
        ctx, which, out.ctypes.data_as(C.POINTER(C.c_uint32)), out.size), ctx)
    return out[:count]


def cloak_shuffle(ctx, tensor: int, logical_dev: int, stream=None):
    _check("cloak_shuffle", load().cloak_shuffle(ctx, tensor, logical_dev, _stream(stream)), ctx)


def cloak_unshuffle(ctx, tensor: int, logical_dev: int, from_twin: int = 0, stream=None):
    _check("cloak_unshuffle", load().cloak_unshuffle(ctx, tensor, logical_dev, from_twin,
                                                     _stream(stream)), ctx)


def cloak_scales(ctx, tensor: int) -> int:
    p = C.c_void_p()
    _check("cloak_scales", load().cloak_scales(ctx, tensor, C.byref(p)), ctx)
    return p.value


def cloak_arena(ctx, which: int = 0):
    p, n = C.c_void_p(), C.c_int64()
    _check("cloak_arena", load().cloak_arena(ctx, which, C.byref(p), C.byref(n)), ctx)
    return p.value, n.value


def cloak_linear(ctx, tensor: int, x_dev: int, y_dev: int, M: int, out_dtype: int,
                 flags: int = 0, stream=None):
    _check("cloak_linear", load().cloak_linear(ctx, tensor, x_dev, y_dev, M, out_dtype, flags,
                                               _stream(stream)), ctx)


def cloak_linear_batch(ctx, tensors, x_devs, y_devs, M: int, out_dtype: int, flags: int = 0,
                       stream=None):
    n = len(tensors)
    ta = (C.c_int32 * n)(*tensors)
    xa = (C.c_void_p * n)(*x_devs)
    ya = (C.c_void_p * n)(*y_devs)
    _check("cloak_linear_batch", load().cloak_linear_batch(ctx, n, ta, xa, ya, M, out_dtype, flags,
                                                           _stream(stream)), ctx)


def cloak_linear_host(ctx, tensor: int, x_host: int, y_host: int, M: int, out_dtype: int,
                      flags: int = 0, stream=None):
    _check("cloak_linear_host", load().cloak_linear_host(ctx, tensor, x_host, y_host, M, out_dtype,
                                                         flags, _stream(stream)), ctx)


def cloak_linear_batch_host(ctx, tensors, x_hosts, y_hosts, M: int, out_dtype: int, flags: int = 0,
                            stream=None):
    n = len(tensors)
    ta = (C.c_int32 * n)(*tensors)
    xa = (C.c_void_p * n)(*x_hosts)
    ya = (C.c_void_p * n)(*y_hosts)
    _check("cloak_linear_batch_host", load().cloak_linear_batch_host(ctx, n, ta, xa, ya, M, out_dtype,
                                                                     flags, _stream(stream)), ctx)


def cloak_linear_noalloc(ctx, tensor: int, x_dev: int, y_dev: int, M: int, out_dtype: int,
                         flags: int = 0, stream=None):
    _check("cloak_linear_noalloc", load().cloak_linear_noalloc(ctx, tensor, x_dev, y_dev, M, out_dtype,
                                                               flags, _stream(stream)), ctx)


def cloak_stack_decode(ctx, desc: StackDesc, h_dev: int, M: int, flags: int = 0, stream=None):
    _check("cloak_stack_decode", load().cloak_stack_decode(ctx, C.byref(desc), h_dev, M, flags,
                                                           _stream(stream)), ctx)


def cloak_serve_step(ctx, desc: ServeDesc, batch: ServeBatch, stream=None):
    _check("cloak_serve_step", load().cloak_serve_step(ctx, C.byref(desc), C.byref(batch),
                                                       _stream(stream)), ctx)


def cloak_rekey(ctx, key: int, new_epoch: int, stream=None):
    _check("cloak_rekey", load().cloak_rekey(ctx, key & (2**64 - 1), new_epoch, _stream(stream)), ctx)


def cloak_autotune(ctx, tensors, x_devs, y_devs, M: int, out_dtype: int, stream=None) -> dict:
    n = len(tensors)
    ta = (C.c_int32 * n)(*tensors)
    xa = (C.c_void_p * n)(*x_devs)
    ya = (C.c_void_p * n)(*y_devs)
    r = TuneResult()
    _check("cloak_autotune", load().cloak_autotune(ctx, n, ta, xa, ya, M, out_dtype, _stream(stream),
                                                   C.byref(r)), ctx)
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def cloak_autotune_stack(ctx, desc, h_dev: int, M: int, stream=None) -> dict:
    r = TuneResult()
    _check("cloak_autotune_stack", load().cloak_autotune_stack(ctx, C.byref(desc), h_dev, M, _stream(stream),
                                                               C.byref(r)), ctx)
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def cloak_tune_save(ctx, path: str):
    _check("cloak_tune_save", load().cloak_tune_save(ctx, str(path).encode()), ctx)


def cloak_tune_load(ctx, path: str) -> int:
    n = C.c_int32(0)
    _check("cloak_tune_load", load().cloak_tune_load(ctx, str(path).encode(), C.byref(n)), ctx)
    return n.value


def cloak_tune_clear(ctx):
    _check("cloak_tune_clear", load().cloak_tune_clear(ctx), ctx)


def cloak_rekey_begin(ctx, key: int, new_epoch: int, side_stream):
    _check("cloak_rekey_begin", load().cloak_rekey_begin(ctx, key & (2**64 - 1), new_epoch,
                                                         _stream(side_stream)), ctx)


def cloak_rekey_advance(ctx, serve_stream, side_stream) -> bool:
    done = C.c_int32(0)
    _check("cloak_rekey_advance", load().cloak_rekey_advance(ctx, _stream(serve_stream),
                                                             _stream(side_stream), C.byref(done)), ctx)
    return bool(done.value)


def cloak_device_status(ctx) -> int:
    return load().cloak_device_status(ctx)


def cloak_last_error(ctx) -> str:
    return (load().cloak_last_error(ctx) or b"").decode()


def cloak_launch_count(ctx) -> int:
    return load().cloak_launch_count(ctx)


def cloak_version() -> str:
    return load().cloak_version().decode()


# ------------------------------------------------------------ convenience

class _DevArray:
    """Minimal __cuda_array_interface__ exporter to view context-owned
    device memory from torch."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def cloak_vmm_stats(ctx) -> dict:
    out = (C.c_int64 * 4)()
    _check("cloak_vmm_stats", load().cloak_vmm_stats(ctx, out), ctx)
    return {"pages_remapped": out[0], "remaps": out[1], "chunks": out[2], "remap_us": out[3]}


def cloak_check_waits(ctx, stream=None):
    _check("cloak_check_waits", load().cloak_check_waits(ctx, _stream(stream)), ctx)


def cloak_moe_ffn(ctx, desc, x_ptr: int, y_ptr: int, M: int, flags: int = 0, experts_out: int = None,
                  logits_out: int = None, stream=None):
    _check("cloak_moe_ffn", load().cloak_moe_ffn(ctx, C.byref(desc), x_ptr, y_ptr, M, flags, experts_out,
                                                 logits_out, _stream(stream)), ctx)


def cloak_upload(ctx, host_ptrs, threads: int = 0, stream=None):
    arr = (C.c_void_p * len(host_ptrs))(*host_ptrs)
    _check("cloak_upload", load().cloak_upload(ctx, arr, threads, _stream(stream)), ctx)


def _storage(uncloaked=False, vmm=False):
    """Flags choosing the weight storage a read goes through."""
    return (LINEAR_UNCLOAKED if uncloaked else 0) | (LINEAR_VMM if vmm else 0)


def _wrap_device(ptr, shape, typestr, device):
    import torch
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device=f"cuda:{device}")


class CloakModel:
    """A context for a ``synth.Model``: owns the ctypes descriptor and the
    C context, and passes torch tensors' device pointers to the C calls."""

    def __init__(self, model: "synth.Model", device: int = 0, twin: bool = False, vmm: bool = False):
        self.model = model
        T, G = len(model.tensors), len(model.groups)
        self._t = (TensorDesc * T)(*[TensorDesc(t.n, t.k, t.layer, t.kind, t.perm_group, t.perm_axis,
                                                getattr(t, "perm_group2", -1)) for t in model.tensors])
        self._g = (GroupDesc * max(G, 1))(*[GroupDesc(g.n_units, g.unit, g.parent, g.ratio)
                                            for g in model.groups])
        self.desc = ModelDesc(T, G, self._t, self._g, model.dtype, model.tile_r, model.tile_c,
                              model.spare_pages, model.tile_scope,
                              (MODEL_TWIN if twin else 0) | (MODEL_VMM if vmm else 0) |
                              (MODEL_TILE_REKEY if getattr(model, "tile_rekey", False) else 0),
                              model.page_bytes)
        self.device = device
        self.ctx = cloak_create(self.desc, device)
        (self.L, self.G, self.tpp, self.NP, self.NPS, self.U, self.tile_bytes,
         self.esize) = cloak_geometry(self.ctx)

    def close(self):
        if self.ctx:
            cloak_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def keygen(self, key, epoch=0, stream=None):
        cloak_keygen(self.ctx, key, epoch, stream)

    def table(self, which):
        n = {TAB_LAYER_PERM: self.L, TAB_GROUP_PERM: self.U,
             TAB_TENSOR_BASE: len(self.model.tensors), TAB_TILE_PERM: self.G,
             TAB_PAGE_ALLOC: self.NPS, TAB_TILE_SLOT: self.G}[which]
        return cloak_export_table(self.ctx, which, n)

    def shuffle(self, t, w_f32, stream=None):
        import torch
        assert w_f32.dtype == torch.float32 and w_f32.is_cuda and w_f32.is_contiguous()
        tt = self.model.tensors[t]
        assert tuple(w_f32.shape) == (tt.n, tt.k)
        cloak_shuffle(self.ctx, t, w_f32.data_ptr(), stream)

    def upload(self, weights, threads=0, stream=None):
        """Keyed upload of every tensor from host FP32 arrays [n, k] (numpy,
        C-contiguous): pages assembled on the host, sent in physical order."""
        import numpy as np
        ws = [np.ascontiguousarray(w, dtype=np.float32) for w in weights]
        assert len(ws) == len(self.model.tensors)
        for w, t in zip(ws, self.model.tensors):
            assert w.shape == (t.n, t.k)
        cloak_upload(self.ctx, [w.ctypes.data for w in ws], threads, stream)

    def unshuffle(self, t, from_twin=False, stream=None):
        import torch
        tt = self.model.tensors[t]
        dt = {F32: torch.float32, BF16: torch.int16, E4M3: torch.uint8}[self.model.dtype]
        out = torch.empty((tt.n, tt.k), dtype=dt, device=f"cuda:{self.device}")
        cloak_unshuffle(self.ctx, t, out.data_ptr(), int(from_twin), stream)
        return out

    def scales(self, t):
        """FP32 per-stored-row scales of tensor t (a device copy)."""
        import torch
        torch.cuda.synchronize(self.device)
        return _wrap_device(cloak_scales(self.ctx, t), (self.model.tensors[t].n,), "<f4",
                            self.device).clone()

    def linear(self, t, x, y=None, out_dtype=OUT_BF16, uncloaked=False, relu=False, stream=None,
               vmm=False, chained=False):
        import torch
        tt = self.model.tensors[t]
        M = x.shape[0]
        if y is None:
            y = torch.empty((M, tt.n), device=x.device,
                            dtype=torch.float32 if out_dtype == OUT_F32 else torch.bfloat16)
        flags = _storage(uncloaked, vmm) | (LINEAR_RELU if relu else 0) | (LINEAR_CHAINED if chained else 0)
        cloak_linear(self.ctx, t, x.data_ptr(), y.data_ptr(), M, out_dtype, flags, stream)
        return y

    def linear_batch(self, tensors, xs, ys=None, out_dtype=OUT_BF16, uncloaked=False, relu=False,
                     stream=None, vmm=False, chained=False):
        import torch
        M = xs[0].shape[0]
        if ys is None:
            ys = [torch.empty((M, self.model.tensors[t].n), device=xs[0].device,
                              dtype=torch.float32 if out_dtype == OUT_F32 else torch.bfloat16)
                  for t in tensors]
        flags = _storage(uncloaked, vmm) | (LINEAR_RELU if relu else 0) | (LINEAR_CHAINED if chained else 0)
        cloak_linear_batch(self.ctx, list(tensors), [x.data_ptr() for x in xs],
                           [y.data_ptr() for y in ys], M, out_dtype, flags, stream)
        return ys

    def stack_desc(self, eps=1e-5):
        """Descriptor of the decoder stack of this model (tensor kinds q, k,
        v, o, gate, up, down per layer)."""
        m = self.model
        order = []
        layers = sorted({t.layer for t in m.tensors if t.kind == synth.K_Q})
        for l in layers:
            ts = {t.kind: i for i, t in enumerate(m.tensors) if t.layer == l}
            order += [ts[k] for k in (synth.K_Q, synth.K_K, synth.K_V, synth.K_O, synth.K_GATE,
                                      synth.K_UP, synth.K_DOWN)]
        self._stack_tensors = (C.c_int32 * len(order))(*order)
        return StackDesc(len(layers), self._stack_tensors, m.d_model, m.n_heads, m.n_kv_heads,
                         m.head_dim, m.d_ff, eps)

    def moe_desc(self, layer=0):
        """Descriptor of MoE FFN block `layer` of a ``synth.moe_block`` model."""
        m = self.model
        flat = [t for e in m.expert_tensors[layer] for t in e]
        arr = (C.c_int32 * len(flat))(*flat)
        d = MoeDesc(m.n_experts, m.top_k, m.d_model, m.d_ff, m.router_tensors[layer],
                    m.expert_groups[layer], arr)
        d._keep = arr
        return d

    def moe_ffn(self, x, desc=None, layer=0, uncloaked=False, vmm=False, experts_out=None,
                logits_out=None, stream=None):
        """MoE FFN of BF16 x [M, d_model] -> FP32 y [M, d_model]."""
        import torch
        assert x.dtype == torch.bfloat16 and x.is_cuda and x.is_contiguous()
        d = desc or self.moe_desc(layer)
        y = torch.empty((x.shape[0], self.model.d_model), dtype=torch.float32, device=x.device)
        cloak_moe_ffn(self.ctx, d, x.data_ptr(), y.data_ptr(), x.shape[0], _storage(uncloaked, vmm),
                      experts_out.data_ptr() if experts_out is not None else None,
                      logits_out.data_ptr() if logits_out is not None else None, stream)
        return y

    def stack_decode(self, h, uncloaked=False, desc=None, stream=None, vmm=False):
        """One decode step of the whole stack; h: FP32 [M, d_model], in place."""
        import torch
        assert h.dtype == torch.float32 and h.is_cuda and h.is_contiguous()
        d = desc or self.stack_desc()
        cloak_stack_decode(self.ctx, d, h.data_ptr(), h.shape[0], _storage(uncloaked, vmm), stream)
        return h

    def rekey(self, key, new_epoch, stream=None):
        cloak_rekey(self.ctx, key, new_epoch, stream)

    def autotune_stack(self, h, desc=None, stream=None) -> dict:
        """Tune the layer-stack launch for h's batch (h is not changed)."""
        return cloak_autotune_stack(self.ctx, desc or self.stack_desc(), h.data_ptr(), h.shape[0], stream)

    def autotune(self, tensors, xs, ys=None, out_dtype=OUT_BF16, stream=None) -> dict:
        """Tune the launch shape of linear_batch(tensors, xs) (ys overwritten)."""
        import torch
        M = xs[0].shape[0]
        if ys is None:
            ys = [torch.empty((M, self.model.tensors[t].n), device=xs[0].device,
                              dtype=torch.float32 if out_dtype == OUT_F32 else torch.bfloat16)
                  for t in tensors]
        return cloak_autotune(self.ctx, list(tensors), [x.data_ptr() for x in xs],
                              [y.data_ptr() for y in ys], M, out_dtype, stream)

    def tune_save(self, path):
        cloak_tune_save(self.ctx, path)

    def tune_load(self, path) -> int:
        return cloak_tune_load(self.ctx, path)

    def tune_clear(self):
        cloak_tune_clear(self.ctx)

    def rekey_begin(self, key, new_epoch, side_stream):
        cloak_rekey_begin(self.ctx, key, new_epoch, side_stream)

    def rekey_advance(self, serve_stream, side_stream) -> bool:
        return cloak_rekey_advance(self.ctx, serve_stream, side_stream)

    def arena_bytes(self, which=0):
        """The arena (0), the twin (1) or the virtual view of a VMM context (2)
        as a uint8 device view (no copy)."""
        import torch
        ptr, n = cloak_arena(self.ctx, which)
        torch.cuda.synchronize(self.device)
        return _wrap_device(ptr, (n,), "|u1", self.device)

    def device_status(self):
        return cloak_device_status(self.ctx)

    def check_waits(self, stream=None):
        """Run the bounded-wait self-test (raises if a wait did not time out)."""
        cloak_check_waits(self.ctx, stream)

    def vmm_stats(self) -> dict:
        return cloak_vmm_stats(self.ctx)

    def launches(self):
        return cloak_launch_count(self.ctx)
