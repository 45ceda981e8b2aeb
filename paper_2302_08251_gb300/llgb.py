"""Thin ctypes binding of the C ABI in ``include/llgb.h``.

Argument marshalling only: every step of a copy, pack, unpack or n-body step
runs in the CUDA library ``libllgb.so``.  The library must have been built
(``paper_2302_08251_gb300.build.build()``); loading raises if it is missing.
There is no CPU fallback.

The raw entry points keep their C names (``llgb_copy`` ...); ``Record`` and
``View`` manage handle lifetimes and, for convenience, device blobs allocated
as torch tensors (PyTorch supplies memory and streams, nothing else).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

TYPES = ["u8", "u16", "u32", "u64", "i8", "i16", "i32", "i64",
         "f16", "bf16", "f32", "f64"]
TYPE_ID = {t: k for k, t in enumerate(TYPES)}
TYPE_SIZE = {"u8": 1, "u16": 2, "u32": 4, "u64": 8, "i8": 1, "i16": 2, "i32": 4,
             "i64": 8, "f16": 2, "bf16": 2, "f32": 4, "f64": 8}
INDEX_TYPES = {"i16": 0, "u16": 1, "i32": 2, "u32": 3, "i64": 4, "u64": 5}
KIND_ID = {"aos": 0, "soa_sb": 1, "soa_mb": 2, "aosoa": 3, "bitpack_int": 4,
           "bitpack_float": 5, "bytesplit": 6, "changetype": 7, "null": 8, "split": 9}
MAX_CT = 4

OK = 0
ERR_INVALID_ARG, ERR_INDEX_OVERFLOW, ERR_MISMATCH, ERR_UNSUPPORTED = 1, 2, 3, 4
ERR_CUDA, ERR_TIMEOUT, ERR_OOM, ERR_UNBOUND = 5, 6, 7, 8


class LlgbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"llgb status {status}: {message}")
        self.status = status


class FieldDesc(ctypes.Structure):
    _fields_ = [("path", ctypes.c_char_p), ("type", ctypes.c_int32)]


class Extents(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("index_type", ctypes.c_int32),
                ("static_mask", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("ext", ctypes.c_uint64 * 4)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("kernel_mode", ctypes.c_int32), ("batch_kernel_mode", ctypes.c_int32),
                ("tile_records", ctypes.c_int32), ("items", ctypes.c_int32),
                ("generic_items", ctypes.c_int32), ("stream_items", ctypes.c_int32), ("tiles", ctypes.c_uint64)]


class MappingDesc(ctypes.Structure):
    pass


MappingDesc._fields_ = [
    ("kind", ctypes.c_int32), ("aos_packed", ctypes.c_int32),
    ("subarray_align", ctypes.c_uint64), ("lanes", ctypes.c_uint64),
    ("bits", ctypes.c_int32), ("exp_bits", ctypes.c_int32), ("man_bits", ctypes.c_int32),
    ("n_ct", ctypes.c_int32), ("ct_from", ctypes.c_int32 * MAX_CT),
    ("ct_to", ctypes.c_int32 * MAX_CT),
    ("field_bits", ctypes.POINTER(ctypes.c_int32)),
    ("field_exp", ctypes.POINTER(ctypes.c_int32)),
    ("field_man", ctypes.POINTER(ctypes.c_int32)),
    ("inner", ctypes.POINTER(MappingDesc)),
    ("split_mask", ctypes.c_uint64),
    ("inner2", ctypes.POINTER(MappingDesc)),
    ("bit_lanes", ctypes.c_uint64),
]


ENGINES = {"auto": 0, "value": 1, "gather": 2}
STAGING = {"tma": 0, "plain_store": 1, "plain_load": 2, "plain": 3}


class LaunchConfig(ctypes.Structure):
    _fields_ = [("tile_records", ctypes.c_int32), ("src_stages", ctypes.c_int32),
                ("dst_stages", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("staging", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k in
                ("tile_records", "src_stages", "dst_stages", "threads", "ctas_per_sm", "staging")}


EXPORTS = [
    "llgb_last_error", "llgb_version", "llgb_record_create", "llgb_record_destroy",
    "llgb_record_leaf_count", "llgb_record_size", "llgb_view_create", "llgb_view_destroy",
    "llgb_nbody_step_instrumented", "llgb_heatmap_counters", "llgb_nbody_update", "llgb_nbody_move",
    "llgb_view_blob_count", "llgb_view_blob_size", "llgb_view_record_count",
    "llgb_view_bind", "llgb_copy", "llgb_pack", "llgb_unpack", "llgb_copy_config",
    "llgb_copy_with", "llgb_nbody_step", "llgb_device_status",
    "llgb_batch_create", "llgb_batch_launch", "llgb_batch_info", "llgb_batch_destroy",
    "llgb_autotune", "llgb_autotune_clear", "llgb_batch_copy_noalloc", "llgb_copy_plan",
    "llgb_wait_selftest", "llgb_fma_probe", "llgb_autotune_save", "llgb_autotune_load", "llgb_batch_arena_create", "llgb_batch_arena_copy", "llgb_batch_arena_destroy",
]

_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "paper_2302_08251_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(path)
        p, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
        L.llgb_last_error.restype = ctypes.c_char_p
        L.llgb_version.restype = ctypes.c_char_p
        L.llgb_record_create.argtypes = [ctypes.POINTER(FieldDesc), i32, ctypes.POINTER(p)]
        L.llgb_record_destroy.argtypes = [p]
        L.llgb_record_leaf_count.argtypes = [p]
        L.llgb_record_size.argtypes = [p, i32, ctypes.POINTER(u64)]
        L.llgb_view_create.argtypes = [p, ctypes.POINTER(Extents), ctypes.POINTER(MappingDesc),
                                       ctypes.POINTER(p)]
        L.llgb_view_destroy.argtypes = [p]
        L.llgb_view_blob_count.argtypes = [p]
        L.llgb_view_blob_size.argtypes = [p, i32]
        L.llgb_view_blob_size.restype = u64
        L.llgb_view_record_count.argtypes = [p]
        L.llgb_view_record_count.restype = u64
        L.llgb_view_bind.argtypes = [p, ctypes.POINTER(p), i32]
        for name in ("llgb_copy", "llgb_pack", "llgb_unpack"):
            getattr(L, name).argtypes = [p, p, p]
        L.llgb_copy_config.argtypes = [p, p, ctypes.POINTER(LaunchConfig)]
        L.llgb_copy_plan.argtypes = [p, p, ctypes.POINTER(LaunchConfig), ctypes.POINTER(PlanInfo)]
        L.llgb_copy_with.argtypes = [p, p, ctypes.POINTER(LaunchConfig), p]
        L.llgb_nbody_step.argtypes = [p, ctypes.c_float, ctypes.c_float, p]
        L.llgb_nbody_step_instrumented.argtypes = [p, ctypes.c_float, ctypes.c_float, p, i32, p, u64, p]
        L.llgb_nbody_update.argtypes = [p, ctypes.c_float, ctypes.c_float, i32, p]
        L.llgb_nbody_move.argtypes = [p, ctypes.c_float, i32, p]
        L.llgb_heatmap_counters.argtypes = [p, u64, ctypes.POINTER(u64)]
        L.llgb_device_status.argtypes = [ctypes.POINTER(i32), i32]
        L.llgb_batch_create.argtypes = [i32, ctypes.POINTER(p), ctypes.POINTER(p), ctypes.POINTER(p)]
        L.llgb_batch_launch.argtypes = [p, p, i32]
        L.llgb_batch_info.argtypes = [p, ctypes.POINTER(i32), ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.llgb_batch_destroy.argtypes = [p]
        L.llgb_autotune.argtypes = [p, p, p, ctypes.POINTER(LaunchConfig)]
        L.llgb_batch_copy_noalloc.argtypes = [i32, ctypes.POINTER(p), ctypes.POINTER(p), p]
        L.llgb_wait_selftest.argtypes = [u64, p, p]
        L.llgb_autotune_save.argtypes = [ctypes.c_char_p]
        L.llgb_autotune_load.argtypes = [ctypes.c_char_p]
        L.llgb_fma_probe.argtypes = [ctypes.c_uint32, p, ctypes.POINTER(u64), p]
        L.llgb_batch_arena_create.argtypes = [i32, i32, ctypes.POINTER(p)]
        L.llgb_batch_arena_copy.argtypes = [p, i32, ctypes.POINTER(p), ctypes.POINTER(p), p]
        L.llgb_batch_arena_destroy.argtypes = [p]
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != OK:
        raise LlgbError(status, lib().llgb_last_error().decode())


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return ctypes.c_void_p(int(stream))


def mapping_desc(m: dict, keep: list) -> MappingDesc:
    """Build an llgb_mapping_desc from the plain-dict mapping description:
    {"kind": "aos", "packed": 0|1}, {"kind": "soa_sb", "subarray_align": a},
    {"kind": "soa_mb"}, {"kind": "aosoa", "lanes": L},
    {"kind": "bitpack_int", "bits": b, "field_bits": [...], "lanes": L},
    {"kind": "bitpack_float", "exp": E, "man": M, "field_exp": [...],
    "field_man": [...], "lanes": L} (bit-packed "lanes": 0 or absent = SoA
    streams, L = the AoSoA organisation), {"kind": "bytesplit", "inner": m},
    {"kind": "changetype", "ct": [(from, to), ...], "inner": m},
    {"kind": "null"}, {"kind": "split", "fields": [...], "inner": m,
    "rest": m}.  `keep` collects the ctypes objects the descriptor points to."""
    c = MappingDesc()
    c.kind = KIND_ID[m["kind"]]
    c.aos_packed = int(m.get("packed", 0))
    c.subarray_align = int(m.get("subarray_align", 0))
    c.lanes = int(m.get("lanes", 1))
    if m["kind"] in ("bitpack_int", "bitpack_float"):
        c.bit_lanes = int(m.get("lanes", 0))  # 0: SoA organisation
    c.bits = int(m.get("bits", 0))
    c.exp_bits = int(m.get("exp", 0))
    c.man_bits = int(m.get("man", 0))
    ct = m.get("ct", [])
    c.n_ct = len(ct)
    for k, (a, b) in enumerate(ct):
        c.ct_from[k] = TYPE_ID[a]
        c.ct_to[k] = TYPE_ID[b]
    for key in ("field_bits", "field_exp", "field_man"):
        if m.get(key) is not None:
            arr = (ctypes.c_int32 * len(m[key]))(*m[key])
            keep.append(arr)
            setattr(c, key, ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32)))
    if m.get("inner") is not None:
        inner = mapping_desc(m["inner"], keep)
        keep.append(inner)
        c.inner = ctypes.pointer(inner)
    if m["kind"] == "split":
        # {"kind": "split", "fields": [leaf indices -> "inner"], "rest": mapping of the others}
        c.split_mask = sum(1 << f for f in m["fields"])
        rest = mapping_desc(m["rest"], keep)
        keep.append(rest)
        c.inner2 = ctypes.pointer(rest)
    return c


def extents_desc(extents, index_type: str = "u64", static=None) -> Extents:
    if isinstance(extents, int):
        extents = (extents,)
    e = Extents()
    e.rank = len(extents)
    e.index_type = INDEX_TYPES[index_type]
    mask = 0
    for d, x in enumerate(extents):
        e.ext[d] = int(x)
        if static is not None and static[d]:
            mask |= 1 << d
    e.static_mask = mask
    return e


class Record:
    def __init__(self, leaves):
        self.leaves = [(str(p), str(t)) for p, t in leaves]
        arr = (FieldDesc * len(self.leaves))()
        self._paths = [p.encode() for p, _ in self.leaves]
        for k, (p, t) in enumerate(self.leaves):
            arr[k].path = self._paths[k]
            arr[k].type = TYPE_ID[t]
        h = ctypes.c_void_p()
        check(lib().llgb_record_create(arr, len(self.leaves), ctypes.byref(h)))
        self.handle = h

    @property
    def types(self):
        return [t for _, t in self.leaves]

    def size(self, packed: bool = False) -> int:
        out = ctypes.c_uint64()
        check(lib().llgb_record_size(self.handle, int(packed), ctypes.byref(out)))
        return out.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.llgb_record_destroy(self.handle)
            self.handle = None


def blob_sizes(record: Record, mapping: dict, extents, index_type: str = "u64") -> list:
    """Blob sizes a view of `record` under `mapping` would have (host planning
    only; nothing is allocated or bound)."""
    keep: list = []
    e = extents_desc(extents, index_type)
    m = mapping_desc(mapping, keep)
    h = ctypes.c_void_p()
    L = lib()
    check(L.llgb_view_create(record.handle, ctypes.byref(e), ctypes.byref(m), ctypes.byref(h)))
    try:
        return [int(L.llgb_view_blob_size(h, k)) for k in range(L.llgb_view_blob_count(h))]
    finally:
        L.llgb_view_destroy(h)


class View:
    """A view: mapping + blobs.  Blobs are torch uint8 tensors on the device
    (allocated here unless given) and are bound to the C view."""

    def __init__(self, record: Record, mapping: dict, extents, index_type: str = "u64",
                 static=None, blobs=None, device=None):
        self.record = record
        self.mapping = mapping
        self._keep: list = []
        self._ext = extents_desc(extents, index_type, static)
        self._map = mapping_desc(mapping, self._keep)
        h = ctypes.c_void_p()
        check(lib().llgb_view_create(record.handle, ctypes.byref(self._ext),
                                     ctypes.byref(self._map), ctypes.byref(h)))
        self.handle = h
        nb = lib().llgb_view_blob_count(h)
        self.blob_sizes = [int(lib().llgb_view_blob_size(h, k)) for k in range(nb)]
        self.n = int(lib().llgb_view_record_count(h))
        if blobs is None:
            import torch
            dev = device if device is not None else torch.device("cuda")
            blobs = [torch.empty(max(1, s), dtype=torch.uint8, device=dev) for s in self.blob_sizes]
        self.bind(blobs)

    def bind(self, blobs) -> None:
        if len(blobs) != len(self.blob_sizes):
            raise ValueError("wrong number of blobs")
        for b, s in zip(blobs, self.blob_sizes):
            if b.numel() * b.element_size() < s:
                raise ValueError("blob too small")
        self.blobs = list(blobs)
        ptrs = (ctypes.c_void_p * max(1, len(blobs)))(*[b.data_ptr() for b in blobs])
        check(lib().llgb_view_bind(self.handle, ptrs, len(blobs)))

    def blob_bytes(self):
        """Host copies (numpy uint8) of every blob, trimmed to the blob size."""
        return [b[:s].cpu().numpy() for b, s in zip(self.blobs, self.blob_sizes)]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.llgb_view_destroy(self.handle)
            self.handle = None


def llgb_copy(src: View, dst: View, stream=None) -> None:
    check(lib().llgb_copy(src.handle, dst.handle, _stream_ptr(stream)))


def llgb_pack(plain: View, packed: View, stream=None) -> None:
    check(lib().llgb_pack(plain.handle, packed.handle, _stream_ptr(stream)))


def llgb_unpack(packed: View, plain: View, stream=None) -> None:
    check(lib().llgb_unpack(packed.handle, plain.handle, _stream_ptr(stream)))


def launch_config(cfg: dict) -> LaunchConfig:
    """An llgb_launch_config from a dict; "engine" and "staging" may be names."""
    c = LaunchConfig()
    for k, v in cfg.items():
        if k == "engine" and isinstance(v, str):
            v = ENGINES[v]
        elif k == "staging" and isinstance(v, str):
            v = STAGING[v]
        setattr(c, k, int(v))
    return c


def llgb_copy_plan(src: View, dst: View, cfg: dict | None = None) -> dict:
    """Host-only plan of llgb_copy(src, dst) (and of the pair as a batch
    entry): kernel modes, tiling and item counts; nothing is launched."""
    return plan_info(src.handle, dst.handle, cfg)


def plan_info(src_handle, dst_handle, cfg: dict | None = None) -> dict:
    """llgb_copy_plan on raw view handles (bound or not)."""
    info = PlanInfo()
    c = launch_config(cfg) if cfg is not None else None
    check(lib().llgb_copy_plan(src_handle, dst_handle, ctypes.byref(c) if c is not None else None,
                               ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in PlanInfo._fields_}


def llgb_copy_config(src: View, dst: View) -> dict:
    c = LaunchConfig()
    check(lib().llgb_copy_config(src.handle, dst.handle, ctypes.byref(c)))
    return c.as_dict()


def llgb_copy_with(src: View, dst: View, cfg: dict, stream=None) -> None:
    """llgb_copy with an explicit launch shape; cfg may also hold
    "engine": "auto" | "value" | "gather"."""
    c = launch_config(cfg)
    check(lib().llgb_copy_with(src.handle, dst.handle, ctypes.byref(c), _stream_ptr(stream)))


def llgb_nbody_step(view: View, eps: float, dt: float, stream=None) -> None:
    check(lib().llgb_nbody_step(view.handle, float(eps), float(dt), _stream_ptr(stream)))


TRAVERSALS = {"index": 0, "blocks": 1}


def llgb_nbody_update(view: View, eps: float, dt: float, traversal="index", stream=None) -> None:
    """The update phase alone; traversal 'index' or 'blocks'."""
    check(lib().llgb_nbody_update(view.handle, float(eps), float(dt), TRAVERSALS[traversal], _stream_ptr(stream)))


def llgb_nbody_move(view: View, dt: float, traversal="index", stream=None) -> None:
    """The move phase alone; traversal 'index' or 'blocks'."""
    check(lib().llgb_nbody_move(view.handle, float(dt), TRAVERSALS[traversal], _stream_ptr(stream)))


COUNT_MODES = {"atomic": 1, "block": 2}


def llgb_heatmap_counters(view: View, granularity: int) -> int:
    out = ctypes.c_uint64()
    check(lib().llgb_heatmap_counters(view.handle, int(granularity), ctypes.byref(out)))
    return out.value


def llgb_nbody_step_instrumented(view: View, eps: float, dt: float, field_counts=None, count_mode="atomic",
                                 heat=None, granularity: int = 1, stream=None) -> None:
    """llgb_nbody_step counting its accesses: field_counts (14 uint64 device
    counters) and/or heat (llgb_heatmap_counters(view, granularity) uint64
    device counters), both incremented."""
    fc = ctypes.c_void_p(field_counts.data_ptr()) if field_counts is not None else None
    ht = ctypes.c_void_p(heat.data_ptr()) if heat is not None else None
    check(lib().llgb_nbody_step_instrumented(view.handle, float(eps), float(dt), fc, COUNT_MODES[count_mode],
                                             ht, int(granularity), _stream_ptr(stream)))


def llgb_wait_selftest(limit_ns: int, waited=None, stream=None) -> None:
    """Queue the bounded-wait self-test kernel (include/llgb.h); `waited`: an
    int64 device tensor of one element that receives the wait's length in ns."""
    w = ctypes.c_void_p(waited.data_ptr()) if waited is not None else None
    check(lib().llgb_wait_selftest(int(limit_ns), w, _stream_ptr(stream)))


def llgb_fma_probe(iters: int, sink, stream=None) -> int:
    """Queue the FP32 FMA throughput probe; returns the FMAs it performs.
    `sink`: a float32 device tensor of at least one element."""
    fmas = ctypes.c_uint64()
    check(lib().llgb_fma_probe(int(iters), ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fmas), _stream_ptr(stream)))
    return fmas.value


def llgb_device_status(reset: bool = False) -> int:
    code = ctypes.c_int32()
    check(lib().llgb_device_status(ctypes.byref(code), int(reset)))
    return code.value


class Batch:
    """Many copies (src[k] -> dst[k]) planned once and launched together."""

    def __init__(self, pairs):
        self.pairs = list(pairs)  # keeps the views (and their blobs) alive
        n = len(self.pairs)
        srcs = (ctypes.c_void_p * max(1, n))(*[s.handle for s, _ in self.pairs])
        dsts = (ctypes.c_void_p * max(1, n))(*[d.handle for _, d in self.pairs])
        h = ctypes.c_void_p()
        check(lib().llgb_batch_create(n, srcs, dsts, ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None, use_graph: bool = False) -> None:
        check(lib().llgb_batch_launch(self.handle, _stream_ptr(stream), int(use_graph)))

    def info(self) -> dict:
        launches, tiles, nbytes = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().llgb_batch_info(self.handle, ctypes.byref(launches), ctypes.byref(tiles),
                                    ctypes.byref(nbytes)))
        return {"launches": launches.value, "tiles": tiles.value, "bytes": nbytes.value}

    def close(self) -> None:
        if getattr(self, "handle", None) and _lib is not None:
            _lib.llgb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


class Arena:
    """Descriptor tables for `slots` batched copies of up to `max_pairs` pairs,
    allocated once; copy() queues one batched copy without allocating."""

    def __init__(self, max_pairs: int = 256, slots: int = 8):
        h = ctypes.c_void_p()
        check(lib().llgb_batch_arena_create(int(max_pairs), int(slots), ctypes.byref(h)))
        self.handle = h
        self.max_pairs = int(max_pairs)

    def copy(self, pairs, stream=None) -> None:
        pairs = list(pairs)
        n = len(pairs)
        srcs = (ctypes.c_void_p * max(1, n))(*[s.handle for s, _ in pairs])
        dsts = (ctypes.c_void_p * max(1, n))(*[d.handle for _, d in pairs])
        check(lib().llgb_batch_arena_copy(self.handle, n, srcs, dsts, _stream_ptr(stream)))

    def close(self) -> None:
        if getattr(self, "handle", None) and _lib is not None:
            _lib.llgb_batch_arena_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def llgb_batch_create(pairs) -> Batch:
    return Batch(pairs)


def llgb_batch_launch(batch: Batch, stream=None, use_graph: bool = False) -> None:
    batch.launch(stream, use_graph)


def llgb_autotune(src: View, dst: View, stream=None) -> dict:
    c = LaunchConfig()
    check(lib().llgb_autotune(src.handle, dst.handle, _stream_ptr(stream), ctypes.byref(c)))
    return c.as_dict()


def llgb_batch_copy_noalloc(pairs, stream=None) -> None:
    """Copy every (src, dst) pair without allocating device memory (at most
    64 pairs; the descriptor tables live in the library's static device
    array, shared by every call on a device -- see include/llgb.h)."""
    pairs = list(pairs)
    n = len(pairs)
    srcs = (ctypes.c_void_p * max(1, n))(*[s.handle for s, _ in pairs])
    dsts = (ctypes.c_void_p * max(1, n))(*[d.handle for _, d in pairs])
    check(lib().llgb_batch_copy_noalloc(n, srcs, dsts, _stream_ptr(stream)))


def llgb_autotune_clear() -> None:
    check(lib().llgb_autotune_clear())


def llgb_autotune_save(path: str) -> None:
    check(lib().llgb_autotune_save(os.fsencode(path)))


def llgb_autotune_load(path: str) -> None:
    check(lib().llgb_autotune_load(os.fsencode(path)))


copy = llgb_copy
pack = llgb_pack
unpack = llgb_unpack
nbody_step = llgb_nbody_step
device_status = llgb_device_status
