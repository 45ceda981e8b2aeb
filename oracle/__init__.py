"""Plain CPU oracle for mapping-driven record layouts (arXiv 2302.08251).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers; the product package
never imports this module.  The C source (``llgb_oracle.c``) shares no code with
the CUDA library.

Records, mappings and views are described with plain data so that the same
description can be handed to the oracle and to the library under test:

* a record is a list of ``(path, type)`` pairs, type one of ``TYPES``;
* a mapping is a dict, e.g. ``{"kind": "aos", "packed": 0}``,
  ``{"kind": "aosoa", "lanes": 32}``, ``{"kind": "bitpack_int", "bits": 12}``,
  ``{"kind": "bitpack_float", "exp": 8, "man": 23}``,
  ``{"kind": "bytesplit", "inner": {...}}``,
  ``{"kind": "changetype", "ct": [("f64", "f32")], "inner": {...}}``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "llgb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")

TYPES = ["u8", "u16", "u32", "u64", "i8", "i16", "i32", "i64",
         "f16", "bf16", "f32", "f64"]
TYPE_ID = {t: k for k, t in enumerate(TYPES)}
TYPE_SIZE = {"u8": 1, "u16": 2, "u32": 4, "u64": 8, "i8": 1, "i16": 2,
             "i32": 4, "i64": 8, "f16": 2, "bf16": 2, "f32": 4, "f64": 8}
KINDS = ["aos", "soa_sb", "soa_mb", "aosoa", "bitpack_int", "bitpack_float",
         "bytesplit", "changetype", "null", "split"]
KIND_ID = {k: n for n, k in enumerate(KINDS)}
MAX_CT = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liborc.so``."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp,
                           _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Mapping(ctypes.Structure):
    pass


_Mapping._fields_ = [
    ("kind", ctypes.c_int32),
    ("aos_packed", ctypes.c_int32),
    ("subarray_align", ctypes.c_uint64),
    ("lanes", ctypes.c_uint64),
    ("bits", ctypes.c_int32),
    ("exp_bits", ctypes.c_int32),
    ("man_bits", ctypes.c_int32),
    ("n_ct", ctypes.c_int32),
    ("ct_from", ctypes.c_int32 * MAX_CT),
    ("ct_to", ctypes.c_int32 * MAX_CT),
    ("field_bits", ctypes.POINTER(ctypes.c_int32)),
    ("field_exp", ctypes.POINTER(ctypes.c_int32)),
    ("field_man", ctypes.POINTER(ctypes.c_int32)),
    ("inner", ctypes.POINTER(_Mapping)),
    ("split_mask", ctypes.c_uint64),
    ("inner2", ctypes.POINTER(_Mapping)),
    ("bit_lanes", ctypes.c_uint64),
]

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i32, p = ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p
        P32 = ctypes.POINTER(ctypes.c_int32)
        PM = ctypes.POINTER(_Mapping)
        PB = ctypes.POINTER(ctypes.c_void_p)
        lib.orc_type_size.argtypes = [i32]
        lib.orc_check.argtypes = [P32, i32, PM]
        lib.orc_blob_count.argtypes = [P32, i32, PM]
        lib.orc_blob_count.restype = i32
        lib.orc_blob_size.argtypes = [P32, i32, PM, u64, i32]
        lib.orc_blob_size.restype = u64
        lib.orc_load.argtypes = [P32, i32, PM, u64, PB, u64, i32]
        lib.orc_load.restype = u64
        lib.orc_store.argtypes = [P32, i32, PM, u64, PB, u64, i32, u64]
        lib.orc_copy.argtypes = [P32, i32, u64, PM, PB, PM, PB]
        lib.orc_copy_range.argtypes = [P32, i32, u64, PM, PB, PM, PB, u64, u64]
        lib.orc_convert.argtypes = [u64, i32, i32, i32, i32]
        lib.orc_convert.restype = u64
        lib.orc_load_field.argtypes = [P32, i32, PM, u64, PB, i32, u64, u64, p]
        lib.orc_store_field.argtypes = [P32, i32, PM, u64, PB, i32, u64, u64, p]
        lib.orc_convert_n.argtypes = [p, p, u64, i32, i32, i32, i32]
        lib.orc_nbody_step.argtypes = [PM, u64, PB, ctypes.c_double,
                                       ctypes.c_double, u64, u64, p, p]
        lib.orc_nbody_move.argtypes = [PM, u64, PB, ctypes.c_double, u64, u64, p]
        lib.orc_nbody_access_counts.argtypes = [u64, u64, p]
        lib.orc_nbody_heatmap.argtypes = [PM, u64, u64, u64, p]
        _lib = lib
    return _lib


def _to_c_mapping(m: dict, keep: list) -> _Mapping:
    c = _Mapping()
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
    for key, attr in (("field_bits", "field_bits"), ("field_exp", "field_exp"),
                      ("field_man", "field_man")):
        if m.get(key) is not None:
            arr = (ctypes.c_int32 * len(m[key]))(*m[key])
            keep.append(arr)
            setattr(c, attr, ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32)))
    if m.get("inner") is not None:
        inner = _to_c_mapping(m["inner"], keep)
        keep.append(inner)
        c.inner = ctypes.pointer(inner)
    if m["kind"] == "split":
        # {"kind": "split", "fields": [leaf indices -> "inner"], "rest": mapping of the others}
        c.split_mask = sum(1 << f for f in m["fields"])
        rest = _to_c_mapping(m["rest"], keep)
        keep.append(rest)
        c.inner2 = ctypes.pointer(rest)
    return c


class OracleView:
    """Host blobs of n records under one mapping, driven by the oracle."""

    def __init__(self, record, mapping: dict, n: int, blobs=None):
        self._lib = _load()
        self.record = list(record)
        self.types = [t for _, t in self.record]
        self.mapping = mapping
        self.n = int(n)
        self._keep: list = []
        self._types_c = (ctypes.c_int32 * len(self.types))(
            *[TYPE_ID[t] for t in self.types])
        self._map_c = _to_c_mapping(mapping, self._keep)
        rc = self._lib.orc_check(self._types_c, len(self.types),
                                 ctypes.byref(self._map_c))
        if rc != 0:
            raise ValueError(f"oracle rejects mapping {mapping} (code {rc})")
        nb = self._lib.orc_blob_count(self._types_c, len(self.types),
                                      ctypes.byref(self._map_c))
        sizes = [int(self._lib.orc_blob_size(self._types_c, len(self.types),
                                             ctypes.byref(self._map_c), self.n, k))
                 for k in range(nb)]
        self.blob_sizes = sizes
        if blobs is None:
            self.blobs = [np.zeros(s, dtype=np.uint8) for s in sizes]
        else:
            blobs = [np.ascontiguousarray(b, dtype=np.uint8) for b in blobs]
            if [b.size for b in blobs] != sizes:
                raise ValueError(f"blob sizes {[b.size for b in blobs]} != {sizes}")
            self.blobs = blobs
        self._refresh_ptrs()

    def _refresh_ptrs(self):
        self._ptrs = (ctypes.c_void_p * max(1, len(self.blobs)))(
            *[b.ctypes.data for b in self.blobs])

    @property
    def nfields(self) -> int:
        return len(self.types)

    def load(self, i: int, f: int) -> int:
        return int(self._lib.orc_load(self._types_c, self.nfields,
                                      ctypes.byref(self._map_c), self.n,
                                      self._ptrs, i, f))

    def store(self, i: int, f: int, v: int) -> None:
        self._lib.orc_store(self._types_c, self.nfields, ctypes.byref(self._map_c),
                            self.n, self._ptrs, i, f, int(v) & (2**64 - 1))

    def copy_to(self, dst: "OracleView", i0: int | None = None,
                i1: int | None = None) -> None:
        if dst.types != self.types or dst.n != self.n:
            raise ValueError("copy needs the same record and the same n")
        if i0 is None:
            self._lib.orc_copy(self._types_c, self.nfields, self.n,
                               ctypes.byref(self._map_c), self._ptrs,
                               ctypes.byref(dst._map_c), dst._ptrs)
        else:
            self._lib.orc_copy_range(self._types_c, self.nfields, self.n,
                                     ctypes.byref(self._map_c), self._ptrs,
                                     ctypes.byref(dst._map_c), dst._ptrs, i0, i1)

    def field_values(self, f: int, i0: int = 0, i1: int | None = None) -> np.ndarray:
        """Logical bit patterns of leaf f for records [i0, i1) (uint64)."""
        if i1 is None:
            i1 = self.n
        out = np.zeros(max(0, i1 - i0), dtype=np.uint64)
        if out.size:
            self._lib.orc_load_field(self._types_c, self.nfields,
                                     ctypes.byref(self._map_c), self.n, self._ptrs,
                                     f, i0, i1, out.ctypes.data)
        return out

    def set_field_values(self, f: int, values, i0: int = 0) -> None:
        """Store logical bit patterns (uint64) into leaf f of records i0.."""
        vals = np.ascontiguousarray(values, dtype=np.uint64)
        if vals.size:
            self._lib.orc_store_field(self._types_c, self.nfields,
                                      ctypes.byref(self._map_c), self.n, self._ptrs,
                                      f, i0, i0 + vals.size, vals.ctypes.data)

    def nbody_step(self, eps: float, dt: float, i0: int = 0, i1: int | None = None):
        """FP64 n-body step; returns (pos, vel) arrays of shape (i1-i0, 3)."""
        if self.types != ["f32"] * 7:
            raise ValueError("n-body needs the 7-leaf f32 particle record")
        if i1 is None:
            i1 = self.n
        pos = np.zeros((i1 - i0, 3), dtype=np.float64)
        vel = np.zeros((i1 - i0, 3), dtype=np.float64)
        self._lib.orc_nbody_step(ctypes.byref(self._map_c), self.n, self._ptrs,
                                 float(eps), float(dt), i0, i1,
                                 pos.ctypes.data, vel.ctypes.data)
        return pos, vel

    def nbody_move(self, dt: float, i0: int = 0, i1: int | None = None):
        """FP64 move phase alone (p + dt v); returns pos of shape (i1-i0, 3)."""
        if self.types != ["f32"] * 7:
            raise ValueError("n-body needs the 7-leaf f32 particle record")
        if i1 is None:
            i1 = self.n
        pos = np.zeros((i1 - i0, 3), dtype=np.float64)
        self._lib.orc_nbody_move(ctypes.byref(self._map_c), self.n, self._ptrs, float(dt), i0, i1,
                                 pos.ctypes.data)
        return pos


def nbody_access_counts(n: int, block: int = 64) -> np.ndarray:
    """FieldAccessCount of one tiled n-body step (Sec. 4): 7 read counters,
    then 7 write counters, for the particle record."""
    out = np.zeros(14, dtype=np.uint64)
    _load().orc_nbody_access_counts(n, block, out.ctypes.data)
    return out


def nbody_heatmap(mapping: dict, n: int, g: int, block: int = 64) -> np.ndarray:
    """Heatmap of one tiled n-body step at granularity g bytes (Sec. 4):
    per-granule access counts, blob after blob."""
    particle = [(f"leaf{k}", "f32") for k in range(7)]
    keep: list = []
    m = _to_c_mapping(mapping, keep)
    total = sum((s + g - 1) // g for s in blob_sizes(particle, mapping, n))
    out = np.zeros(max(1, total), dtype=np.uint64)
    _load().orc_nbody_heatmap(ctypes.byref(m), n, block, g, out.ctypes.data)
    return out[:total]


def blob_sizes(record, mapping: dict, n: int) -> list:
    """Blob sizes of n records under `mapping`, without allocating them."""
    lib = _load()
    keep: list = []
    types = (ctypes.c_int32 * len(record))(*[TYPE_ID[t] for _, t in record])
    m = _to_c_mapping(mapping, keep)
    nb = lib.orc_blob_count(types, len(record), ctypes.byref(m))
    return [int(lib.orc_blob_size(types, len(record), ctypes.byref(m), int(n), k))
            for k in range(nb)]


def copy(src: OracleView, dst: OracleView) -> None:
    src.copy_to(dst)


def convert(bits: int, src_e: int, src_m: int, dst_e: int, dst_m: int) -> int:
    """RNE conversion of one bit pattern between (E, M) binary formats."""
    return int(_load().orc_convert(int(bits) & (2**64 - 1), src_e, src_m, dst_e, dst_m))


def convert_array(bits, src_e: int, src_m: int, dst_e: int, dst_m: int) -> np.ndarray:
    """Element-wise ``convert`` over a uint64 array."""
    inp = np.ascontiguousarray(bits, dtype=np.uint64)
    out = np.zeros_like(inp)
    if inp.size:
        _load().orc_convert_n(inp.ctypes.data, out.ctypes.data, inp.size,
                              src_e, src_m, dst_e, dst_m)
    return out


def type_size(t: str) -> int:
    return int(_load().orc_type_size(TYPE_ID[t]))
