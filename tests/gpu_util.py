"""Helpers for the GPU parity tests: move views between the oracle (host)
and the CUDA library (device) and compare every byte."""
import numpy as np
import torch

import oracle
from paper_2302_08251_gb300 import build, llgb

_built = False


def ensure_library():
    global _built
    if not _built:
        build.build()
        _built = True
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    return llgb.lib()


def device_view_of(ov: oracle.OracleView, index_type="u64"):
    """A device view with the oracle view's record, mapping and bytes."""
    rec = llgb.Record(ov.record)
    v = llgb.View(rec, ov.mapping, (ov.n,), index_type=index_type)
    for b, host in zip(v.blobs, ov.blobs):
        if host.size:
            b[:host.size].copy_(torch.from_numpy(host))
    return v


def empty_device_view(record, mapping, n, fill=0xAB, index_type="u64", extents=None, static=None):
    rec = llgb.Record(record)
    v = llgb.View(rec, mapping, extents if extents is not None else (n,), index_type=index_type,
                  static=static)
    for b in v.blobs:
        b.fill_(fill)
    return v


def assert_same_bytes(dev_view, ov: oracle.OracleView, what=""):
    got = dev_view.blob_bytes()
    assert len(got) == len(ov.blobs)
    for k, (g, e) in enumerate(zip(got, ov.blobs)):
        if not np.array_equal(g, e):
            bad = np.flatnonzero(g != e)
            raise AssertionError(f"{what}: blob {k} differs at {bad.size} bytes, first at {bad[:8]} "
                                 f"(got {g[bad[:8]]}, want {e[bad[:8]]})")


def sync_and_check_status():
    torch.cuda.synchronize()
    assert llgb.llgb_device_status(reset=True) == 0
