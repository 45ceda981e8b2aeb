"""Helpers for the GPU parity tests: move views between the oracle (host)
and the CUDA library (device) and compare every byte."""
import numpy as np
import torch

import oracle
from paper_2302_08251_gb300 import build, llgb, synth

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


# ---- sampled windows of large copies ----
#
# Records [a, a + w) with a a multiple of 256 occupy, in every blob of every
# AoS, SoA, AoSoA (lanes dividing 256), bit-packed SoA or Bytesplit-over-SoA
# mapping, the byte range [size(a), size(a + w)), size(m) being the blob size
# of m records -- itself taken from the oracle.  Each window of the source is
# handed to the oracle as a view of w records and its copy compared with the
# same window of the GPU result, byte for byte.

W = 4096


def windows(n, seed, count=4):
    if n <= W:
        return [0]
    g = synth.rng(seed)
    starts = {0, (n - W) // 256 * 256}
    starts.update(int(x) // 256 * 256 for x in g.integers(0, n - W, count))
    return sorted(starts)


def window_of(view, record, mapping, a, w):
    lo = oracle.blob_sizes(record, mapping, a)
    hi = oracle.blob_sizes(record, mapping, a + w)
    return [b[x:y].cpu().numpy() for b, x, y in zip(view.blobs, lo, hi)]


def check_windows(src, dst, record, src_map, dst_map, n, seed):
    for a in windows(n, seed):
        w = min(W, n - a)
        src_o = oracle.OracleView(record, src_map, w, blobs=window_of(src, record, src_map, a, w))
        dst_o = oracle.OracleView(record, dst_map, w)
        src_o.copy_to(dst_o)
        got = window_of(dst, record, dst_map, a, w)
        for k, (g, e) in enumerate(zip(got, dst_o.blobs)):
            assert np.array_equal(g, e), (src_map, dst_map, a, k)
