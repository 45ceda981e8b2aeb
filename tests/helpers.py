"""Helpers shared by the tests: field arrays <-> oracle views."""
import numpy as np

import oracle

UINT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


def bits_of(arr: np.ndarray) -> np.ndarray:
    """Little-endian bit patterns of a leaf array, zero-extended to uint64."""
    arr = np.ascontiguousarray(arr)
    return arr.view(UINT[arr.dtype.itemsize]).astype(np.uint64)


def oracle_view(record, mapping, fields=None, n=None):
    """Oracle view holding `fields` (stored through the oracle's own store)."""
    if n is None:
        n = len(fields[0])
    v = oracle.OracleView(record, mapping, n)
    if fields is not None:
        for f, arr in enumerate(fields):
            v.set_field_values(f, bits_of(arr))
    return v


AFFINE = [
    {"kind": "aos", "packed": 0},
    {"kind": "aos", "packed": 1},
    {"kind": "soa_mb"},
    {"kind": "soa_sb"},
    {"kind": "soa_sb", "subarray_align": 64},
    {"kind": "aosoa", "lanes": 8},
    {"kind": "aosoa", "lanes": 32},
    {"kind": "aosoa", "lanes": 3},
]
