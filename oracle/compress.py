"""Full compression of visibility records (Section 3.3.5, "Full Compression").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Records that fall on the same pixel of the virtual nearest-neighbour grid
are added before gridding.  With an oversampled w-projection GCF the record's
kernel is fixed by its oversampled position (k, o), its w-plane and the sign
of w, so records sharing all of (k_u, k_v, o_u, o_v, plane, sign of w) are
merged: their weighted visibilities are summed into one record.  Gridding is
linear, so gridding the compressed records reproduces gridding the originals.
"""
from __future__ import annotations

import numpy as np

from .index import FLAG_CONJ


def record_keys(idx: dict) -> np.ndarray:
    """[n, 6] int64 keys (ku, kv, ou, ov, plane, conj) of every record."""
    conj = ((idx["flags"] & FLAG_CONJ) != 0).astype(np.int64)
    return np.stack([idx["ku"], idx["kv"], idx["ou"], idx["ov"], idx["plane"], conj], 1)


def full_compression(idx: dict, vis, weight=None):
    """(compressed index dict, compressed visibilities [m, npol] complex128).

    Only valid records take part; the output records are all valid and sorted
    by key (ku, kv, ou, ov, plane, conj)."""
    valid = idx["valid"]
    n = valid.shape[0]
    v = np.asarray(vis, dtype=np.complex128).reshape(n, -1)
    if weight is not None:
        v = v * np.asarray(weight, dtype=np.float64).reshape(n, -1)
    keys = record_keys(idx)[valid]
    uk, inv = np.unique(keys, axis=0, return_inverse=True)
    out = np.zeros((uk.shape[0], v.shape[1]), dtype=np.complex128)
    np.add.at(out, inv.reshape(-1), v[valid])
    conj = uk[:, 5].astype(bool)
    cidx = {"ku": uk[:, 0], "kv": uk[:, 1], "ou": uk[:, 2], "ov": uk[:, 3], "plane": uk[:, 4],
            "valid": np.ones(uk.shape[0], dtype=bool),
            "conj": conj,
            "flags": (1 | (conj.astype(np.int64) << 1)).astype(np.int64)}
    return cidx, out
