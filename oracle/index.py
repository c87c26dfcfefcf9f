"""uvw -> grid index selection, FP64 (bit-exact reference).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For each visibility (row r, channel c) with uvw in metres and frequency f:

* s_c = f / c0                               (one factor per channel, 1/lambda)
* u_lambda = u * s_c                         (wavelengths)
* x = u_lambda * L + N/2                     (pixel coordinate; the uv origin
                                              sits on pixel N/2, Section 2.1.2)
* q = floor(beta * x + 0.5)                  (nearest point of the
                                              beta-oversampled grid, ties up)
* k = floor((q + beta/2) / beta), o = q - k beta, o in [-beta/2, beta/2)
* the same for v; the record sits at pixel k + o / beta.
* w-plane (P > 1): the plane nearest in sqrt(|w|), ties up, as a count of
  thresholds: T_j = ((j - 1/2) / (P - 1))^2 * w_max, j = 1 .. P - 1 (each
  step rounded), p = #{j : T_j <= |w_lambda|} (so p <= P - 1 and records
  beyond w_max use the outermost plane); w_lambda must be finite;
  conj = (w_lambda < 0).  P = 1 ignores w.
* valid (Bounded Records Assumption, Section 2.3.1): every tap of the
  plane's S_p x S_p footprint lands inside [0, N); also q finite and
  |q| < 2^30.

Each line is one IEEE-754 double operation in the order written (numpy
evaluates each ufunc separately, so nothing is fused); the CUDA path must
execute the same sequence.  Parity: pinned by hand-computed ties and edges
in tests/test_oracle_index.py.
"""
from __future__ import annotations

import numpy as np

from .wkernel import C0, Params, plane_support

Q_LIMIT = float(2 ** 30)

FLAG_VALID = 1
FLAG_CONJ = 2


def chan_scale(freq: np.ndarray) -> np.ndarray:
    """s_c = f / c0 per channel (wavelengths per metre)."""
    return np.asarray(freq, dtype=np.float64) / C0


def plane_thresholds(prm: Params) -> np.ndarray:
    """T_j = ((j - 1/2) / (P - 1))^2 w_max, j = 1 .. P - 1: |w| at which the
    nearest plane in sqrt(|w|) steps from j - 1 to j."""
    P = prm.n_wplanes
    t = (np.arange(1, P, dtype=np.float64) - 0.5) / float(P - 1)
    return (t * t) * float(prm.w_max_lambda)


def _axis(coord_m: np.ndarray, freq: np.ndarray, prm: Params):
    L = float(prm.grid_n) * float(prm.cell_rad)
    lam = coord_m[:, None] * chan_scale(freq)[None, :]
    x = lam * L + float(prm.grid_n // 2)
    q = np.floor(float(prm.oversample) * x + 0.5)
    ok = np.isfinite(q) & (np.abs(q) < Q_LIMIT)
    qi = np.where(ok, q, 0.0).astype(np.int64)
    b = int(prm.oversample)
    k = np.floor_divide(qi + b // 2, b)
    o = qi - k * b
    return k, o, ok


def index_vis(uvw_m: np.ndarray, freq_hz: np.ndarray, prm: Params) -> dict:
    """Index records for all nrow * nchan visibilities, flattened (row, chan)."""
    uvw_m = np.ascontiguousarray(uvw_m, dtype=np.float64)
    freq_hz = np.ascontiguousarray(freq_hz, dtype=np.float64)
    ku, ou, oku = _axis(uvw_m[:, 0], freq_hz, prm)
    kv, ov, okv = _axis(uvw_m[:, 1], freq_hz, prm)
    P = prm.n_wplanes
    shape = ku.shape
    if P == 1:
        plane = np.zeros(shape, dtype=np.int64)
        conj = np.zeros(shape, dtype=bool)
        okw = np.ones(shape, dtype=bool)
    else:
        wl = uvw_m[:, 2][:, None] * chan_scale(freq_hz)[None, :]
        okw = np.isfinite(wl)
        cnt = np.searchsorted(plane_thresholds(prm), np.abs(np.where(okw, wl, 0.0)),
                              side="right")
        plane = np.where(okw, cnt, 0).astype(np.int64)
        conj = wl < 0.0
    S = plane_support(prm)[plane]
    h = (S - 1) // 2
    N = prm.grid_n
    inside = (ku - h >= 0) & (ku + h <= N - 1) & (kv - h >= 0) & (kv + h <= N - 1)
    valid = oku & okv & okw & inside
    flags = valid.astype(np.int64) * FLAG_VALID + (conj & valid).astype(np.int64) * FLAG_CONJ
    out = dict(ku=ku, kv=kv, ou=ou, ov=ov, plane=plane, valid=valid, conj=conj & valid,
               flags=flags)
    # invalid records carry zeros, so that integer comparison is well defined
    for key in ("ku", "kv", "ou", "ov", "plane"):
        out[key] = np.where(valid, out[key], 0).reshape(-1)
    for key in ("valid", "conj", "flags"):
        out[key] = out[key].reshape(-1)
    return out
