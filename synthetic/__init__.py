"""Seeded synthetic interferometer observations.

This module builds the inputs that both the CUDA path and the CPU oracle
consume: antenna layouts, baseline uvw tracks (metres), channel
frequencies, complex visibilities and the imaging parameters that go with
them.  It holds none of the gridding arithmetic (no index selection, no
kernels, no accumulation); it only manufactures observations.

The observations stand in for the LOFAR / GMRT / VLA measurement sets the
thesis uses (Section 3.5.2, "Input and Simulation Parameters"), which are
not available here.  Array geometry follows the usual Earth-rotation
synthesis model: antennas in a local East-North-Up frame, baselines rotated
to (u, v, w) for a source at declination ``dec`` observed from latitude
``lat`` over evenly spaced hour angles (Thompson, Moran & Swenson,
Interferometry and Synthesis in Radio Astronomy, eq. 4.1).

Rows are ordered time-major (all baselines of time step 0, then time step
1, ...), as a measurement set stores them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

C0 = 299_792_458.0  # speed of light, m/s
BASE_SEED = 20211104


@dataclasses.dataclass
class Observation:
    """One synthetic observation plus the imaging parameters derived from it."""

    name: str
    uvw_m: np.ndarray          # float64 [nrow, 3], metres
    freq_hz: np.ndarray        # float64 [nchan]
    vis: np.ndarray            # complex64 [nrow, nchan, npol]
    grid_n: int
    cell_rad: float
    support_min: int
    support_max: int
    oversample: int
    n_wplanes: int
    w_max_lambda: float
    npol: int
    weight: Optional[np.ndarray] = None  # float32 [nrow, nchan, npol] or None

    @property
    def nrow(self) -> int:
        return int(self.uvw_m.shape[0])

    @property
    def nchan(self) -> int:
        return int(self.freq_hz.shape[0])

    @property
    def nvis(self) -> int:
        return self.nrow * self.nchan

    def plan_kwargs(self) -> dict:
        return dict(grid_n=self.grid_n, cell_rad=self.cell_rad,
                    support_min=self.support_min, support_max=self.support_max,
                    oversample=self.oversample, n_wplanes=self.n_wplanes,
                    w_max_lambda=self.w_max_lambda, npol=self.npol)


# --------------------------------------------------------------------------
# array layouts (local East-North-Up, metres)
# --------------------------------------------------------------------------

def antennas_disk(n_ant: int, diameter_m: float, rng: np.random.Generator) -> np.ndarray:
    """Antennas uniformly distributed over a disk of the given diameter."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    enu = np.zeros((n_ant, 3))
    enu[:, 0] = r * np.cos(th)
    enu[:, 1] = r * np.sin(th)
    return enu


def antennas_spiral_core(n_ant: int, extent_m: float, rng: np.random.Generator,
                         core_frac: float = 0.5, arms: int = 3) -> np.ndarray:
    """A dense Gaussian core plus logarithmic-spiral arms out to extent/2."""
    n_core = int(round(core_frac * n_ant))
    n_arm = n_ant - n_core
    enu = np.zeros((n_ant, 3))
    core_sigma = 0.015 * extent_m
    enu[:n_core, :2] = rng.normal(0.0, core_sigma, size=(n_core, 2))
    r_min = 0.04 * extent_m
    r_max = 0.5 * extent_m
    k = np.arange(n_arm)
    frac = (k // arms) / max(1, (n_arm + arms - 1) // arms - 1)
    r = r_min * (r_max / r_min) ** frac
    th = 2.0 * np.pi * (k % arms) / arms + 1.2 * np.log(r / r_min)
    r = r * (1.0 + 0.03 * rng.normal(size=n_arm))
    enu[n_core:, 0] = r * np.cos(th)
    enu[n_core:, 1] = r * np.sin(th)
    return enu


def baselines(enu: np.ndarray) -> np.ndarray:
    """All antenna pairs i < j as ENU difference vectors [nbl, 3]."""
    i, j = np.triu_indices(enu.shape[0], k=1)
    return enu[j] - enu[i]


def uvw_tracks(bl_enu: np.ndarray, n_times: int, dec_deg: float = -30.0,
               lat_deg: float = -30.0, ha_half_span_h: float = 4.0) -> np.ndarray:
    """Earth-rotation uvw tracks (metres), rows ordered (time, baseline).

    Hour angles are evenly spaced in [-span, +span).
    """
    lat = math.radians(lat_deg)
    dec = math.radians(dec_deg)
    e, n, up = bl_enu[:, 0], bl_enu[:, 1], bl_enu[:, 2]
    # local ENU -> equatorial (X towards H=0 meridian, Y east, Z north pole)
    X = -n * math.sin(lat) + up * math.cos(lat)
    Y = e
    Z = n * math.cos(lat) + up * math.sin(lat)
    span = ha_half_span_h * math.pi / 12.0
    ha = -span + 2.0 * span * np.arange(n_times) / n_times
    sH = np.sin(ha)[:, None]
    cH = np.cos(ha)[:, None]
    u = sH * X + cH * Y
    v = -math.sin(dec) * cH * X + math.sin(dec) * sH * Y + math.cos(dec) * Z
    w = math.cos(dec) * cH * X - math.cos(dec) * sH * Y + math.sin(dec) * Z
    return np.stack([u.reshape(-1), v.reshape(-1), w.reshape(-1)], axis=1)


def cn_vis(nrow: int, nchan: int, npol: int, rng: np.random.Generator) -> np.ndarray:
    """Circular complex normal CN(0, 1) visibilities, complex64."""
    shape = (nrow, nchan, npol)
    re = rng.standard_normal(shape, dtype=np.float32)
    im = rng.standard_normal(shape, dtype=np.float32)
    out = np.empty(shape, dtype=np.complex64)
    out.real = re * np.float32(math.sqrt(0.5))
    out.imag = im * np.float32(math.sqrt(0.5))
    return out


def fit_cell(uvw_m: np.ndarray, freq_hz: np.ndarray, grid_n: int, support_max: int,
             fill: float = 0.45) -> float:
    """Cell size that puts the longest |u|,|v| at fill*N - S_max/2 pixels from the centre."""
    f_max = float(np.max(freq_hz))
    uv_max = float(np.max(np.abs(uvw_m[:, :2]))) * f_max / C0
    field = (fill * grid_n - 0.5 * support_max) / uv_max
    return field / grid_n


def w_extent(uvw_m: np.ndarray, freq_hz: np.ndarray) -> float:
    return float(np.max(np.abs(uvw_m[:, 2]))) * float(np.max(freq_hz)) / C0


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

def _observation(name, enu, n_times, freq, npol, grid_n, s_min, s_max, beta, n_w,
                 rng, row_subsample=None, dec_deg=-30.0, lat_deg=-30.0, with_vis=True):
    uvw = uvw_tracks(baselines(enu), n_times, dec_deg=dec_deg, lat_deg=lat_deg)
    cell = fit_cell(uvw, freq, grid_n, s_max)
    wmax = w_extent(uvw, freq) if n_w > 1 else 0.0
    if row_subsample is not None:
        uvw = uvw[row_subsample]
    # without visibilities (vis None) a caller draws its own CN(0, 1) values,
    # e.g. on the device for a large timing workload
    vis = cn_vis(uvw.shape[0], freq.shape[0], npol, rng) if with_vis else None
    return Observation(name=name, uvw_m=uvw, freq_hz=freq, vis=vis, grid_n=grid_n,
                       cell_rad=cell, support_min=s_min, support_max=s_max,
                       oversample=beta, n_wplanes=n_w, w_max_lambda=wmax, npol=npol)


def config_2d(seed_offset: int = 0) -> Observation:
    """2-D gridding, no w-term: 16 antennas in a 1 km disk, 32 hour angles, one
    150 MHz channel, 1 pol; 256^2 grid, support 7, oversampling 8."""
    rng = np.random.default_rng(BASE_SEED + 0 + seed_offset)
    enu = antennas_disk(16, 1000.0, rng)
    return _observation("2d-256-S7", enu, 32, np.array([150e6]), 1, 256, 7, 7, 8, 1, rng)


def config_wproj(seed_offset: int = 0, n_times: int = 256, n_chan: int = 16,
                 row_subsample=None) -> Observation:
    """W-projection, 4 pols: 64 antennas in a 5 km disk, 256 times x 16 channels
    over 120-180 MHz; 4096^2 x 4 grid, 32 w-planes, support 7->63, oversampling 8."""
    rng = np.random.default_rng(BASE_SEED + 1 + seed_offset)
    enu = antennas_disk(64, 5000.0, rng)
    freq = np.linspace(120e6, 180e6, n_chan)
    return _observation("wproj-4096-P32-S7to63-4pol", enu, n_times, freq, 4, 4096, 7, 63,
                        8, 32, rng, row_subsample=row_subsample)


def config_autograd(seed_offset: int = 0, n_times: int = 516) -> Observation:
    """Differentiable imaging: 128 antennas (8,128 baselines) x 516 times, one
    channel, 1 pol; 2048^2 grid, 16 w-planes, support 31, oversampling 8."""
    rng = np.random.default_rng(BASE_SEED + 3 + seed_offset)
    enu = antennas_disk(128, 10000.0, rng)
    return _observation("autograd-2048-P16-S31", enu, n_times, np.array([150e6]), 1, 2048,
                        31, 31, 8, 16, rng)


def config_precision(seed_offset: int = 0, n_times: int = 512, n_chan: int = 8,
                     row_subsample=None, with_vis: bool = True) -> Observation:
    """Mixed precision at scale: 256 antennas spiral+core over 20 km, 512 times x
    8 channels, 4 pols; 8192^2 x 4 grid, 128 w-planes, support 7->127."""
    rng = np.random.default_rng(BASE_SEED + 4 + seed_offset)
    enu = antennas_spiral_core(256, 20000.0, rng)
    freq = np.linspace(120e6, 180e6, n_chan)
    return _observation("precision-8192-P128-S7to127-4pol", enu, n_times, freq, 4, 8192, 7,
                        127, 8, 128, rng, row_subsample=row_subsample, with_vis=with_vis)


def small_case(n_ant: int = 8, n_times: int = 12, n_chan: int = 3, npol: int = 4,
               grid_n: int = 128, s_min: int = 7, s_max: int = 15, beta: int = 8,
               n_w: int = 4, diameter_m: float = 2000.0, seed: int = 7) -> Observation:
    """A small observation for tests: any shape, seeded."""
    rng = np.random.default_rng(BASE_SEED + 100 + seed)
    enu = antennas_disk(n_ant, diameter_m, rng)
    freq = np.linspace(120e6, 180e6, n_chan) if n_chan > 1 else np.array([150e6])
    return _observation(f"small-{grid_n}-P{n_w}", enu, n_times, freq, npol, grid_n, s_min,
                        s_max, beta, n_w, rng)


def random_weights(obs: Observation, seed: int = 11) -> np.ndarray:
    rng = np.random.default_rng(BASE_SEED + 200 + seed)
    return rng.uniform(0.25, 1.75, size=obs.vis.shape).astype(np.float32)


# --------------------------------------------------------------------------
# serving stream: a set of imaging setups and a mixed, Poisson-arriving stream
# --------------------------------------------------------------------------

def serving_setups(n_setups: int = 8, max_vis: int = 10_000_000, seed_offset: int = 0,
                   grid_sizes=(1024, 2048, 4096, 8192), max_rows=None) -> list:
    """Imaging setups for the serving stream.  Each setup: a random array of
    32-256 antennas in a disk (scaled so the field of view is 0.2-0.8 rad
    at the setup's grid size), 1, 4 or 8 channels over 120-180 MHz,
    grid side from ``grid_sizes`` (cycled so every size appears), 1 or 4
    pols, odd S_max in [7, 63] with S_min = 7, 16 w-planes, oversampling 8.
    Returns dicts with the plan arguments, channels, a time-ordered uvw pool
    of at least max_vis / nchan rows ("sorted") and the same rows shuffled."""
    rng = np.random.default_rng(BASE_SEED + 2 + seed_offset)
    out = []
    for k in range(n_setups):
        N = int(grid_sizes[k % len(grid_sizes)])
        npol = (1, 4)[(k // len(grid_sizes) + k) % 2]
        smax = int(2 * rng.integers(3, 32) + 1)
        n_ant = int(rng.integers(32, 257))
        diam = 5e3
        nchan = int(rng.choice([1, 4, 8]))
        freq = np.linspace(120e6, 180e6, nchan) if nchan > 1 else np.array([150e6])
        enu = antennas_disk(n_ant, diam, rng)
        bl = baselines(enu)
        rows = -(-max_vis // nchan) if max_rows is None else int(max_rows)
        n_times = -(-rows // bl.shape[0])
        uvw = uvw_tracks(bl, n_times)
        # scale the array so the field of view L = N cell lands in [0.2, 0.8] rad
        field = fit_cell(uvw, freq, N, smax) * N
        scale = field / float(rng.uniform(0.2, 0.8))
        uvw = uvw * scale
        cell = fit_cell(uvw, freq, N, smax)
        wmax = w_extent(uvw, freq)
        shuffled = uvw[rng.permutation(uvw.shape[0])]
        out.append(dict(
            name=f"setup{k}-N{N}-S{smax}-pol{npol}-ch{nchan}",
            plan_kwargs=dict(grid_n=N, cell_rad=cell, support_min=7, support_max=smax,
                             oversample=8, n_wplanes=16, w_max_lambda=wmax, npol=npol),
            freq_hz=freq, uvw_sorted=uvw, uvw_shuffled=shuffled))
    return out


def serving_jobs(setups: list, n_jobs: int = 256, min_vis: int = 10_000,
                 max_vis: int = 10_000_000, seed_offset: int = 0) -> list:
    """Job specs: kind grid/degrid 50/50, setup uniform, visibility count
    log-uniform in [min_vis, max_vis], uvw rows sorted (a contiguous run of
    the time-ordered pool) or shuffled, 50/50.  Arrival times are set later
    (``poisson_arrivals``)."""
    rng = np.random.default_rng(BASE_SEED + 5 + seed_offset)
    jobs = []
    for i in range(n_jobs):
        s = setups[int(rng.integers(len(setups)))]
        nchan = s["freq_hz"].shape[0]
        nvis = int(np.exp(rng.uniform(np.log(min_vis), np.log(max_vis))))
        nrow = max(1, nvis // nchan)
        pool = s["uvw_sorted"].shape[0]
        jobs.append(dict(id=i, kind=("grid", "degrid")[int(rng.integers(2))], setup=s["name"],
                         nrow=nrow, offset=int(rng.integers(0, pool - nrow + 1)),
                         shuffled=bool(rng.integers(2))))
    return jobs


def poisson_arrivals(n: int, rate_per_s: float, seed_offset: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(BASE_SEED + 6 + seed_offset)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
