"""Python face of the libgw C ABI: a Plan object over torch CUDA tensors.

Only argument marshalling happens here; every step of gridding,
degridding, index selection, binning, table generation and correction runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import GwError, PlanDesc, PlanInfo, check

_DTYPES = {"c64": _lib.GW_C64, "bf16": _lib.GW_BF16X2, "f16": _lib.GW_F16X2}
# torch storage of each kind: complex64 [..., npol], or 16-bit reals [..., npol, 2]
_TORCH = {"c64": torch.complex64, "bf16": torch.bfloat16, "f16": torch.float16}


def vis_shape(kind: str, nrow: int, nchan: int, npol: int):
    return (nrow, nchan, npol) if kind == "c64" else (nrow, nchan, npol, 2)


def to_storage(vis: torch.Tensor, kind: str) -> torch.Tensor:
    """complex64 visibilities -> the storage layout of ``kind`` (rounded to nearest)."""
    if kind == "c64":
        return vis.to(torch.complex64).contiguous()
    return torch.view_as_real(vis.to(torch.complex64)).to(_TORCH[kind]).contiguous()


def from_storage(vis: torch.Tensor) -> torch.Tensor:
    """Visibilities in any storage layout -> complex64 (exact widening)."""
    if vis.dtype == torch.complex64:
        return vis
    if vis.dtype == torch.complex32:
        return vis.to(torch.complex64)
    return torch.view_as_complex(vis.float().contiguous())


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream, device):
    s = torch.cuda.current_stream(device) if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, name: str, dtype, device, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class Plan:
    """A gridding/degridding plan on one CUDA device (see include/gw.h)."""

    def __init__(self, grid_n: int, cell_rad: float, support_min: int, support_max: int,
                 oversample: int = 8, n_wplanes: int = 1, w_max_lambda: float = 0.0,
                 npol: int = 1, vis_dtype: str = "c64", table_dtype: str = "c64",
                 max_vis_per_call: int = 0, device=None, stream=None):
        self._lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        d = PlanDesc(grid_n=int(grid_n), cell_rad=float(cell_rad), support_min=int(support_min),
                     support_max=int(support_max), oversample=int(oversample),
                     n_wplanes=int(n_wplanes), w_max_lambda=float(w_max_lambda), npol=int(npol),
                     vis_dtype=_DTYPES[vis_dtype], table_dtype=_DTYPES[table_dtype],
                     max_vis_per_call=int(max_vis_per_call))
        self.desc = d
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._lib.gw_plan_create(ctypes.byref(d), _stream_ptr(stream, self.device),
                                           ctypes.byref(self._h)), "gw_plan_create")
        info = PlanInfo()
        check(self._lib.gw_plan_info_get(self._h, ctypes.byref(info)), "gw_plan_info_get")
        self.info = info
        self.grid_n = int(grid_n)
        self.npol = int(npol)
        self.vis_dtype = vis_dtype
        self.table_dtype = table_dtype

    def clone(self, max_vis_per_call: int = 0, stream=None) -> "Plan":
        """A plan sharing this plan's kernel tables with its own scratch
        (gw_plan_clone): clones may run concurrently on different streams."""
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._lib.gw_plan_clone(self._h, int(max_vis_per_call),
                                          _stream_ptr(stream, self.device), ctypes.byref(h)),
                  "gw_plan_clone")
        c = Plan.__new__(Plan)
        c._lib, c.device, c._h = self._lib, self.device, h
        d = PlanDesc()
        ctypes.pointer(d)[0] = self.desc
        d.max_vis_per_call = int(max_vis_per_call)
        c.desc = d
        info = PlanInfo()
        check(self._lib.gw_plan_info_get(h, ctypes.byref(info)), "gw_plan_info_get")
        c.info = info
        c.grid_n, c.npol = self.grid_n, self.npol
        c.vis_dtype, c.table_dtype = self.vis_dtype, self.table_dtype
        return c

    def get_tuning(self) -> dict:
        t = _lib.Tuning()
        check(self._lib.gw_plan_get_tuning(self._h, ctypes.byref(t)), "gw_plan_get_tuning")
        return {"item_max": t.item_max, "degrid_kernel": t.degrid_kernel,
                "grid_kernel": t.grid_kernel, "compress_min_gain": t.compress_min_gain,
                "plane_groups": t.plane_groups}

    def set_tuning(self, item_max: int = 0, degrid_kernel: int = 0, grid_kernel: int = 0,
                   compress_min_gain: int = 0, plane_groups: int = 0):
        t = _lib.Tuning(item_max=int(item_max), degrid_kernel=int(degrid_kernel),
                        grid_kernel=int(grid_kernel), compress_min_gain=int(compress_min_gain),
                        plane_groups=int(plane_groups))
        check(self._lib.gw_plan_set_tuning(self._h, ctypes.byref(t)), "gw_plan_set_tuning")
        info = PlanInfo()   # plane_groups follows the tuning
        check(self._lib.gw_plan_info_get(self._h, ctypes.byref(info)), "gw_plan_info_get")
        self.info = info

    @classmethod
    def from_observation(cls, obs, **kw):
        args = dict(obs.plan_kwargs())
        args.update(kw)
        return cls(**args)

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            with torch.cuda.device(self.device):
                torch.cuda.synchronize(self.device)
                self._lib.gw_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def _coords(self, uvw, freq):
        _need(uvw, "uvw", torch.float64, self.device)
        _need(freq, "freq", torch.float64, self.device)
        if uvw.dim() != 2 or uvw.shape[1] != 3:
            raise ValueError("uvw must be [nrow, 3]")
        if freq.dim() != 1:
            raise ValueError("freq must be [nchan]")
        return int(uvw.shape[0]), int(freq.shape[0])

    def _vis_arg(self, vis, name, nrow, nchan):
        """Validate a visibility tensor in the plan's storage kind."""
        k = self.vis_dtype
        if k == "f16" and isinstance(vis, torch.Tensor) and vis.dtype == torch.complex32:
            vis = torch.view_as_real(vis)
        _need(vis, name, _TORCH[k], self.device, vis_shape(k, nrow, nchan, self.npol))
        return vis

    def new_vis(self, nrow: int, nchan: int) -> torch.Tensor:
        return torch.empty(vis_shape(self.vis_dtype, nrow, nchan, self.npol),
                           dtype=_TORCH[self.vis_dtype], device=self.device)

    def new_grid(self) -> torch.Tensor:
        return torch.zeros((self.npol, self.grid_n, self.grid_n), dtype=torch.complex64,
                           device=self.device)

    def grid(self, uvw, freq, vis, weight=None, out=None, stream=None, return_dropped=False,
             err=None):
        """Accumulate vis (plan's storage kind, [nrow, nchan, npol] complex64 or
        [nrow, nchan, npol, 2] 16-bit) onto out (new zero grid if None).

        With ``err`` (a [npol, N, N] complex64 tensor, zeroed with the grid)
        commits are compensated (gw_grid_vis_compensated); call ``fold`` once
        all calls into the grid are done."""
        nrow, nchan = self._coords(uvw, freq)
        vis = self._vis_arg(vis, "vis", nrow, nchan)
        if weight is not None:
            _need(weight, "weight", torch.float32, self.device, (nrow, nchan, self.npol))
        if out is None:
            out = self.new_grid()
        gshape = (self.npol, self.grid_n, self.grid_n)
        _need(out, "grid", torch.complex64, self.device, gshape)
        dropped = ctypes.c_int64(-1)
        dp = ctypes.byref(dropped) if return_dropped else None
        with torch.cuda.device(self.device):
            if err is None:
                check(self._lib.gw_grid_vis(self._h, _ptr(uvw), _ptr(freq), nrow, nchan,
                                            _ptr(vis), _ptr(weight), _ptr(out), dp,
                                            _stream_ptr(stream, self.device)), "gw_grid_vis")
            else:
                _need(err, "err", torch.complex64, self.device, gshape)
                check(self._lib.gw_grid_vis_compensated(
                    self._h, _ptr(uvw), _ptr(freq), nrow, nchan, _ptr(vis), _ptr(weight),
                    _ptr(out), _ptr(err), dp, _stream_ptr(stream, self.device)),
                    "gw_grid_vis_compensated")
        return (out, int(dropped.value)) if return_dropped else out

    def grid_devcount(self, uvw, freq, d_nrow, vis, out, stream=None):
        """gw_grid_vis_devcount: rows [0, d_nrow[0]) of uvw/vis (buffers sized
        for uvw.shape[0] rows) onto ``out``; capturable in a CUDA graph."""
        max_nrow, nchan = self._coords(uvw, freq)
        vis = self._vis_arg(vis, "vis", max_nrow, nchan)
        _need(d_nrow, "d_nrow", torch.int64, self.device, (1,))
        _need(out, "grid", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        check(self._lib.gw_grid_vis_devcount(self._h, _ptr(uvw), _ptr(freq), _ptr(d_nrow),
                                             max_nrow, nchan, _ptr(vis), _ptr(out),
                                             _stream_ptr(stream, self.device)),
              "gw_grid_vis_devcount")
        return out

    def grid_devcount_readback(self, uvw, freq, d_nrow, vis, out, host_out, n_bands=8,
                               stream=None):
        """gw_grid_vis_devcount_readback: as grid_devcount, and the grid is
        copied band by band to ``host_out`` (a page-locked host tensor of the
        grid's shape) while later bands grid; work issued later on the stream
        waits for the copies.  Capturable in a CUDA graph after the plan's
        first call."""
        max_nrow, nchan = self._coords(uvw, freq)
        vis = self._vis_arg(vis, "vis", max_nrow, nchan)
        _need(d_nrow, "d_nrow", torch.int64, self.device, (1,))
        gshape = (self.npol, self.grid_n, self.grid_n)
        _need(out, "grid", torch.complex64, self.device, gshape)
        if (not isinstance(host_out, torch.Tensor) or host_out.device.type != "cpu"
                or host_out.dtype != torch.complex64 or tuple(host_out.shape) != gshape
                or not host_out.is_contiguous()):
            raise TypeError(f"host_out must be a contiguous host complex64 tensor of shape {gshape}")
        if not host_out.is_pinned():
            raise ValueError("host_out must be page-locked (pin_memory())")
        check(self._lib.gw_grid_vis_devcount_readback(
            self._h, _ptr(uvw), _ptr(freq), _ptr(d_nrow), max_nrow, nchan, _ptr(vis), _ptr(out),
            _ptr(host_out), int(n_bands), _stream_ptr(stream, self.device)),
            "gw_grid_vis_devcount_readback")
        return out

    def degrid_devcount(self, uvw, freq, d_nrow, grid, out, stream=None):
        """gw_degrid_vis_devcount: rows [0, d_nrow[0]) of ``out`` from ``grid``."""
        max_nrow, nchan = self._coords(uvw, freq)
        _need(d_nrow, "d_nrow", torch.int64, self.device, (1,))
        _need(grid, "grid", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        out = self._vis_arg(out, "vis_out", max_nrow, nchan)
        check(self._lib.gw_degrid_vis_devcount(self._h, _ptr(uvw), _ptr(freq), _ptr(d_nrow),
                                               max_nrow, nchan, _ptr(grid), _ptr(out),
                                               _stream_ptr(stream, self.device)),
              "gw_degrid_vis_devcount")
        return out

    def grid_compressed(self, uvw, freq, vis, weight=None, out=None, stream=None):
        """Gridding with full compression (gw_grid_vis_compressed).  Returns
        (grid, records gridded after compression, dropped)."""
        nrow, nchan = self._coords(uvw, freq)
        vis = self._vis_arg(vis, "vis", nrow, nchan)
        if weight is not None:
            _need(weight, "weight", torch.float32, self.device, (nrow, nchan, self.npol))
        if out is None:
            out = self.new_grid()
        _need(out, "grid", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        ng, nd = ctypes.c_int64(-1), ctypes.c_int64(-1)
        with torch.cuda.device(self.device):
            check(self._lib.gw_grid_vis_compressed(self._h, _ptr(uvw), _ptr(freq), nrow, nchan,
                                                   _ptr(vis), _ptr(weight), _ptr(out),
                                                   ctypes.byref(ng), ctypes.byref(nd),
                                                   _stream_ptr(stream, self.device)),
                  "gw_grid_vis_compressed")
        return out, int(ng.value), int(nd.value)

    def grid_wstack(self, uvw, freq, vis, n_layers, w_min, w_max, weight=None, out=None,
                    stream=None, return_dropped=False):
        """W-stacking gridding (gw_grid_vis_wstack) onto [n_layers, npol, N, N]."""
        nrow, nchan = self._coords(uvw, freq)
        vis = self._vis_arg(vis, "vis", nrow, nchan)
        if weight is not None:
            _need(weight, "weight", torch.float32, self.device, (nrow, nchan, self.npol))
        shape = (int(n_layers), self.npol, self.grid_n, self.grid_n)
        if out is None:
            out = torch.zeros(shape, dtype=torch.complex64, device=self.device)
        _need(out, "layers", torch.complex64, self.device, shape)
        nd = ctypes.c_int64(-1)
        with torch.cuda.device(self.device):
            check(self._lib.gw_grid_vis_wstack(self._h, _ptr(uvw), _ptr(freq), nrow, nchan,
                                               _ptr(vis), _ptr(weight), int(n_layers),
                                               float(w_min), float(w_max), _ptr(out),
                                               ctypes.byref(nd) if return_dropped else None,
                                               _stream_ptr(stream, self.device)),
                  "gw_grid_vis_wstack")
        return (out, int(nd.value)) if return_dropped else out

    def wstack_combine(self, layer_images, w_min, w_max, image, stream=None):
        """image += sum over layers of the layer image times its w-screen."""
        L = int(layer_images.shape[0])
        _need(layer_images, "layer_images", torch.complex64, self.device,
              (L, self.npol, self.grid_n, self.grid_n))
        _need(image, "image", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        with torch.cuda.device(self.device):
            check(self._lib.gw_wstack_combine(self._h, _ptr(layer_images), L, float(w_min),
                                              float(w_max), _ptr(image),
                                              _stream_ptr(stream, self.device)),
                  "gw_wstack_combine")
        return image

    def hybrid_grid(self, uvw, freq, vis, sz, weight=None, out=None, stream=None,
                    return_dropped=False):
        """Hybrid Gridding Step onto the fine grid [beta N, N, npol]
        (polarisations interleaved)."""
        nrow, nchan = self._coords(uvw, freq)
        vis = self._vis_arg(vis, "vis", nrow, nchan)
        if weight is not None:
            _need(weight, "weight", torch.float32, self.device, (nrow, nchan, self.npol))
        shape = self.fine_shape()
        if out is None:
            out = torch.zeros(shape, dtype=torch.complex64, device=self.device)
        _need(out, "fine", torch.complex64, self.device, shape)
        nd = ctypes.c_int64(-1)
        with torch.cuda.device(self.device):
            check(self._lib.gw_hybrid_grid(self._h, _ptr(uvw), _ptr(freq), nrow, nchan, _ptr(vis),
                                           _ptr(weight), int(sz), _ptr(out),
                                           ctypes.byref(nd) if return_dropped else None,
                                           _stream_ptr(stream, self.device)), "gw_hybrid_grid")
        return (out, int(nd.value)) if return_dropped else out

    def fine_shape(self):
        """Shape of the Hybrid Gridding fine grid: (beta N, N, npol)."""
        return (self.desc.oversample * self.grid_n, self.grid_n, self.npol)

    def hybrid_prune(self, sz, fine, out=None, stream=None):
        shape = (self.npol, 2 * self.grid_n, self.grid_n)
        _need(fine, "fine", torch.complex64, self.device, self.fine_shape())
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device=self.device)
        _need(out, "pruned", torch.complex64, self.device, shape)
        with torch.cuda.device(self.device):
            check(self._lib.gw_hybrid_prune(self._h, int(sz), _ptr(fine), _ptr(out),
                                            _stream_ptr(stream, self.device)), "gw_hybrid_prune")
        return out

    def hybrid_shift(self, pruned, stream=None):
        _need(pruned, "pruned", torch.complex64, self.device,
              (self.npol, 2 * self.grid_n, self.grid_n))
        with torch.cuda.device(self.device):
            check(self._lib.gw_hybrid_shift(self._h, _ptr(pruned), _stream_ptr(stream, self.device)),
                  "gw_hybrid_shift")
        return pruned

    def hybrid_image(self, sz, raw, out=None, stream=None):
        _need(raw, "raw", torch.complex64, self.device, (self.npol, 2 * self.grid_n, self.grid_n))
        if out is None:
            out = self.new_grid()
        _need(out, "image", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        with torch.cuda.device(self.device):
            check(self._lib.gw_hybrid_image(self._h, int(sz), _ptr(raw), _ptr(out),
                                            _stream_ptr(stream, self.device)), "gw_hybrid_image")
        return out

    def grid_host(self, uvw, freq, vis, weight=None, out=None, stream=None,
                  return_dropped=False):
        """gw_grid_vis_host: uvw/freq/vis (and weight) are HOST tensors
        (page-locked for overlap); their copies to the device are pipelined
        with the gridding.  ``out`` is a device grid."""
        def host(t, name, dtype):
            if not isinstance(t, torch.Tensor) or t.device.type != "cpu" or t.dtype != dtype:
                raise TypeError(f"{name} must be a host {dtype} tensor")
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
        host(uvw, "uvw", torch.float64)
        host(freq, "freq", torch.float64)
        nrow, nchan = int(uvw.shape[0]), int(freq.shape[0])
        k = self.vis_dtype
        vt = vis
        if k == "f16" and vis.dtype == torch.complex32:
            vt = torch.view_as_real(vis)
        host(vt, "vis", _TORCH[k])
        if tuple(vt.shape) != vis_shape(k, nrow, nchan, self.npol):
            raise ValueError("vis has the wrong shape")
        if weight is not None:
            host(weight, "weight", torch.float32)
        if out is None:
            out = self.new_grid()
        _need(out, "grid", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        nd = ctypes.c_int64(-1)
        with torch.cuda.device(self.device):
            check(self._lib.gw_grid_vis_host(self._h, _ptr(uvw), _ptr(freq), nrow, nchan,
                                             _ptr(vt), _ptr(weight), _ptr(out),
                                             ctypes.byref(nd) if return_dropped else None,
                                             _stream_ptr(stream, self.device)),
                  "gw_grid_vis_host")
        return (out, int(nd.value)) if return_dropped else out

    def fold(self, grid, err, stream=None):
        """grid += err; err = 0 (ends a compensated gridding sequence)."""
        gshape = (self.npol, self.grid_n, self.grid_n)
        _need(grid, "grid", torch.complex64, self.device, gshape)
        _need(err, "err", torch.complex64, self.device, gshape)
        with torch.cuda.device(self.device):
            check(self._lib.gw_grid_fold(self._h, _ptr(grid), _ptr(err),
                                         _stream_ptr(stream, self.device)), "gw_grid_fold")
        return grid

    def degrid(self, uvw, freq, grid, out=None, stream=None, return_dropped=False):
        """Visibilities (plan's storage kind) from grid [npol, N, N] (overwrites out)."""
        nrow, nchan = self._coords(uvw, freq)
        _need(grid, "grid", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        if out is None:
            out = self.new_vis(nrow, nchan)
        out = self._vis_arg(out, "vis_out", nrow, nchan)
        dropped = ctypes.c_int64(-1)
        with torch.cuda.device(self.device):
            check(self._lib.gw_degrid_vis(self._h, _ptr(uvw), _ptr(freq), nrow, nchan, _ptr(grid),
                                          _ptr(out),
                                          ctypes.byref(dropped) if return_dropped else None,
                                          _stream_ptr(stream, self.device)), "gw_degrid_vis")
        return (out, int(dropped.value)) if return_dropped else out

    def degrid_static(self, uvw, freq, grid, out=None, stream=None, return_dropped=False):
        """Degrid without allocating device memory (gw_degrid_vis_static).

        For callers that cannot allocate while running: scratch comes from a
        fixed device array inside the library (<= 65536 visibilities per call,
        grid_n <= 8192).  ``out`` must be supplied by such callers; calls that
        overlap on the GPU race on the shared array.
        """
        nrow, nchan = self._coords(uvw, freq)
        _need(grid, "grid", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        if out is None:
            out = self.new_vis(nrow, nchan)
        out = self._vis_arg(out, "vis_out", nrow, nchan)
        dropped = ctypes.c_int64(-1)
        with torch.cuda.device(self.device):
            check(self._lib.gw_degrid_vis_static(self._h, _ptr(uvw), _ptr(freq), nrow, nchan,
                                                 _ptr(grid), _ptr(out),
                                                 ctypes.byref(dropped) if return_dropped else None,
                                                 _stream_ptr(stream, self.device)),
                  "gw_degrid_vis_static")
        return (out, int(dropped.value)) if return_dropped else out

    def correct(self, image, direction: int = 1, stream=None):
        _need(image, "image", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        with torch.cuda.device(self.device):
            check(self._lib.gw_grid_correct(self._h, _ptr(image), int(direction),
                                            _stream_ptr(stream, self.device)), "gw_grid_correct")
        return image

    def shift(self, grid, stream=None):
        _need(grid, "grid", torch.complex64, self.device, (self.npol, self.grid_n, self.grid_n))
        with torch.cuda.device(self.device):
            check(self._lib.gw_grid_shift(self._h, _ptr(grid), _stream_ptr(stream, self.device)),
                  "gw_grid_shift")
        return grid

    def index(self, uvw, freq, stream=None):
        """Raw index records as an int32 tensor [nvis, 4] plus the drop count.

        Column 0 = ku, 1 = kv, 2 = (ou & 0xffff) | (ov << 16), 3 = plane | flags << 16.
        """
        nrow, nchan = self._coords(uvw, freq)
        out = torch.empty((nrow * nchan, 4), dtype=torch.int32, device=self.device)
        dropped = ctypes.c_int64(-1)
        with torch.cuda.device(self.device):
            check(self._lib.gw_index_vis(self._h, _ptr(uvw), _ptr(freq), nrow, nchan, _ptr(out),
                                         ctypes.byref(dropped), _stream_ptr(stream, self.device)),
                  "gw_index_vis")
        return out, int(dropped.value)

    @staticmethod
    def unpack_index(raw: np.ndarray) -> dict:
        raw = np.ascontiguousarray(raw, dtype=np.int32)
        h16 = raw[:, 2:4].copy().view(np.int16).reshape(-1, 4)
        return dict(ku=raw[:, 0].astype(np.int64), kv=raw[:, 1].astype(np.int64),
                    ou=h16[:, 0].astype(np.int64), ov=h16[:, 1].astype(np.int64),
                    plane=h16[:, 2].astype(np.int64),
                    flags=h16[:, 3].astype(np.uint16).astype(np.int64))

    def tables(self):
        P = self.info.n_wplanes
        buf = np.empty(2 * self.info.table_elems, dtype=np.float32)
        offs = np.empty(P + 1, dtype=np.int64)
        sup = np.empty(P, dtype=np.int32)
        with torch.cuda.device(self.device):
            check(self._lib.gw_plan_copy_tables(self._h, buf.ctypes.data_as(ctypes.c_void_p),
                                                offs.ctypes.data_as(ctypes.c_void_p),
                                                sup.ctypes.data_as(ctypes.c_void_p)),
                  "gw_plan_copy_tables")
        return buf.view(np.complex64), offs, sup

    def stored_tables(self):
        """The tables as stored: complex64 for c64 plans, else uint16 [..., 2]
        raw 16-bit pairs (scaled by 2^info.table_exp2), flat like ``tables``."""
        n = self.info.table_elems
        if self.table_dtype == "c64":
            buf = np.empty(n, dtype=np.complex64)
        else:
            buf = np.empty((n, 2), dtype=np.uint16)
        with torch.cuda.device(self.device):
            check(self._lib.gw_plan_copy_stored_tables(self._h, buf.ctypes.data_as(ctypes.c_void_p)),
                  "gw_plan_copy_stored_tables")
        return buf

    def corrector(self):
        h = np.empty(self.grid_n, dtype=np.float64)
        with torch.cuda.device(self.device):
            check(self._lib.gw_plan_copy_corrector(self._h, h.ctypes.data_as(ctypes.c_void_p)),
                  "gw_plan_copy_corrector")
        return h

    def device_status(self, stream=None):
        """Synchronise the stream and raise GwError (GW_ETIMEDOUT) if a
        bounded device-side wait gave up since the last check."""
        with torch.cuda.device(self.device):
            check(self._lib.gw_plan_device_status(self._h, _stream_ptr(stream, self.device)),
                  "gw_plan_device_status")

    def timing(self, enable=None):
        """With ``enable`` set, switch stage timing on/off; otherwise return and
        reset the accumulated per-stage timings and work counters as a dict."""
        if enable is not None:
            check(self._lib.gw_plan_timing_enable(self._h, int(bool(enable))),
                  "gw_plan_timing_enable")
            return None
        t = _lib.Timing()
        with torch.cuda.device(self.device):
            check(self._lib.gw_plan_timing_get(self._h, ctypes.byref(t)), "gw_plan_timing_get")
        return {name: getattr(t, name) for name, _ in t._fields_}

    def debug_bins(self, uvw, freq, mode: int = 0, capacity: Optional[int] = None, stream=None):
        nrow, nchan = self._coords(uvw, freq)
        if mode == 0:
            tu, tv = self.info.grid_tile_u, self.info.grid_tile_v
        else:
            tu = tv = self.info.degrid_tile
        ntiles = ((self.grid_n + tu - 1) // tu) * ((self.grid_n + tv - 1) // tv)
        offs = np.empty(ntiles + 1, dtype=np.int64)
        cap = capacity if capacity is not None else max(1, nrow * nchan * 16)
        ent = np.empty(cap, dtype=np.uint32)
        with torch.cuda.device(self.device):
            check(self._lib.gw_debug_bins(self._h, _ptr(uvw), _ptr(freq), nrow, nchan, int(mode),
                                          offs.ctypes.data_as(ctypes.c_void_p),
                                          ent.ctypes.data_as(ctypes.c_void_p), cap,
                                          _stream_ptr(stream, self.device)), "gw_debug_bins")
        return offs, ent[:offs[-1]]


def ffma_peak(iters: int = 4096, stream=None) -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s (gw_ffma_peak)."""
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    dev = torch.device("cuda", torch.cuda.current_device())
    check(lib.gw_ffma_peak(int(iters), ctypes.byref(out), _stream_ptr(stream, dev)), "gw_ffma_peak")
    return float(out.value)


def launch_count() -> int:
    return int(_lib.load().gw_launch_count())


def debug_fail_alloc(n: int) -> None:
    """Test hook: the n-th library allocation from now fails (0 = off)."""
    check(_lib.load().gw_debug_fail_alloc(int(n)), "gw_debug_fail_alloc")


def live_plans() -> int:
    """Plans and clones created and not yet destroyed in this process."""
    return int(_lib.load().gw_debug_live_plans())


def live_bytes() -> int:
    """Device bytes the library has allocated and not freed (all plans)."""
    return int(_lib.load().gw_debug_live_bytes())
