"""Page-locked host buffers on transparent huge pages.

The GPU reaches page-locked host memory through address translations, and
their reach is limited.  On the Grace host of a GB300 (64 KiB base pages),
device-to-host copies into ``cudaHostAlloc`` buffers ran at 15-110 GB/s
instead of the link's 193 GB/s once about 20 GB of such buffers were in
rotation (each buffer fast again only after a warm-up copy).  The same
buffers on transparent huge pages (512 MiB on that host), mapped with
``mmap`` + ``MADV_HUGEPAGE``, touched, and page-locked with
``cudaHostRegister``, stayed at 193 GB/s in every pass.  Serving keeps
several GB of result staging and job inputs in rotation, so its host buffers
come from here.

Where huge pages are not available (no ``MADV_HUGEPAGE``, a failed
registration) the buffer is an ordinary ``pin_memory`` tensor.  Buffers
stay registered until ``release`` or process exit.
"""
import mmap
import threading

import torch

# buffers smaller than this use the ordinary page-locked allocator
MIN_HUGE_BYTES = 64 << 20

_lock = threading.Lock()
_live = {}   # data_ptr -> (mmap, uint8 view, nbytes)


def _itemsize(dtype) -> int:
    return torch.empty((), dtype=dtype).element_size()


def pinned_empty(shape, dtype=torch.complex64) -> torch.Tensor:
    """An uninitialised page-locked host tensor, on huge pages when it is at
    least MIN_HUGE_BYTES and the host allows it."""
    shape = (shape,) if isinstance(shape, int) else tuple(int(s) for s in shape)
    n = 1
    for s in shape:
        n *= s
    nbytes = n * _itemsize(dtype)
    if nbytes < MIN_HUGE_BYTES or not hasattr(mmap, "MADV_HUGEPAGE"):
        return torch.empty(shape, dtype=dtype, pin_memory=True)
    try:
        mm = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        mm.madvise(mmap.MADV_HUGEPAGE)
    except (OSError, ValueError):
        return torch.empty(shape, dtype=dtype, pin_memory=True)
    raw = torch.frombuffer(mm, dtype=torch.uint8)
    raw.zero_()   # fault every page in now, as huge pages
    err = torch.cuda.cudart().cudaHostRegister(raw.data_ptr(), nbytes, 0)
    if int(err) != 0:
        del raw
        mm.close()
        return torch.empty(shape, dtype=dtype, pin_memory=True)
    with _lock:
        _live[raw.data_ptr()] = (mm, raw, nbytes)
    return raw.view(dtype).view(shape)


def release(t: torch.Tensor) -> None:
    """Unregister and unmap a tensor from ``pinned_empty`` (no-op for any
    other tensor).  The caller guarantees that no copy into or out of it is
    pending and that no view of it is used afterwards."""
    with _lock:
        ent = _live.pop(t.data_ptr(), None)
    if ent is None:
        return
    mm, raw, _ = ent
    torch.cuda.cudart().cudaHostUnregister(raw.data_ptr())
    del raw
    try:
        mm.close()
    except BufferError:
        pass   # views still export the buffer: the mapping lives until they go


def live_bytes() -> int:
    """Bytes currently held by ``pinned_empty`` huge-page buffers."""
    with _lock:
        return sum(e[2] for e in _live.values())
