"""Page-locked host memory on transparent huge pages.

The GPU reaches page-locked host memory through address translations, and
their reach is limited.  On the Grace host of a GB300 (64 KiB base pages,
512 MiB transparent huge pages), device-to-host copies into 2 GiB
``cudaHostAlloc`` buffers ran at 15-110 GB/s instead of the link's 193 GB/s
once about 20 GB of such buffers were used in turn (each buffer fast again
only after a warm-up copy), on a host whose free memory had been churned by
earlier processes.  The same buffers on huge pages (``mmap`` +
``MADV_HUGEPAGE``, touched, then page-locked with ``cudaHostRegister``)
stayed at 193 GB/s (and 211 GB/s host-to-device) in every pass.  Huge pages
only pay for whole pages, so many small buffers are carved from one
``PinnedArena`` instead of being mapped one by one.

Where huge pages are not available (no ``MADV_HUGEPAGE``, a failed
registration) an arena is an ordinary ``pin_memory`` buffer.  Arenas stay
registered until ``release`` or process exit.
"""
import mmap
import threading

import torch

# buffers smaller than this use the ordinary page-locked allocator
MIN_HUGE_BYTES = 64 << 20

_lock = threading.Lock()
_live = {}   # data_ptr of a registered arena's first byte -> arena


def huge_page_bytes() -> int:
    """The transparent huge page size of the host (2 MiB if unknown)."""
    try:
        with open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size") as f:
            return int(f.read().strip())
    except (OSError, ValueError):
        return 2 << 20


def _itemsize(dtype) -> int:
    return torch.empty((), dtype=dtype).element_size()


class PinnedArena:
    """One page-locked host mapping on huge pages; ``take`` hands out
    aligned, non-overlapping tensors from it."""

    def __init__(self, nbytes: int):
        self.nbytes = int(nbytes)
        self.huge = False
        self._mm = None
        self._used = 0
        hp = huge_page_bytes()
        if self.nbytes >= MIN_HUGE_BYTES and hasattr(mmap, "MADV_HUGEPAGE"):
            mm = None
            try:
                # one huge page extra, so the usable part can start on a
                # huge-page boundary wherever the mapping lands
                total = -(-self.nbytes // hp) * hp + hp
                mm = mmap.mmap(-1, total, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
                mm.madvise(mmap.MADV_HUGEPAGE)
                whole = torch.frombuffer(mm, dtype=torch.uint8)
                start = (-whole.data_ptr()) % hp
                raw = whole[start:start + self.nbytes]
                raw.zero_()   # fault every page in now, as huge pages
                err = torch.cuda.cudart().cudaHostRegister(raw.data_ptr(), self.nbytes, 0)
                if int(err) == 0:
                    self._mm, self._raw, self.huge = mm, raw, True
            except (OSError, ValueError, BufferError, RuntimeError, AttributeError):
                self.huge = False
            if not self.huge and mm is not None:
                raw = whole = None
                try:
                    mm.close()
                except BufferError:
                    pass
        if not self.huge:
            self._raw = torch.empty(max(self.nbytes, 1), dtype=torch.uint8, pin_memory=True)
        else:
            # a registered mapping must be unregistered before it is unmapped:
            # the registry keeps it (and its views' memory) alive until release
            with _lock:
                _live[self._raw.data_ptr()] = self

    def take(self, shape, dtype=torch.complex64, align: int = 4096) -> torch.Tensor:
        shape = (shape,) if isinstance(shape, int) else tuple(int(s) for s in shape)
        n = 1
        for s in shape:
            n *= s
        nbytes = n * _itemsize(dtype)
        off = -(-self._used // align) * align
        if off + nbytes > self.nbytes:
            raise ValueError(f"arena of {self.nbytes} bytes cannot hold {nbytes} more bytes "
                             f"after {self._used}")
        self._used = off + nbytes
        return self._raw[off:off + nbytes].view(dtype).view(shape)

    def release(self) -> None:
        """Unregister and unmap (the caller guarantees no pending copy and no
        further use of the tensors taken from the arena)."""
        with _lock:
            _live.pop(self._raw.data_ptr(), None)
        if self.huge:
            torch.cuda.cudart().cudaHostUnregister(self._raw.data_ptr())
            self.huge = False
        self._raw = torch.empty(0, dtype=torch.uint8)
        if self._mm is not None:
            try:
                self._mm.close()
            except BufferError:
                pass   # tensors still view the mapping: it lives until they go
            self._mm = None


def arena_bytes(specs, align: int = 4096) -> int:
    """Bytes an arena needs for tensors of the given (shape, dtype) pairs."""
    total = 0
    for shape, dtype in specs:
        shape = (shape,) if isinstance(shape, int) else tuple(shape)
        n = 1
        for s in shape:
            n *= int(s)
        total = -(-total // align) * align + n * _itemsize(dtype)
    return total


def pinned_empty(shape, dtype=torch.complex64) -> torch.Tensor:
    """An uninitialised page-locked host tensor, on huge pages when it is at
    least MIN_HUGE_BYTES and the host allows it (an arena of its own)."""
    arena = PinnedArena(arena_bytes([(shape, dtype)]))
    t = arena.take(shape, dtype)
    t._gw_arena = arena   # the arena lives as long as the tensor object
    return t


def release(t: torch.Tensor) -> None:
    """Release the arena of a tensor from ``pinned_empty`` (no-op otherwise)."""
    arena = getattr(t, "_gw_arena", None)
    if arena is not None:
        arena.release()


def live_bytes() -> int:
    """Bytes held by registered huge-page arenas."""
    with _lock:
        return sum(a.nbytes for a in _live.values())
