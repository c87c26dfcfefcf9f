"""Host logic of hostmem (no GPU): arena sizing and the carving of aligned,
non-overlapping tensors from one arena."""
import pytest
import torch

from paper_2111_04141_gb300 import hostmem


def _arena_over(buf: torch.Tensor) -> hostmem.PinnedArena:
    # an arena over a plain host buffer: the carving logic without page locking
    a = object.__new__(hostmem.PinnedArena)
    a.nbytes, a.huge, a._mm, a._used, a._raw = buf.numel(), False, None, 0, buf
    return a


def test_arena_bytes_aligns_every_tensor():
    specs = [((10, 3), torch.float64), (5, torch.complex64), ((7,), torch.uint8)]
    # 240 B, then 4096 + 40, then 8192 + 7
    assert hostmem.arena_bytes(specs) == 8192 + 7
    assert hostmem.arena_bytes(specs, align=16) == 240 + 40 + 7 + 8
    assert hostmem.arena_bytes([]) == 0


def test_take_carves_aligned_disjoint_views_and_refuses_overflow():
    specs = [((10, 3), torch.float64), (5, torch.complex64), ((7,), torch.uint8)]
    buf = torch.zeros(hostmem.arena_bytes(specs), dtype=torch.uint8)
    a = _arena_over(buf)
    ts = [a.take(shape, dtype) for shape, dtype in specs]
    assert [tuple(t.shape) for t in ts] == [(10, 3), (5,), (7,)]
    assert [t.dtype for t in ts] == [torch.float64, torch.complex64, torch.uint8]
    offs = [t.data_ptr() - buf.data_ptr() for t in ts]
    assert offs == [0, 4096, 8192]
    for t, v in zip(ts, (1.5, 2 + 3j, 7)):
        t.fill_(v)
    assert torch.all(ts[0] == 1.5) and torch.all(ts[1] == 2 + 3j) and torch.all(ts[2] == 7)
    with pytest.raises(ValueError):
        a.take(1, torch.uint8)


def test_huge_page_size_is_a_power_of_two():
    hp = hostmem.huge_page_bytes()
    assert hp >= 4096 and hp & (hp - 1) == 0
