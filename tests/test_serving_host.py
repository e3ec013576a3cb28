"""Host-side logic of the serving loop (no GPU): the device-memory arena's
first-fit allocation, release and coalescing, and the per-request memory
estimate."""
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300.serve import ALIGN, Arena


def test_arena_first_fit_release_and_coalesce():
    a = Arena(64 * ALIGN, "cpu")
    x = a.alloc(10 * ALIGN)
    y = a.alloc(1)            # rounded up to one block
    z = a.alloc(20 * ALIGN)
    assert (x, y, z) == (0, 10 * ALIGN, 11 * ALIGN)
    assert a.alloc(40 * ALIGN) is None          # 33 blocks left
    a.release(y, 1)
    assert a.alloc(2 * ALIGN) == 31 * ALIGN     # the hole of one block is too small
    a.release(x, 10 * ALIGN)
    a.release(z, 20 * ALIGN)                    # x, y, z merge into one free run
    assert a.free[0] == (0, 31 * ALIGN)
    assert a.alloc(31 * ALIGN) == 0
    assert a.used == 33 * ALIGN


def test_arena_views_are_aligned_and_typed():
    a = Arena(16 * ALIGN, "cpu")
    off = a.alloc(3 * 8)
    v = a.view(off, 3, torch.float64)
    v[:] = torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64)
    assert v.data_ptr() % ALIGN == a.base % ALIGN
    assert a.view(off, 3, torch.float64).tolist() == [1.0, 2.0, 3.0]
