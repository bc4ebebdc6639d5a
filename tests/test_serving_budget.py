"""Host logic of the serving loop: families are built under a device-memory
budget, idle families are evicted least recently used first, a family that
does not fit waits while every built family is busy (and is not built while
it waits: its size is known beforehand), and a family larger than the whole
budget is an error.  The engines are stand-ins with the interface the server
uses (estimate_bytes, bytes, busy, close, last_used), so no GPU work is
involved."""
import pytest

import numpy as np

from paper_2412_10910_gb300.serving import Server, batch_width, pack_plan, parallel_copy


class FakeEngine:
    sizes = {}
    clock = [0.0]
    built = []

    @staticmethod
    def estimate_bytes(name, spec, **kw):
        return FakeEngine.sizes[name]

    def __init__(self, name, spec, **kw):
        FakeEngine.built.append(name)
        self.name = name
        self.kw = kw
        self.is_busy = False
        self.closed = False
        FakeEngine.clock[0] += 1.0
        self.last_used = FakeEngine.clock[0]

    def bytes(self):
        return FakeEngine.sizes[self.name]

    def busy(self):
        return self.is_busy

    def close(self):
        self.closed = True


def _server(sizes, budget):
    FakeEngine.sizes = dict(sizes)
    FakeEngine.built = []
    return Server({n: None for n in sizes}, budget_bytes=budget, engine_factory=FakeEngine)


def test_families_fill_the_budget_then_evict_least_recently_used():
    s = _server({"a": 40, "b": 40, "c": 40}, 100)
    a, b = s.engine("a"), s.engine("b")
    assert s.used_bytes() == 80 and s.evictions == 0
    assert s.engine("a") is a                      # cached, not rebuilt
    a.last_used, b.last_used = 10.0, 5.0           # b is the least recently used
    c = s.engine("c")
    assert c is not None and b.closed and not a.closed
    assert sorted(s.engines) == ["a", "c"] and s.evictions == 1
    assert s.used_bytes() <= 100


def test_busy_families_are_not_evicted_and_the_newcomer_waits():
    s = _server({"a": 60, "b": 60}, 100)
    a = s.engine("a")
    a.is_busy = True
    for _ in range(5):
        assert s.engine("b") is None               # must wait, nothing evicted
    assert not a.closed and s.evictions == 0 and list(s.engines) == ["a"]
    assert FakeEngine.built == ["a"] and s.builds == 1   # "b" never built while it waits
    a.is_busy = False
    b = s.engine("b")
    assert b is not None and a.closed and s.evictions == 1


def test_a_family_larger_than_the_budget_is_an_error():
    s = _server({"big": 500}, 100)
    with pytest.raises(MemoryError):
        s.engine("big")
    assert FakeEngine.built == []                  # rejected before anything is built


def test_server_passes_the_solver_settings_to_its_engines():
    s = _server({"a": 1}, 100)
    e = s.engine("a")
    assert e.kw == {"nslots": 16, "mode": 1, "rtol": 1e-8, "maxit": 200}
    s.close()
    assert e.closed and not s.engines


def test_batch_width_rounds_up_to_even_within_the_slots():
    assert [batch_width(n, 16) for n in (0, 1, 2, 3, 8, 9, 15, 16, 17)] == \
        [1, 1, 2, 4, 8, 10, 16, 16, 16]
    assert batch_width(5, 4) == 4


def test_pack_plan_moves_occupied_slots_first_and_sets_the_width():
    A, B, Cq = object(), object(), object()
    owner = [A, None, B, None, Cq] + [None] * 11
    # three occupied of 16 columns: packed in order into 4 columns
    assert pack_plan(owner, 16, 3, 16) == (4, [0, 2, 4, -1])
    # room for two more columns being admitted: 5 -> 6 columns
    assert pack_plan(owner, 16, 5, 16) == (6, [0, 2, 4, -1, -1, -1])
    # already packed at the right width: nothing to do
    packed = [A, B] + [None] * 14
    assert pack_plan(packed, 2, 2, 16) is None
    # packed, but a new request needs 7 more columns: widen, keep the order
    assert pack_plan(packed, 2, 9, 16) == (10, [0, 1] + [-1] * 8)
    # a retired column in front: the others move up even at the same width
    assert pack_plan([None, A] + [None] * 14, 2, 1, 16) == (1, [1])
    # never narrower than the occupied columns, never wider than the slots
    assert pack_plan(owner, 16, 0, 16) == (4, [0, 2, 4, -1])
    full = [A] * 16
    assert pack_plan(full, 16, 20, 16) is None


@pytest.mark.parametrize("shape", [(5,), (1000, 3), (700_001, 4)])
def test_parallel_copy_equals_a_plain_copy(shape):
    rng = np.random.default_rng(1)
    src = rng.standard_normal(shape)
    dst = np.zeros(shape)
    parallel_copy(dst, src, chunk_bytes=1 << 16)
    assert np.array_equal(dst, src)
    col = np.zeros((shape[-1], shape[0])).T          # column-major destination
    parallel_copy(col[:, 0] if col.ndim == 2 else col, src[:, 0] if src.ndim == 2 else src,
                  chunk_bytes=1 << 12)
    assert np.array_equal(col[:, 0] if col.ndim == 2 else col, src[:, 0] if src.ndim == 2 else src)
