"""Host logic of the unrolled engine pool (paper_2209_11002_gb300/autograd.py):
engines are created per shape, reused after release, never shared by two
live contexts, and destroyed by free_engines().  A fake library stands in for
libedaa (no GPU needed)."""
import ctypes

import pytest

from paper_2209_11002_gb300 import autograd as AG
from paper_2209_11002_gb300 import edaa


class _FakeLib:
    def __init__(self):
        self.created, self.destroyed, self.next = [], [], 1

    def edaa_unrolled_create(self, out, L, N, p, T, K1, K2, stream):
        out._obj.value = self.next
        self.created.append((self.next, (L, N, p, T, K1, K2)))
        self.next += 1
        return 0

    def edaa_unrolled_destroy(self, h):
        self.destroyed.append(h.value)


@pytest.fixture
def fake(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(edaa, "load_library", lambda: lib)
    monkeypatch.setattr(AG.torch.cuda, "current_device", lambda: 0)
    AG._POOL.clear()
    yield lib
    AG._POOL.clear()


def test_pool_reuses_released_engines_per_shape(fake):
    e1 = AG._Engine(10, 100, 3, 2, 5, 5, None)
    e2 = AG._Engine(10, 100, 3, 2, 5, 5, None)       # e1 still held: a second engine
    assert len(fake.created) == 2 and e1.h.value != e2.h.value
    h1 = e1.h.value
    e1.release()
    e3 = AG._Engine(10, 100, 3, 2, 5, 5, None)       # takes e1's engine back
    assert len(fake.created) == 2 and e3.h.value == h1
    e4 = AG._Engine(11, 100, 3, 2, 5, 5, None)       # another shape: a new engine
    assert len(fake.created) == 3
    e5 = AG._Engine(10, 100, 3, 2, 5, 5, ctypes.c_void_p(1234))  # another stream: a new engine
    assert len(fake.created) == 4
    for e in (e2, e3, e4, e5):
        e.release()
    e2.release()                                      # a second release is a no-op
    assert sum(len(v) for v in AG._POOL.values()) == 4
    AG.free_engines()
    assert sorted(fake.destroyed) == [1, 2, 3, 4] and not AG._POOL


def test_dropped_engine_returns_to_pool(fake):
    e = AG._Engine(8, 50, 2, 1, 1, 1, None)
    h = e.h.value
    del e                                             # a context freed without a backward
    assert AG._POOL and list(AG._POOL.values())[0][0].value == h
