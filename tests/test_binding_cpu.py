"""Host logic of the Python binding without a GPU: the version tracking that
tells the library when a borrowed leaf tensor changed in place."""
import pytest

torch = pytest.importorskip("torch")


class _FakeLib:
    def __init__(self):
        self.calls = []

    def cola_linop_cache_prepared(self, h, on):
        self.calls.append(("cache", h, on))
        return 0

    def cola_linop_touch(self, h):
        self.calls.append(("touch", h))
        return 0


@pytest.fixture()
def fake(monkeypatch):
    import paper_2309_03060_gb300 as cola
    lib = _FakeLib()
    monkeypatch.setattr(cola, "_lib", lambda: lib)
    return cola, lib


def test_leaf_enables_cache_and_touches_only_after_in_place_change(fake):
    cola, lib = fake
    t = torch.zeros(4, 4)
    leaf = cola.LinOp(None, 11, keep=[t])
    assert lib.calls == [("cache", 11, 1)]
    assert leaf.handle == 11 and leaf.handle == 11
    assert [c for c in lib.calls if c[0] == "touch"] == []
    t.add_(1.0)                      # in place: the version counter moves
    assert leaf.handle == 11
    assert [c for c in lib.calls if c[0] == "touch"] == [("touch", 11)]
    assert leaf.handle == 11         # seen: no second touch
    assert len([c for c in lib.calls if c[0] == "touch"]) == 1
    leaf._h = None                   # keep __del__ from calling the library


def test_composite_syncs_its_children(fake):
    cola, lib = fake
    a, b = torch.zeros(3), torch.zeros(5)
    la, lb = cola.LinOp(None, 1, keep=[a]), cola.LinOp(None, 2, keep=[b])
    comp = cola.LinOp(None, 3, children=[la, lb])
    assert ("cache", 3, 1) not in lib.calls  # composites keep no tensors
    b.mul_(2.0)
    assert comp.handle == 3
    assert [c for c in lib.calls if c[0] == "touch"] == [("touch", 2)]
    a.copy_(torch.ones(3))
    b.add_(1.0)
    _ = comp.handle
    assert [c for c in lib.calls if c[0] == "touch"] == [("touch", 2), ("touch", 1), ("touch", 2)]
    for op in (la, lb, comp):
        op._h = None
