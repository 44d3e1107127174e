"""Autotuner logic on a fake target (no GPU): coordinate descent, the
same-count guard, the cache table."""
import pytest

from paper_2403_02997_gb300 import autotune


class FakeTarget:
    """ms_total falls as hash_chunk approaches 4096 and edges_per_item 256."""

    def __init__(self, count=42, cheat=None):
        self.p = {}
        self.count_value = count
        self.cheat = cheat

    def set_params(self, **kw):
        self.p = dict(kw)

    def count(self, roots):
        if self.cheat and all(self.p.get(k) == v for k, v in self.cheat.items()):
            return self.count_value + 1
        return self.count_value

    def stats(self):
        ms = 100.0 + abs(self.p.get("hash_chunk", 8192) - 4096) / 100.0
        ms += abs(self.p.get("edges_per_item", 512) - 256) / 10.0
        return {"ms_total": ms}


@pytest.fixture(autouse=True)
def defaults(monkeypatch):
    import paper_2403_02997_gb300 as tc
    monkeypatch.setattr(tc, "tc_params_default",
                        lambda: dict(small_max_degree=32, medium_max_degree=0, hash_chunk=8192,
                                     edges_per_item=512,
                                     bfs_alpha=15, bfs_beta=18, sorted_lookup=0))


def test_descent_finds_the_minimum(tmp_path):
    t = FakeTarget()
    res = autotune.tune(t, 0, trials=1)
    assert res["params"]["hash_chunk"] == 4096 and res["params"]["edges_per_item"] == 256
    assert res["ms"] < res["default_ms"]
    assert t.p == res["params"]          # the target is left on the best parameters
    path = str(tmp_path / "cache.json")
    sig = autotune.signature(1 << 20, 1 << 24, 5000, "rmat")
    autotune.store(sig, res, path)
    assert autotune.lookup(sig, path) == res["params"]
    assert autotune.lookup("missing", path) is None


def test_a_changed_count_is_an_error():
    t = FakeTarget(cheat={"hash_chunk": 4096})
    with pytest.raises(RuntimeError):
        autotune.tune(t, 0, trials=1)
