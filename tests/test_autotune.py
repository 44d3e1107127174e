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


class FakeGraph:
    """count(): the cover-edge count, count_forward(): the forward count, with given times."""

    def __init__(self, ms_cetc, ms_fwd, num_cover=300, m=1000, tri=7, fwd_tri=7):
        self.ms_cetc, self.ms_fwd, self.num_cover, self.m = ms_cetc, ms_fwd, num_cover, m
        self.tri, self.fwd_tri, self.last = tri, fwd_tri, 0.0

    def count(self, root):
        self.last = self.ms_cetc
        return self.tri

    def count_forward(self):
        self.last = self.ms_fwd
        return self.fwd_tri

    def stats(self):
        return {"ms_total": self.last, "num_cover": self.num_cover}


def test_fe_threshold_follows_the_faster_count(tmp_path):
    fast_fwd = autotune.learn_fe_threshold(FakeGraph(10.0, 6.0), 0, trials=1)
    assert fast_fwd["forward_faster"] and fast_fwd["threshold"] < 0.3      # c = 0.3 switches
    slow_fwd = autotune.learn_fe_threshold(FakeGraph(6.0, 10.0), 0, trials=1)
    assert not slow_fwd["forward_faster"] and slow_fwd["threshold"] > 0.3  # c = 0.3 stays
    path = str(tmp_path / "cache.json")
    autotune.store_fe("rmat:n24", fast_fwd, path)
    autotune.store("rmat:n24", {"params": {"hash_chunk": 4096}, "ms": 1.0, "default_ms": 2.0}, path)
    assert autotune.lookup_fe("rmat:n24", path) == fast_fwd["threshold"]   # both kept
    assert autotune.lookup("rmat:n24", path) == {"hash_chunk": 4096}
    assert autotune.lookup_fe("missing", path) is None
    with pytest.raises(RuntimeError):                                    # counts must agree
        autotune.learn_fe_threshold(FakeGraph(10.0, 6.0, fwd_tri=8), 0, trials=1)


class JointTarget(FakeTarget):
    """Faster only with 1024-thread blocks, 12288-entry chunks and 4096-edge items together."""

    def stats(self):
        shape = (self.p.get("hash_block"), self.p.get("hash_chunk"), self.p.get("edges_per_item"))
        return {"ms_total": 80.0 if shape == (1024, 12288, 4096) else 100.0 + (shape[0] == 1024)}


def test_shape_move_reaches_a_joint_optimum(monkeypatch):
    import paper_2403_02997_gb300 as tc
    monkeypatch.setattr(tc, "tc_params_default",
                        lambda: dict(small_max_degree=32, medium_max_degree=0, hash_block=512,
                                     hash_chunk=8192, edges_per_item=512, bfs_alpha=15,
                                     bfs_beta=18))
    res = autotune.tune(JointTarget(), 0, trials=1)
    p = res["params"]
    assert (p["hash_block"], p["hash_chunk"], p["edges_per_item"]) == (1024, 12288, 4096)
    # without the joint moves, single-coordinate steps never leave the default shape
    res = autotune.tune(JointTarget(), 0, trials=1, grid=autotune.GRID)
    assert res["params"]["hash_block"] == 512 and res["ms"] == 100.0
