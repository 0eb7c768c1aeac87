"""The all-bins autotuner's choices, on the CPU: the library calls are
replaced by a fake whose timings are given, so the test checks only the
tuner's own logic -- coordinate descent, the 1% rule that keeps a choice
against run-to-run noise, the exact path as a bin-tile option, read ranges
tried only when the sample spans several, and the result cache."""
import pytest

torch = pytest.importorskip("torch")


class FakeIndex:
    def __init__(self, f, path):
        self.f, self.path = f, path
        self.threads, self.range_kb, self.switch = 640, 48 << 10, 0
        self.closed = False

    @property
    def desc(self):
        class D:
            pass

        d = D()
        d.cta_threads, d.read_range_kb, d.read_switch = self.threads, self.range_kb, self.switch
        return d

    def close(self):
        self.closed = True


def _patch(monkeypatch, cost):
    """Replace the library calls the tuner makes; cost(index) gives the ms of a
    filter call with the index's current shape."""
    from paper_1708_04329_gb300 import autotune, grim

    built, timed = [], []

    def build_ex(ref, B, q, mrl, layouts, f, all_bins_path=0, **kw):
        built.append((f, all_bins_path))
        return FakeIndex(f, all_bins_path)

    def set_shape(index, cta_threads=0, read_range_kb=0, read_switch=0, all_bins_path=0):
        index.threads = cta_threads or 640
        index.range_kb = read_range_kb or (48 << 10)
        index.switch = read_switch
        index.path = all_bins_path or index.path

    last = {}

    def grim_filter(index, **kw):
        last["ms"] = cost(index)

    def fake_time(fn, repeats):
        fn()
        timed.append(last["ms"])
        return last["ms"]

    monkeypatch.setattr(grim, "grim_build_ex", build_ex)
    monkeypatch.setattr(grim, "grim_index_set_shape", set_shape)
    monkeypatch.setattr(grim, "grim_filter", grim_filter)
    monkeypatch.setattr(grim, "grim_default_coarse_factor", lambda B, q, mrl: 2)
    monkeypatch.setattr(grim, "Workspace", lambda: None)
    monkeypatch.setattr(autotune, "_time", fake_time)
    monkeypatch.setattr(autotune, "_device_name", lambda: "fake GPU")
    return built, timed


REF = torch.zeros(1000, dtype=torch.uint8)  # only its size keys the cache


def _sample(n):
    return {"reads": torch.zeros(1, dtype=torch.uint8), "lens": torch.zeros(n, dtype=torch.int32)}


def test_picks_the_fastest_options_and_keeps_near_ties(monkeypatch):
    from paper_1708_04329_gb300 import autotune, grim

    def cost(ix):
        ms = {2: 100.0, 4: 90.0}[ix.f] if ix.path == grim.GRIM_PATH_TWO_LEVEL else 120.0
        ms *= {512: 0.995, 640: 1.0, 768: 0.95}[ix.threads]  # 512: within 1%, kept out
        ms *= {0: 1.0, 1: 1.1, 2: 1.0}[ix.switch]
        return ms

    built, _ = _patch(monkeypatch, cost)
    out = autotune.tune_all_bins(REF, 200, 5, 100, _sample(500_000), cache=None)
    assert out["factor"] == 4 and out["all_bins_path"] == grim.GRIM_PATH_TWO_LEVEL
    assert out["cta_threads"] == 768          # 5% faster: taken
    assert out["read_switch"] == 0           # the other modes are no better
    assert out["read_range_kb"] == 48 << 10  # every range costs the same: kept
    assert {"f=2", "f=4", "exact", "threads=512", "threads=768", "switch=1", "switch=2"} <= set(out["ms"])
    # the default factor is built first, the exact pass timed on it, then
    # the neighbour; the pick is rebuilt for the shape trials
    assert built[:3] == [(2, 1), (4, 1), (4, 1)]


def test_exact_pass_wins_when_faster(monkeypatch):
    from paper_1708_04329_gb300 import autotune, grim

    def cost(ix):
        return 80.0 if ix.path == grim.GRIM_PATH_EXACT else {2: 100.0, 4: 130.0}[ix.f]

    _patch(monkeypatch, cost)
    out = autotune.tune_all_bins(REF, 200, 5, 250, _sample(100_000), cache=None)
    assert out["all_bins_path"] == grim.GRIM_PATH_EXACT and out["factor"] == 2


def test_small_gains_do_not_move_a_choice(monkeypatch):
    from paper_1708_04329_gb300 import autotune, grim

    def cost(ix):  # every alternative within 0.5% of the default
        base = {2: 100.0, 4: 99.6}[ix.f] if ix.path == grim.GRIM_PATH_TWO_LEVEL else 99.7
        return base * (0.996 if ix.threads == 512 else 1.0)

    _patch(monkeypatch, cost)
    out = autotune.tune_all_bins(REF, 200, 5, 100, _sample(500_000), cache=None)
    assert (out["factor"], out["all_bins_path"], out["cta_threads"]) == (2, grim.GRIM_PATH_TWO_LEVEL, 640)


def test_ranges_only_when_the_sample_spans_several(monkeypatch):
    from paper_1708_04329_gb300 import autotune

    _patch(monkeypatch, lambda ix: 100.0 * (0.9 if ix.range_kb == 12 << 10 else 1.0))
    # 20,000 reads of 100 bp: 20,000 x 96-token rows x 2 B = 3.8 MB, less than
    # every candidate range: none is tried
    out = autotune.tune_all_bins(REF, 200, 5, 100, _sample(20_000), cache=None)
    assert not any(k.startswith("range_kb=") and k != "range_kb=49152" for k in out["ms"])
    assert out["read_range_kb"] == 48 << 10
    # 500,000 reads: 96 MB of token rows; 12, 24 and 48 MB split it
    out = autotune.tune_all_bins(REF, 200, 5, 100, _sample(500_000), cache=None)
    assert {"range_kb=12288", "range_kb=24576"} <= set(out["ms"])
    assert "range_kb=98304" not in out["ms"]
    assert out["read_range_kb"] == 12 << 10


def test_results_are_cached(monkeypatch, tmp_path):
    from paper_1708_04329_gb300 import autotune

    _, timed = _patch(monkeypatch, lambda ix: 100.0)
    cache = tmp_path / "tune.json"
    first = autotune.tune_all_bins(REF, 200, 5, 100, _sample(1000), cache=cache)
    n = len(timed)
    again = autotune.tune_all_bins(REF, 200, 5, 100, _sample(1000), cache=cache)
    assert again == first and len(timed) == n  # nothing timed the second time
