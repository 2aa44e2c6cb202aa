"""Host logic of the autotuners (no GPU): the stages, the pick, the cache.
The timings are stand-ins keyed on the configuration, so the test checks
which candidates are timed and which one is kept, not GPU behaviour."""
import pytest

from paper_2303_02471_gb300 import autotune
from paper_2303_02471_gb300.ops import Config


def _fake_times(table, calls):
    """A timing function over a dict of config -> ms (by the knobs named in
    the table's keys); unknown configurations take 10 ms, a None entry
    raises like an unsupported configuration."""
    def timed(cfg):
        conf = {k: getattr(cfg, k) for k in ("t", "hash_cta_max", "cta_threads", "small_accumulator",
                                             "table_slots_pct", "group_promote")}
        calls.append(conf)
        for key, ms in table:
            if all(conf.get(k) == v for k, v in key):
                if ms is None:
                    raise RuntimeError("unsupported")
                return ms
        return 10.0
    return timed


GRID = {"t": [33, 65], "hash_cta_max": [2048], "cta_threads": [128, 256],
        "table_slots_pct": [150, 250], "group_promote": [0, 1]}


def test_batch_tuner_stages_pick_and_cache(tmp_path, monkeypatch):
    calls = []
    table = [((("t", 65), ("cta_threads", 256), ("table_slots_pct", 250), ("group_promote", 0)), 3.0),
             ((("t", 65), ("cta_threads", 256)), 5.0),
             ((("t", 33), ("cta_threads", 128)), None)]
    timed = _fake_times(table, calls)
    monkeypatch.setattr(autotune, "_time", lambda As, Bs, cfg, repeats: timed(cfg))
    monkeypatch.setattr(autotune, "signature", lambda As, Bs: "sig")
    cache = str(tmp_path / "tune.json")
    cfg, rep = autotune.tune([], [], grid=GRID, cache=cache)
    # the grid (4 candidates) then the three non-default refine combinations
    assert len(calls) == 4 + 3
    assert [c["table_slots_pct"] for c in calls[:4]] == [None] * 4
    assert all(c["t"] == 65 and c["cta_threads"] == 256 for c in calls[4:])
    assert cfg == Config(t=65, hash_cta_max=2048, cta_threads=256, table_slots_pct=250, group_promote=0)
    assert rep["ms"] == 3.0
    err = [r for r in rep["candidates"] if r["error"]]
    assert len(err) == 1 and err[0]["config"]["t"] == 33 and err[0]["ms"] == float("inf")
    # cached: no timing on the second call, the same pick
    calls.clear()
    cfg2, _ = autotune.tune([], [], grid=GRID, cache=cache)
    assert not calls and cfg2 == cfg
    # refresh times again
    autotune.tune([], [], grid=GRID, cache=cache, refresh=True)
    assert len(calls) == 7


def test_batch_tuner_spells_out_the_defaults_it_kept(tmp_path, monkeypatch):
    calls = []
    timed = _fake_times([((("t", 33), ("cta_threads", 128), ("table_slots_pct", None)), 1.0)], calls)
    monkeypatch.setattr(autotune, "_time", lambda As, Bs, cfg, repeats: timed(cfg))
    monkeypatch.setattr(autotune, "signature", lambda As, Bs: "sig")
    cfg, rep = autotune.tune([], [], grid=GRID, cache=str(tmp_path / "t.json"))
    assert cfg.t == 33 and cfg.cta_threads == 128
    assert cfg.table_slots_pct == 150 and cfg.group_promote == 0  # the first values, written out
    assert rep["config"]["table_slots_pct"] == 150


def test_batch_tuner_fails_when_nothing_runs(tmp_path, monkeypatch):
    def boom(As, Bs, cfg, repeats):
        raise RuntimeError("unsupported")
    monkeypatch.setattr(autotune, "_time", boom)
    monkeypatch.setattr(autotune, "signature", lambda As, Bs: "sig")
    with pytest.raises(RuntimeError):
        autotune.tune([], [], grid=GRID, cache=str(tmp_path / "t.json"))


@pytest.mark.parametrize("single_ms, form", [(2.0, "single_pass"), (9.0, "two_pass")])
def test_product_tuner_form_stage(tmp_path, monkeypatch, single_ms, form):
    calls, sp = [], []
    grid = {"t": [129, 257], "small_accumulator": ["hash", "esc"], "table_slots_pct": [150, 250],
            "group_promote": [0, 1], "form": autotune.FORMS}
    timed = _fake_times([((("t", 257), ("small_accumulator", "esc")), 4.0)], calls)
    monkeypatch.setattr(autotune, "_time_product", lambda A, B, cfg, repeats: timed(cfg))

    def single(A, B, cfg, repeats):
        sp.append(cfg)
        return single_ms
    monkeypatch.setattr(autotune, "_time_single_pass", single)
    monkeypatch.setattr(autotune, "product_signature", lambda A, B: "psig")
    cfg, rep = autotune.tune_product(None, None, grid=grid, cache=str(tmp_path / "p.json"))
    assert len(calls) == 4 + 3
    # the single pass is timed once, with the pick's configuration
    assert len(sp) == 1 and sp[0].t == 257 and sp[0].small_accumulator == "esc"
    assert cfg.t == 257 and cfg.small_accumulator == "esc"
    assert rep["form"] == form
    assert rep["ms"] == min(4.0, single_ms)
    assert rep["candidates"][-1]["config"]["form"] == "single_pass"


def test_product_tuner_without_forms_keeps_two_passes(tmp_path, monkeypatch):
    calls = []
    monkeypatch.setattr(autotune, "_time_product", lambda A, B, cfg, repeats: _fake_times([], calls)(cfg))
    monkeypatch.setattr(autotune, "_time_single_pass",
                        lambda *a: pytest.fail("the single pass is not in the grid"))
    monkeypatch.setattr(autotune, "product_signature", lambda A, B: "psig")
    cfg, rep = autotune.tune_product(None, None, grid={"t": [129]}, cache=str(tmp_path / "p.json"))
    assert len(calls) == 1 and rep["form"] == "two_pass" and cfg.t == 129


def test_cache_path_follows_xdg(monkeypatch, tmp_path):
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    assert autotune._cache_path(None) == str(tmp_path / "spgemm_gb300" / "autotune.json")
    assert autotune._cache_path("x.json") == "x.json"
