"""Host logic of the autotuner (no GPU): the candidate lists it walks and its cache key.

Sec. 4 and Sec. 6: the best coarsening shape and work size are found by timing candidates, per
number of polarizations and GCF size, and remembered. The candidates must cover every schedule
the library offers, with plan arguments the C ABI accepts, and a cached result tuned over other
candidates must not be reused.
"""
import pytest

from paper_1605_07023_gb300 import autotune


def test_grid_candidates_cover_the_gridding_schedules():
    """By default the chunked, sorted and lazy schedules; the patch schedule (about 5x slower on GB300)
    only when asked for."""
    c = list(autotune._candidates("grid"))
    assert {x["schedule"] for x in c} == {"chunked", "sorted", "lazy"}
    c_all = list(autotune._candidates("grid", ("chunked", "sorted", "patch", "lazy")))
    assert {x["schedule"] for x in c_all} == {"chunked", "sorted", "patch", "lazy"}
    for x in c_all:
        assert x["vis_per_chunk"] > 0
        if x["schedule"] == "lazy":
            assert (x["Bu"], x["Bv"]) in autotune.LAZY_SHAPES and x["threads"] % 32 == 0
        else:
            assert (x["Bu"], x["Bv"]) in autotune.BLOCK_CANDIDATES
        if x["schedule"] in ("chunked", "sorted"):
            assert x["threads"] in autotune.CTA_THREADS
    # Sec. 6: near-square shapes are the ones worth trying; the list stays within 4:1
    for bu, bv in autotune.BLOCK_CANDIDATES:
        assert max(bu, bv) <= 4 * min(bu, bv)


def test_degrid_candidates_include_the_tile_schedule_in_whole_warps():
    c = list(autotune._candidates("degrid"))
    scheds = {x["schedule"] for x in c}
    assert scheds == {"chunked", "tile"}
    tiles = [x for x in c if x["schedule"] == "tile"]
    assert sorted((x["threads"], x["tile_group"]) for x in tiles) == sorted(
        (t, g) for t in autotune.TILE_THREADS for g in autotune.TILE_GROUPS)
    assert set(autotune.TILE_GROUPS) == {32, 8}
    assert all(x["threads"] % 32 == 0 and 32 <= x["threads"] <= 1024 for x in tiles)
    # no duplicate candidates
    keys = [tuple(sorted(x.items())) for x in c]
    assert len(keys) == len(set(keys))


def test_plan_kwargs_pass_every_field():
    cfg = dict(schedule="tile", Bu=2, Bv=2, vis_per_chunk=0, threads=64)
    kw = autotune.plan_kwargs(cfg)
    assert kw == dict(Bu=2, Bv=2, schedule="tile", vis_per_chunk=0, threads=64, precision="f32", bin_u=0, bin_v=0,
                      tile_group=0)
    assert autotune.plan_kwargs(dict(cfg, tile_group=8))["tile_group"] == 8
    kw = autotune.plan_kwargs(dict(schedule="lazy", Bu=4, Bv=2, vis_per_chunk=512, threads=128, bin_u=12, bin_v=10))
    assert (kw["schedule"], kw["bin_u"], kw["bin_v"]) == ("lazy", 12, 10)


def test_cache_key_depends_on_problem_and_candidates(monkeypatch):
    pytest.importorskip("torch")
    k1 = autotune._key("both", 2048, 7, 8, 4, "f32")
    assert k1 != autotune._key("both", 2048, 7, 8, 1, "f32")
    assert k1 != autotune._key("both", 2048, 9, 8, 4, "f32")
    assert k1 != autotune._key("both", 2048, 7, 8, 4, "bf16")
    monkeypatch.setattr(autotune, "TILE_THREADS", (256,))
    assert autotune._key("both", 2048, 7, 8, 4, "f32") != k1


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("GB300_GRIDDER_CACHE", str(tmp_path / "sub" / "tune.json"))
    assert autotune.load_cache() == {}
    autotune.save_cache({"k": {"grid": {"Bu": 2}}})
    assert autotune.load_cache() == {"k": {"grid": {"Bu": 2}}}
    (tmp_path / "sub" / "tune.json").write_text("not json")
    assert autotune.load_cache() == {}
