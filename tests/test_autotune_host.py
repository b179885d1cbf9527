"""Host logic of the batched engine's tile autotuner (no GPU): table loading, per-instance
choices with the size-rule fallback, and the consistency of the committed table."""
import json

from paper_2307_00391_gb300 import autotune


def test_missing_or_corrupt_table_means_no_choices(tmp_path):
    assert autotune.load_table(str(tmp_path / "absent.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert autotune.load_table(str(bad)) == {}
    assert autotune.choices_for([(6, 8)], table={}) is None


def test_choices_follow_the_table_and_fall_back_per_size():
    table = {"6,8": {"best": 0, "ms": {"0": 1.0, "128": 2.0}},
             "9,10": {"best": 256, "ms": {"128": 3.0, "256": 2.5}}}
    assert autotune.choices_for([(6, 8), (9, 10), (7, 8)], table=table) == [0, 256, -1]


def test_committed_table_covers_the_batch_sizes_and_keeps_each_fastest_choice():
    table = autotune.load_table()
    assert table, "tuning.json is missing"
    for n_s in range(6, 13):
        for n_c in range(8, 13):
            ent = table[f"{n_s},{n_c}"]
            assert ent["best"] in (0, 128, 256)
            ms = {int(k): v for k, v in ent["ms"].items()}
            assert ent["best"] == min(ms, key=ms.get)
    json.dumps(table)
