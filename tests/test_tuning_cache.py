"""The batched form's tuning cache (host side, no GPU): keys, a round trip
through the JSON file, per-GPU separation, and robustness to a damaged or
foreign file.  A stand-in batch object provides the class and tuning calls
of SimSenseBatch."""
import json
import os

import pytest

from paper_2201_11924_gb300 import tuning


def _prm(W, H, D, w, h, paths):
    return {"W": W, "H": H, "D": D, "census_win": w | (h << 8), "P1": 7, "P2": 86, "paths": paths,
            "uniq_ratio": 15, "lr_max_diff": 1}


class FakeBatch:
    device = 0

    def __init__(self, classes):
        self.classes = classes
        self.t = [{"prefetch": 16, "select_blocks": 1} for _ in classes]

    def num_classes(self):
        return len(self.classes)

    def class_info(self, c):
        return self.classes[c], 1

    def get_tuning(self, c):
        return dict(self.t[c])

    def set_tuning(self, c, prefetch, select_blocks):
        self.t[c] = {"prefetch": prefetch, "select_blocks": select_blocks}

    schedule = {"fused": 1, "prefetch": 16, "keep_paths": 1, "lag": 1, "order": 1}

    def get_schedule(self):
        return dict(self.schedule)

    def set_schedule(self, **sc):
        self.schedule = dict(sc)


CLASSES = [_prm(640, 360, 64, 7, 7, 8), _prm(1280, 720, 128, 7, 7, 8), _prm(1920, 1080, 256, 9, 7, 8)]


def test_class_key():
    assert tuning.class_key("GB300", CLASSES[1]) == "GB300|1280x720|D128|census7x7|paths8"
    assert tuning.class_key("GB300", _prm(320, 240, 64, 5, 0, 4)) == "GB300|320x240|D64|census5x5|paths4"


def test_round_trip_applies_the_stored_choices(tmp_path):
    path = str(tmp_path / "tuning.json")
    tuned = FakeBatch(CLASSES)
    tuned.set_tuning(0, 8, 2)
    tuned.set_tuning(2, 12, 1)
    cache = tuning.TuningCache(path)
    assert tuning.store(tuned, cache, gpu="GB300") == 3
    cache.save()
    assert [f for f in os.listdir(tmp_path)] == ["tuning.json"]          # no temporary file left
    fresh = FakeBatch(CLASSES + [_prm(848, 480, 96, 7, 7, 8)])
    missing = tuning.apply(fresh, tuning.TuningCache(path), gpu="GB300")
    assert missing == [3]
    assert fresh.t[:3] == tuned.t


def test_another_gpu_does_not_share_entries(tmp_path):
    path = str(tmp_path / "tuning.json")
    cache = tuning.TuningCache(path)
    b = FakeBatch(CLASSES)
    b.set_tuning(1, 8, 2)
    tuning.store(b, cache, gpu="GB300")
    other = FakeBatch(CLASSES)
    assert tuning.apply(other, cache, gpu="B200") == [0, 1, 2]
    assert other.t == FakeBatch(CLASSES).t


@pytest.mark.parametrize("content", ["{not json", json.dumps({"version": 99, "entries": {}}), json.dumps([1, 2]),
                                     json.dumps({"version": 2, "entries": {"k": {"prefetch": 7, "select_blocks": 1}}}),
                                     json.dumps({"version": 1, "entries": {"k": {"prefetch": 8, "select_blocks": 1}}})])
def test_damaged_or_foreign_files_count_as_empty(tmp_path, content):
    path = tmp_path / "tuning.json"
    path.write_text(content)
    cache = tuning.TuningCache(str(path))
    assert cache.entries == {}
    assert tuning.apply(FakeBatch(CLASSES), cache, gpu="GB300") == [0, 1, 2]
    cache.put("k", {"prefetch": 12, "select_blocks": 2})
    cache.save()
    assert tuning.TuningCache(str(path)).get("k") == {"prefetch": 12, "select_blocks": 2}


def test_only_the_autotuners_choices_are_stored(tmp_path):
    cache = tuning.TuningCache(str(tmp_path / "t.json"))
    with pytest.raises(ValueError):
        cache.put("k", {"prefetch": 10, "select_blocks": 1})


def test_the_batch_schedule_round_trips_per_set_of_classes(tmp_path):
    path = str(tmp_path / "tuning.json")
    tuned = FakeBatch(CLASSES)
    tuned.set_schedule(fused=1, prefetch=16, keep_paths=0, lag=2, order=0)
    cache = tuning.TuningCache(path)
    tuning.store(tuned, cache, gpu="GB300")
    cache.save()
    fresh = FakeBatch(list(reversed(CLASSES)))          # the same classes in another order: the same key
    tuning.apply(fresh, tuning.TuningCache(path), gpu="GB300")
    assert fresh.schedule == tuned.schedule
    other = FakeBatch(CLASSES[:2])                      # other classes: no stored schedule
    tuning.apply(other, tuning.TuningCache(path), gpu="GB300")
    assert other.schedule == FakeBatch.schedule
    with pytest.raises(ValueError):
        cache.put_schedule("k", {"fused": 1, "prefetch": 8, "keep_paths": 0, "lag": 1, "order": 0})
    # a damaged schedule entry counts as absent
    data = json.load(open(path))
    data["schedules"]["bad"] = {"fused": 3}
    json.dump(data, open(path, "w"))
    assert "bad" not in tuning.TuningCache(path).schedules
