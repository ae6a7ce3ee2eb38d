"""Host logic of the collide+stream launch-shape autotuner: candidate timing
per (nx, storage) class, the JSON cache, and the batch-wide choice.  No GPU."""
import json

from paper_2408_15115_gb300 import autotune as AT


class FakeRun:
    def __init__(self, name):
        self.name = name


def _runs():
    a, b, c = FakeRun("a"), FakeRun("b"), FakeRun("c")
    return [AT.RunInfo(64, "f32", 64 ** 3, a), AT.RunInfo(96, "f16", 96 * 96 * 192, b),
            AT.RunInfo(64, "f32", 64 ** 3, c)]


def _timer_table(calls):
    # us per launch: 256-thread blocks are best for nx = 64 FP32, 128 for nx = 96 FP16,
    # by a margin that makes (128, 3) the better batch-wide block size
    def timer(handle, threads, tx, minb):
        calls.append((handle.name, threads, tx, minb))
        if handle.name == "b":
            base = 400.0 if (threads, minb) == (128, 2) else 480.0
            return base - (10.0 if tx == 64 else 0.0)
        base = 40.0 if (threads, minb) == (256, 3) else 44.0
        return base - (1.0 if tx == 128 else 0.0)
    return timer


def test_one_timing_per_class_and_candidate(tmp_path):
    calls = []
    ch = AT.tune(_runs(), _timer_table(calls), cache_path=str(tmp_path / "c.json"), device_name="dev")
    # runs a and c share a class: only a is timed
    assert {c[0] for c in calls} == {"a", "b"}
    assert len(calls) == 2 * len(AT.CANDIDATES)


def test_batch_wide_choice_minimises_weighted_time(tmp_path):
    calls = []
    ch = AT.tune(_runs(), _timer_table(calls), cache_path=str(tmp_path / "c.json"), device_name="dev")
    # weighted: b dominates (1.77M cells), so (128, 2) wins over a's favourite (256, 3)
    assert (ch.threads, ch.minb) == (128, 2)
    assert ch.tx == [128, 64, 128]
    # predicted time = sum over runs of the chosen candidates' us
    assert abs(ch.predicted_us - (43.0 + 390.0 + 43.0)) < 1e-9


def test_cache_round_trip_and_device_separation(tmp_path):
    path = str(tmp_path / "c.json")
    calls = []
    ch1 = AT.tune(_runs(), _timer_table(calls), cache_path=path, device_name="dev")
    n1 = len(calls)
    ch2 = AT.tune(_runs(), _timer_table(calls), cache_path=path, device_name="dev")
    assert len(calls) == n1 and ch2 == ch1
    data = json.load(open(path))
    assert data["version"] == AT.CACHE_VERSION
    assert set(data["devices"]["dev"]) == {"k1/nx=64/f32", "k1/nx=96/f16"}
    # timings are stored per million cells
    v = data["devices"]["dev"]["k1/nx=64/f32"][AT.cand_key(256, 128, 3)]
    assert abs(v - 39.0 * 1e6 / 64 ** 3) < 1e-9
    AT.tune(_runs(), _timer_table(calls), cache_path=path, device_name="other")
    assert len(calls) == 2 * n1


def test_stale_cache_version_is_ignored(tmp_path):
    path = tmp_path / "c.json"
    path.write_text(json.dumps({"version": -1, "devices": {"dev": {"k1/nx=64/f32": {}}}}))
    calls = []
    AT.tune(_runs(), _timer_table(calls), cache_path=str(path), device_name="dev")
    assert len(calls) == 2 * len(AT.CANDIDATES)


def test_no_cache_path_times_every_call():
    calls = []
    AT.tune(_runs()[:1], _timer_table(calls))
    AT.tune(_runs()[:1], _timer_table(calls))
    assert len(calls) == 2 * len(AT.CANDIDATES)
