"""Host logic of the batched launch-plan autotuner (no GPU)."""
import json

import numpy as np
import pytest

from paper_2309_08079_gb300 import autotune as at
from workload import gen


def test_horizon_classes_and_histogram():
    Ns = np.array([1, 2, 3, 32, 33, 64, 65, 512])
    assert at.horizon_classes(Ns) == [1, 2, 4, 32, 64, 128, 512]
    assert at.histogram_key(Ns) == "1:1,2:1,4:1,32:1,64:2,128:1,512:1"
    assert at.histogram_key(np.array([40, 50, 60])) == "64:3"


@pytest.mark.parametrize("Ns", [
    gen.batch_horizons(256, 32, 512, 3),      # the ragged 256-instance workload
    np.array([512] * 9),                       # one class
    np.array([1, 1, 2]),
    np.array([3, 700, 40, 40, 129]),
    gen.batch_horizons(1024, 64, 256, 5),
])
def test_every_plan_covers_every_instance_once_longest_first(Ns):
    plans = at.candidate_plans(Ns)
    assert "single_auto" in plans
    for name, plan in plans.items():
        groups = at.group_instances(Ns, plan)
        idx = np.concatenate([i for _, i in groups])
        assert sorted(idx.tolist()) == list(range(len(Ns))), name
        for g, i in groups:
            assert np.all(np.diff(Ns[i]) <= 0), name        # longest first
            assert np.all((Ns[i] > g["lo"]) & (Ns[i] <= g["hi"])), name
            assert g["mode"] in (0, 1, 2, 3, 4)


def test_group_instances_rejects_overlap_and_gaps():
    Ns = np.array([10, 20, 30])
    with pytest.raises(ValueError):
        at.group_instances(Ns, [{"lo": 0, "hi": 20, "mode": 0, "cluster": 0},
                                {"lo": 10, "hi": 40, "mode": 0, "cluster": 0}])
    with pytest.raises(ValueError):
        at.group_instances(Ns, [{"lo": 0, "hi": 20, "mode": 0, "cluster": 0}])


def test_cache_round_trip(tmp_path):
    path = tmp_path / "sub" / "tune.json"
    t = at.Autotuner(solver=None, cache_path=str(path))
    assert t._load() == {}
    e = {"plan": "classes_auto", "groups": at.candidate_plans(np.array([5, 50]))["classes_auto"],
         "ms": 1.5}
    t._store("k1", e)
    t._store("k2", {"plan": "single_auto", "groups": [], "ms": 2.0})
    d = json.loads(path.read_text())
    assert d["k1"] == e and d["k2"]["plan"] == "single_auto"
    path.write_text("not json")
    assert t._load() == {}


def test_step_plans_give_each_instance_its_own_cluster_size():
    """The 32-knot step plan puts every instance in the group whose upper
    edge is its horizon rounded up to a multiple of 32 (so the launch's
    cluster holds ceil(N / 32) CTAs of 32 knots); the tiled-short variant
    sends horizons up to a quarter of the longest class to the tiled kernel."""
    Ns = gen.batch_horizons(256, 32, 512, 3)
    plans = at.candidate_plans(Ns)
    for g, i in at.group_instances(Ns, plans["steps32_auto"]):
        assert g["hi"] % 32 == 0 and g["hi"] - g["lo"] == 32
        assert np.all(-(-Ns[i] // 32) * 32 == g["hi"])
    groups = at.group_instances(Ns, plans["steps64_tile_short"])
    tiled = [(g, i) for g, i in groups if g["mode"] == 3]
    assert len(tiled) == 1 and tiled[0][0]["hi"] == 128 and np.all(Ns[tiled[0][1]] <= 128)
    assert all(g["mode"] == 0 and g["hi"] - g["lo"] == 64 for g, _ in groups if g["mode"] != 3)
