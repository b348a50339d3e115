"""The JSON form of a cell configuration (host logic, no GPU)."""
import json

import pytest

from paper_2609_15043_b300 import workloads


def test_round_trip_and_overrides(tmp_path):
    cfg = workloads.cell60().replace(see_gamma=0.1, sm_every=50, sm_target=200, sm_min=100, sm_max=400)
    assert workloads.load_config(workloads.dump_config(cfg)) == cfg
    path = tmp_path / "cell.json"
    path.write_text(json.dumps({"workload": "cell100", "p_target": 80, "turn_r": [0.03, 0.06], "winding": [1, -1],
                                "implicit_es": 1}))
    c = workloads.load_config(str(path))
    assert (c.nr, c.nz, c.p_target, c.turn_r, c.winding, c.implicit_es) == (256, 384, 80.0, [0.03, 0.06], [1, -1], 1)
    assert isinstance(c.p_target, float) and isinstance(c.implicit_es, int)


def test_unknown_and_mistyped_keys_are_refused():
    with pytest.raises(KeyError):
        workloads.load_config({"n_r": 64})
    with pytest.raises(TypeError):
        workloads.load_config({"nr": "64"})
    with pytest.raises(TypeError):
        workloads.load_config({"turn_r": 0.05})
    with pytest.raises(KeyError):
        workloads.load_config({"workload": "cell7"})
