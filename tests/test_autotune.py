"""Autotuner: selection logic and cache on CPU; a tuned configuration on the GPU."""
import json

import numpy as np
import pytest

from paper_2006_09167_gb300 import autotune, synth


def test_choose_split_prefers_fastest_then_larger():
    assert autotune.choose_split({16: 1.0, 32: 0.8, 64: 0.9}) == 32
    assert autotune.choose_split({16: 0.8, 32: 0.8}) == 32
    with pytest.raises(ValueError):
        autotune.choose_split({})


def test_choose_parts_requires_no_missed_pairs():
    missed = {1: 0, 2: 0, 4: 3, 8: 10}
    step = {1: 0.5, 2: 0.45, 4: 0.40, 8: 0.38}
    assert autotune.choose_parts(missed, step) == 2
    assert autotune.choose_parts({1: 2, 2: 5}, {1: 0.5, 2: 0.4}) == 1


def test_cache_roundtrip(tmp_path):
    s = synth.water_648()
    k1 = autotune.config_key(s, "GB300")
    k2 = autotune.config_key(synth.water_box(216, 1.9, seed=1, coulomb=0, rc=0.9, rlist=1.0), "GB300")
    assert k1 != k2 and k1.startswith("GB300:")
    path = str(tmp_path / "tune.json")
    autotune.save_cache(path, {k1: {"split": 48, "n_parts": 2}})
    assert autotune.load_cache(path)[k1]["split"] == 48
    assert json.load(open(path))[k1]["n_parts"] == 2


@pytest.mark.gpu
def test_tune_on_gpu_gives_a_valid_correct_configuration(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2006_09167_gb300 import api
    from helpers import TOL_F, rms_rel
    s = synth.water_box(3375, 4.66, seed=91, rc=1.0, rlist=1.1, r_in=1.03)
    x = torch.tensor(s.x, device="cuda")
    v = torch.tensor(synth.maxwell_boltzmann(s, 300.0, seed=1), dtype=torch.float32, device="cuda")
    res = autotune.tune(s, x, v, nstlist=40, reps=3, cache_path=str(tmp_path / "c.json"))
    assert res["split"] in autotune.SPLITS
    assert res["n_parts"] in autotune.PARTS
    assert res["missed"][res["n_parts"]] == 0 or res["n_parts"] == 1
    # the cache answers the second call
    assert autotune.tune(s, x, v, cache_path=str(tmp_path / "c.json"))["split"] == res["split"]
    ctx = api.NbContext.from_system(s)
    ctx.nb_set_split(res["split"])
    ctx.build(x, s.box)
    f, e, w = ctx.forces(x, energy=True, virial=True)
    assert rms_rel(f.cpu().numpy(), oracle.celllist(s)["F"]) < TOL_F
