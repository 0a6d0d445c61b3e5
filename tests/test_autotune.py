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
    from helpers import assert_forces
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
    assert_forces(f.cpu().numpy(), oracle.celllist(s))


@pytest.mark.gpu
def test_tune_batched_times_the_batched_launch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api
    systems = [synth.water_box(n, 9.86 * (n / 32000) ** (1 / 3), seed=200 + n, rc=1.0, rlist=1.1)
               for n in (1000, 1500, 2500)]
    xs = [torch.tensor(s.x, device="cuda") for s in systems]
    res = autotune.tune_batched(systems, xs, splits=(8, 16, 32), reps=2)
    assert res["split"] in (8, 16, 32)
    assert set(res["split_ms"]) == {8, 16, 32} and all(t > 0 for t in res["split_ms"].values())
    # the tuned split evaluates the batch like the plain contexts do
    ctxs = []
    for s, xr in zip(systems, xs):
        c = api.NbContext.from_system(s)
        c.nb_set_split(res["split"])
        c.build(xr, s.box)
        ctxs.append(c)
    b = api.NbBatch(ctxs)
    xcat = torch.cat(xs).contiguous()
    fcat = torch.empty_like(xcat)
    e = torch.empty(6, dtype=torch.float64, device="cuda")
    b.nb_forces_batched(api.NB_ENERGY, xcat, fcat, e)
    for k, (c, xr) in enumerate(zip(ctxs, xs)):
        f, ek, _ = c.forces(xr, energy=True)
        o = int(b.offsets[k])
        assert torch.allclose(fcat[o:o + len(xr)], f, rtol=0, atol=1e-3)
        assert torch.allclose(e[2 * k:2 * k + 2], ek, rtol=1e-9, atol=0)
