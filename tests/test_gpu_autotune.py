"""The autotuner (lwacm_autotune): measures every candidate configuration, keeps
the fastest, records it in a JSON cache that later contexts of the same problem
read instead of measuring, and leaves the context ready for set_fields."""
import json

import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_2142_gb300 import lwacm
    return lwacm


def ensemble(n, seed):
    rng = np.random.default_rng(seed)
    dims = [(int(rng.integers(8, 90)), int(rng.integers(8, 90))) for _ in range(n)]
    nus = [float(rng.uniform(0.005, 0.05)) for _ in range(n)]
    fields = [inputs.smooth_random((d[1], d[0]), seed=seed + b, u_amp=0.04, d_amp=0.01) for b, d in enumerate(dims)]
    return dims, nus, fields


def test_batch_autotune_measures_caches_and_reuses(lw, tmp_path):
    cache = tmp_path / "tune.json"
    dims, nus, fields = ensemble(24, seed=3)
    sim = lw.LwacmBatch(lw.D2Q9, dims, nus)
    rep = sim.autotune(cache=cache, steps=64)
    assert rep["source"] == "measured" and rep["cache_written"]
    cands = rep["candidates"]
    assert len(cands) == 14  # 7 tile layouts x 2 launch forms
    best = min(cands, key=lambda c: c["us_per_step"])
    assert (rep["choice"]["tile"], rep["choice"]["mode"]) == (best["tile"], best["mode"])
    assert sim.kernel_name == rep["choice"]["name"] == best["name"]
    text = cache.read_text()
    assert rep["key"] in text
    json.loads(text)  # the cache is valid JSON
    # the tuned context computes the method
    sim.set_domains(fields)
    sim.step(30)
    got = sim.get_domains()
    for b in (0, 7, 23):
        ref = oracle.step(9, *fields[b], nu=nus[b], nsteps=30)
        eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[b][1:], ref[1:])) / 0.04
        assert eu < 1e-5
    with pytest.raises(lw.LwacmError) as ei:
        sim.autotune(cache=cache)  # fields are set now
    assert ei.value.status == lw.E_STATE
    sim.close()
    # same problem: the cache answers, nothing is timed
    again = lw.LwacmBatch(lw.D2Q9, dims, nus)
    rep2 = again.autotune(cache=cache, steps=64)
    assert rep2["source"] == "cache" and rep2["candidates"] == []
    assert rep2["choice"]["name"] == rep["choice"]["name"] == again.kernel_name
    again.close()
    # another problem adds its own entry
    other = lw.LwacmBatch(lw.D2Q9, dims[:5], nus[:5])
    rep3 = other.autotune(cache=cache, steps=32)
    assert rep3["source"] == "measured"
    entries = json.loads(cache.read_text())
    assert rep["key"] in entries and rep3["key"] in entries
    other.close()


def test_single_domain_autotune_and_unreadable_cache(lw, tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("this is not a cache\n")
    sim = lw.Lwacm(lw.D3Q19, 256, 16, 8, 0.01)
    rep = sim.autotune(cache=cache, steps=32)
    assert rep["source"] == "measured"
    names = sorted(c["name"] for c in rep["candidates"])
    assert any(n.startswith("half") for n in names) and any(n.startswith("generic") for n in names)
    print("single-domain candidates:", [(c["name"], round(c["us_per_step"], 2)) for c in rep["candidates"]])
    f = inputs.smooth_random((8, 16, 256), seed=4, u_amp=0.03, d_amp=0.01)
    sim.set_fields(*f)
    sim.step(12)
    got = sim.get_fields()
    ref = oracle.step(19, *f, nu=0.01, nsteps=12)
    eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], ref[1:])) / 0.03
    assert eu < 1e-5
    assert rep["key"] in json.loads(cache.read_text())
    sim.close()
