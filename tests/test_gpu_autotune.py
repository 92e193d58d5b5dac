"""The autotuner picks an allowed pass split by timing, caches it, and the
transforms stay bit-exact with the oracle under the chosen split."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, batch_inputs
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_autotune_choice_is_cached_and_exact(tmp_path, monkeypatch):
    torch = require_gpu()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("NTT_AUTOTUNE_CACHE", str(cache))
    p, L, batch = P_NTT30, 1 << 15, 8
    o = oracle.get()
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    split = plan.autotune(batch, use_cache=False)
    assert sum(split) == 15 and list(plan.info().log_r)[:len(split)] == split
    data = json.loads(cache.read_text())
    assert any(v == split for v in data.values())
    plan2 = ntt.ntt_plan(p, w, L)
    assert plan2.autotune(batch, use_cache=True) == split  # served from the cache
    a = batch_inputs(31, batch, L, p)
    d = to_dev(a, torch)
    ntt.ntt_forward_batch(plan2, d, batch)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(d, np.uint32).reshape(batch, L).astype(np.uint64),
                          o.ntt_ref(p, w, a.astype(np.uint64)))


def test_uneven_autotune_per_length_class(tmp_path, monkeypatch):
    """Per-class splits for an uneven batch: tuned inside the persistent launch
    on a scratch copy (the batch's data untouched), cached under uneven/ keys,
    served from the cache, and the batch stays exact under the chosen splits
    (including a launch prepared before the splits changed)."""
    from paper_1205_2926_gb300.inputs import uneven_batch_spec, uniform_residues
    torch = require_gpu()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("NTT_AUTOTUNE_CACHE", str(cache))
    o = oracle.get()
    spec = uneven_batch_spec(seed=21, n=300, lmin=10, lmax=16)
    plans, items = {}, []
    for d in spec:
        L = 1 << d["logL"]
        if (d["p"], L) not in plans:
            plans[(d["p"], L)] = ntt.ntt_plan(d["p"], o.root_of_unity(d["p"], L), L)
        a = uniform_residues(5000 + d["id"], L, d["p"]).astype(np.uint32)
        items.append((d, a, to_dev(a, torch)))
    descs = [(plans[(d["p"], 1 << d["logL"])], t, d["inverse"]) for d, _, t in items]
    ntt.ntt_execute_uneven(descs)  # prepared with the default splits
    torch.cuda.synchronize()
    for d, a, t in items:  # restore the inputs
        t.copy_(torch.from_numpy(a.view(np.int32)).cuda())
    before = {k: list(pl.info().log_r)[:pl.info().n_passes] for k, pl in plans.items()}
    ntt.ntt_uneven_autotune(descs, use_cache=False)
    for d, a, t in items:  # the tuner must not have touched the batch's data
        assert np.array_equal(from_dev(t, np.uint32), a), "autotune wrote into the batch"
    data = json.loads(cache.read_text())
    keys = [k for k in data if k.startswith("uneven/")]
    multi = {k: pl for k, pl in plans.items() if k[1] > (1 << 11)}
    lengths = sorted({k[1].bit_length() - 1 for k in multi})
    assert sorted(int(k.split("/l")[1].split("/")[0]) for k in keys) == lengths, keys  # one class per length
    after = {k: list(pl.info().log_r)[:pl.info().n_passes] for k, pl in plans.items()}
    for k, pl in multi.items():
        assert sum(after[k]) == pl.info().log_L
        same_len = [after[j] for j in multi if j[1] == k[1]]
        assert all(s == after[k] for s in same_len), "plans of one length took different splits"
    changed = [k for k in multi if after[k] != before[k]]
    print("uneven splits changed by tuning:", {k[1]: (before[k], after[k]) for k in changed})
    ntt.ntt_execute_uneven(descs)
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    for d, a, t in items:
        L = 1 << d["logL"]
        w = o.root_of_unity(d["p"], L)
        want = (o.intt_ref if d["inverse"] else o.ntt_ref)(d["p"], w, a.astype(np.uint64))
        assert np.array_equal(from_dev(t, np.uint32).astype(np.uint64), want), f"transform {d['id']}"
    # served from the cache: fresh plans get the tuned splits without timing
    fresh = {k: ntt.ntt_plan(k[0], o.root_of_unity(k[0], k[1]), k[1]) for k in plans}
    fdescs = [(fresh[(d["p"], 1 << d["logL"])], t, d["inverse"]) for d, _, t in items]
    ntt.ntt_uneven_autotune(fdescs, use_cache=True)
    for k in multi:
        assert list(fresh[k].info().log_r)[:fresh[k].info().n_passes] == after[k]


def test_autotune_picks_the_row_body(tmp_path, monkeypatch):
    """For a short single-pass transform the tuner also times the row pass's
    body (radix-8 CTA rows against one warp per row), caches the choice under
    the "/warp" key, serves it from the cache, and the transform stays exact."""
    torch = require_gpu()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("NTT_AUTOTUNE_CACHE", str(cache))
    o = oracle.get()
    for logL, batch in ((6, 1), (8, 64)):
        p, L = P_NTT30, 1 << logL
        w = o.root_of_unity(p, L)
        plan = ntt.ntt_plan(p, w, L)
        split = plan.autotune(batch, use_cache=False)
        assert sum(split) == logL
        data = json.loads(cache.read_text())
        wkeys = [k for k in data if k.endswith(f"/l{logL}/b{batch.bit_length() - 1}/warp")]
        assert len(wkeys) == 1 and data[wkeys[0]] in ([0], [1]), data
        plan2 = ntt.ntt_plan(p, w, L)
        assert plan2.autotune(batch, use_cache=True) == split
        a = batch_inputs(41 + logL, batch, L, p)
        d = to_dev(a, torch)
        ntt.ntt_forward_batch(plan2, d, batch)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(d, np.uint32).reshape(batch, L).astype(np.uint64),
                              o.ntt_ref(p, w, a.astype(np.uint64)))
        print(f"L=2^{logL} batch {batch}: split {split}, warp rows chosen = {data[wkeys[0]][0]}")
