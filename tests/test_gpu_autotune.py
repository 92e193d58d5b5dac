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
