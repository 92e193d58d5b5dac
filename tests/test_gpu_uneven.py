"""One persistent launch over many transforms of uneven lengths, primes and
directions (ntt_execute_uneven): every result equals the oracle's transform of
that vector alone; the launch can be captured in a CUDA graph and replayed;
a wait that cannot be satisfied ends with NTT_ERR_TIMEOUT instead of a hang."""
import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_UNEVEN, P_NTT30, uneven_batch_spec, uniform_residues
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


class Batch:
    def __init__(self, spec, torch, seed=9):
        o = oracle.get()
        self.plans = {}
        self.items = []
        for d in spec:
            L = 1 << d["logL"]
            key = (d["p"], L)
            if key not in self.plans:
                self.plans[key] = ntt.ntt_plan(d["p"], o.root_of_unity(d["p"], L), L)
            a = uniform_residues(seed * 100003 + d["id"], L, d["p"]).astype(np.uint32)
            self.items.append((d, a, to_dev(a, torch)))

    def descs(self):
        return [(self.plans[(d["p"], 1 << d["logL"])], t, d["inverse"]) for d, _, t in self.items]

    def check(self, rounds=1):
        o = oracle.get()
        for d, a, t in self.items:
            L = 1 << d["logL"]
            w = o.root_of_unity(d["p"], L)
            want = a.astype(np.uint64)
            for _ in range(rounds):
                want = o.intt_ref(d["p"], w, want) if d["inverse"] else o.ntt_ref(d["p"], w, want)
            got = from_dev(t, np.uint32).astype(np.uint64)
            assert np.array_equal(got, want), f"transform {d['id']} (L=2^{d['logL']}, p={d['p']}, inv={d['inverse']})"


def test_uneven_small_mix():
    torch = require_gpu()
    spec = uneven_batch_spec(seed=11, n=200, lmin=3, lmax=16)
    b = Batch(spec, torch)
    ntt.ntt_execute_uneven(b.descs())
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    b.check()


@pytest.mark.parametrize("variant", [0, 1])
def test_uneven_full_workload_4096(variant):
    """4096 transforms, L = 2^8..2^16 log-uniform, three 30-bit primes, half
    inverse; lazy (Algorithms 3-4) and NTL-style (Algorithm 2) butterflies."""
    torch = require_gpu()
    spec = uneven_batch_spec()
    b = Batch(spec, torch)
    for pl in b.plans.values():
        pl.set_variant(variant)
    ntt.ntt_execute_uneven(b.descs())
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    b.check()


def test_uneven_graph_capture_and_replay():
    torch = require_gpu()
    spec = uneven_batch_spec(seed=12, n=120, lmin=8, lmax=15)
    b = Batch(spec, torch)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ntt.ntt_execute_uneven(b.descs(), stream=s)  # warm-up: prepares and uploads the batch
    torch.cuda.synchronize()
    b.check(rounds=1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ntt.ntt_execute_uneven(b.descs(), stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    b.check(rounds=3)


def test_two_batches_in_two_graphs_stay_valid():
    """Preparing a second batch keeps the first one's work list: graphs captured
    on either replay correctly in any order; ntt_uneven_release frees both."""
    torch = require_gpu()
    b1 = Batch(uneven_batch_spec(seed=31, n=60, lmin=8, lmax=14), torch, seed=31)
    b2 = Batch(uneven_batch_spec(seed=32, n=70, lmin=9, lmax=16), torch, seed=32)
    s = torch.cuda.Stream()
    graphs = []
    for b in (b1, b2):
        with torch.cuda.stream(s):
            ntt.ntt_execute_uneven(b.descs(), stream=s)  # prepares this batch (outside any capture)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ntt.ntt_execute_uneven(b.descs(), stream=s)
        graphs.append(g)
    g1, g2 = graphs
    g1.replay()
    g2.replay()
    g1.replay()
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    b1.check(rounds=3)
    b2.check(rounds=2)
    del g1, g2, graphs
    ntt.ntt_uneven_release()
    b3 = Batch(uneven_batch_spec(seed=33, n=40, lmin=8, lmax=13), torch, seed=33)
    ntt.ntt_execute_uneven(b3.descs())
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    b3.check()


def test_uneven_wait_times_out_with_status():
    """A dependency that never completes: the bounded wait gives up, the launch
    ends, the status says NTT_ERR_TIMEOUT and the context stays usable."""
    torch = require_gpu()
    spec = [{"id": 0, "logL": 16, "p": P_UNEVEN[0], "inverse": False},
            {"id": 1, "logL": 14, "p": P_UNEVEN[1], "inverse": True}]
    b = Batch(spec, torch)
    try:
        ntt.ntt_uneven_set_wait_budget(20_000_000, stall_stage=1)  # ~10 ms
        ntt.ntt_execute_uneven(b.descs())
        torch.cuda.synchronize()
        assert ntt.ntt_uneven_status() == -7
    finally:
        ntt.ntt_uneven_set_wait_budget(2_000_000_000, stall_stage=-1)
    b2 = Batch(spec, torch, seed=10)
    ntt.ntt_execute_uneven(b2.descs())
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    b2.check()


def test_uneven_rejects_unsupported():
    torch = require_gpu()
    from paper_1205_2926_gb300.inputs import P_NTT62
    o = oracle.get()
    plan64 = ntt.ntt_plan(P_NTT62, o.root_of_unity(P_NTT62, 1024), 1024)
    t = torch.zeros(2048, dtype=torch.int64, device="cuda")
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_execute_uneven([(plan64, t, False)])
    assert e.value.code == -9
    plan = ntt.ntt_plan(P_NTT30, o.root_of_unity(P_NTT30, 1024), 1024)
    t32 = torch.zeros(2048, dtype=torch.int32, device="cuda")
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_execute_uneven([(plan, t32.data_ptr() + 4, False)])
    assert e.value.code == -8


def test_uneven_ntl_variant_and_variant_rules():
    """The persistent launch with the NTL-style butterflies (Algorithm 2): the
    same results as the oracle, including rows of p - 1 (the top of its input
    interval [0, p)); a batch mixing variants is refused (NTT_ERR_ARG), and the
    Montgomery variant is not carried (NTT_ERR_RANGE)."""
    torch = require_gpu()
    spec = uneven_batch_spec(seed=13, n=300, lmin=3, lmax=16)
    b = Batch(spec, torch, seed=17)
    for i, (d, a, t) in enumerate(b.items):
        if i % 5 == 0:  # top of Algorithm 2's interval
            a[:] = d["p"] - 1
            t.copy_(torch.from_numpy(a.view(np.int32)).cuda())
    for pl in b.plans.values():
        pl.set_variant(ntt.VARIANT_NTL)
    ntt.ntt_execute_uneven(b.descs())
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    b.check()
    plans = list(b.plans.values())
    plans[0].set_variant(ntt.VARIANT_LAZY)
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_execute_uneven(b.descs())
    assert e.value.code == -4
    for pl in plans:
        pl.set_variant(ntt.VARIANT_MONT)
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_execute_uneven(b.descs())
    assert e.value.code == -9
    for pl in plans:
        pl.set_variant(ntt.VARIANT_LAZY)
