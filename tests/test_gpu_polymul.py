"""polymul_mod_p through the C ABI against the oracle's schoolbook product
(small sizes) and its convolution-theorem product (large sizes)."""
import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, P_UNEVEN, uniform_residues, word_dtype
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def gpu_polymul(p, a, b, torch):
    dt = word_dtype(p)
    da, db = to_dev(a.astype(dt), torch), to_dev(b.astype(dt), torch)
    n = a.size + b.size - 1
    dc = torch.zeros(n, dtype=torch.int32 if dt == np.uint32 else torch.int64, device="cuda")
    ntt.polymul_mod_p(p, da, a.size, db, b.size, dc)
    torch.cuda.synchronize()
    return from_dev(dc, dt)


@pytest.mark.parametrize("p", [P_NTT30, P_UNEVEN[1], P_NTT62])
@pytest.mark.parametrize("na,nb", [(1, 1), (1, 2), (2, 1), (3, 5), (8, 9), (64, 65), (100, 1), (257, 300),
                                   (1000, 999), (2049, 31)])
def test_polymul_small(p, na, nb):
    torch = require_gpu()
    a = uniform_residues(na * 7 + 1, na, p)
    b = uniform_residues(nb * 11 + 2, nb, p)
    got = gpu_polymul(p, a, b, torch)
    want = oracle.get().polymul_schoolbook(p, a, b)
    assert np.array_equal(got.astype(np.uint64), want)


@pytest.mark.parametrize("p,na,nb", [(P_NTT30, (1 << 20) + 1, (1 << 20) + 1), (P_NTT30, 70000, 3),
                                     (P_NTT62, 1 << 19, (1 << 19) + 7)])
def test_polymul_large(p, na, nb):
    torch = require_gpu()
    a = uniform_residues(na, na, p)
    b = uniform_residues(nb + 5, nb, p)
    got = gpu_polymul(p, a, b, torch)
    want = oracle.get().polymul_ntt(p, a, b)
    assert np.array_equal(got.astype(np.uint64), want)


def test_polymul_errors():
    torch = require_gpu()
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(ntt.NTTError) as e:
        ntt.polymul_mod_p(P_NTT30, d, 0, d, 4, d)
    assert e.value.code == -4
    with pytest.raises(ntt.NTTError) as e:
        ntt.polymul_mod_p(P_NTT30 + 2, d, 4, d, 4, d)
    assert e.value.code == -1
    with pytest.raises(ntt.NTTError) as e:  # needs L = 2^17 but 2^17 does not divide p-1
        ntt.polymul_mod_p(P_UNEVEN[1], d, 1 << 16, d, 1 << 16, d)
    assert e.value.code == -2
