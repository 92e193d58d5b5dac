"""Big-integer products through the transform (Section 1's application):
bigint_mul against the oracle's exact product, limb for limb, for ragged
sizes, maximal carries, zeros and unit factors, up to a 2^22-limb product."""
import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _dev(torch, x):
    return torch.from_numpy(np.asarray(x, dtype=np.uint32).view(np.int32).copy()).cuda()


def _mul(torch, a, b):
    da, db = _dev(torch, a), _dev(torch, b)
    dc = torch.full((len(a) + len(b),), -1, dtype=torch.int32, device="cuda")
    ntt.bigint_mul(da, len(a), db, len(b), dc)
    torch.cuda.synchronize()
    return dc.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("na,nb", [(1, 1), (1, 2), (2, 1), (3, 5), (17, 1000), (1000, 17), (4096, 4096),
                                   (65536, 65535), (100000, 3), (1 << 20, 1 << 20)])
def test_random(na, nb):
    torch = require_gpu()
    rng = np.random.default_rng(na * 7 + nb)
    a = rng.integers(0, 1 << 32, size=na, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 1 << 32, size=nb, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(_mul(torch, a, b), oracle.bigint_mul(a, b))


@pytest.mark.parametrize("n", [1, 5, 4097, 1 << 18])
def test_maximal_carries(n):
    """All limbs 0xFFFFFFFF: every coefficient is at its bound and carries
    ripple through the whole product."""
    torch = require_gpu()
    ones = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    assert np.array_equal(_mul(torch, ones, ones), oracle.bigint_mul(ones, ones))


def test_zero_and_one():
    torch = require_gpu()
    rng = np.random.default_rng(5)
    x = rng.integers(0, 1 << 32, size=3001, dtype=np.uint64).astype(np.uint32)
    assert not _mul(torch, x, np.zeros(7, dtype=np.uint32)).any()
    got = _mul(torch, x, np.array([1], dtype=np.uint32))
    assert np.array_equal(got[:3001], x) and got[3001] == 0


def test_largest_product():
    """na + nb - 1 = 2^23 - 1 limbs: the largest accepted size (coefficients
    near 2^22 (2^32 - 1)^2 < 2^86)."""
    torch = require_gpu()
    rng = np.random.default_rng(6)
    a = rng.integers(0, 1 << 32, size=1 << 22, dtype=np.uint64).astype(np.uint32)
    b = np.full(1 << 22, 0xFFFFFFFF, dtype=np.uint32)
    assert np.array_equal(_mul(torch, a, b), oracle.bigint_mul(a, b))


def test_range_errors():
    """na + nb - 1 > 2^23 is refused (NTT_ERR_RANGE) before anything runs;
    a zero length is an argument error."""
    torch = require_gpu()
    a = _dev(torch, np.ones(1 << 22, dtype=np.uint32))
    b = _dev(torch, np.ones((1 << 22) + 2, dtype=np.uint32))
    c = torch.zeros((1 << 23) + 2, dtype=torch.int32, device="cuda")
    with pytest.raises(ntt.NTTError) as e:
        ntt.bigint_mul(a, 1 << 22, b, (1 << 22) + 2, c)
    assert e.value.code == -9
    with pytest.raises(ntt.NTTError) as e:
        ntt.bigint_mul(a, 0, b, 1, c)
    assert e.value.code == -4
