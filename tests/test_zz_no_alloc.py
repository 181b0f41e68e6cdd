"""sstep_block_gram_noalloc: block Gram products for callers that cannot allocate device
memory at call time (their framework holds the device's memory in its own pool, or they must
not pay for the allocator).  Checked through the C ABI:

* bit for bit against sstep_block_gram on the same inputs (same kernel, same launch), twice in
  a row so that the second call proves the shared scratch area is re-armed;
* against the FP64 oracle's X^T Y at the rounding bound the other Gram tests use;
* that it takes nothing from the device's current memory pool (the pool cudaMallocAsync draws
  on, which sstep_block_gram uses), read through the driver API before and after the call.

The file name sorts last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_09790_gb300 import sstep

pytestmark = pytest.mark.gpu

USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # CUmemPool_attribute values (cuda.h)


class _Pool:
    """The current memory pool of device 0, through libcuda (the driver API)."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        self.pool = ctypes.c_void_p()
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0


def _inputs(n, nl, nr, seed):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(seed)
    Lh = [rng.standard_normal(n) for _ in range(nl)]
    Rh = [rng.standard_normal(n) for _ in range(nr)]
    L = [torch.from_numpy(v).to(dev) for v in Lh]
    R = [torch.from_numpy(v).to(dev) for v in Rh]
    pairs = [(i, j) for i in range(nl) for j in range(nr) if (i + 2 * j) % 3 != 1]
    return Lh, Rh, L, R, pairs


def test_noalloc_matches_block_gram_and_oracle_twice():
    n, nl, nr = 300007, 9, 11
    Lh, Rh, L, R, pairs = _inputs(n, nl, nr, 42)
    dev = L[0].device
    ref = torch.zeros(len(pairs), dtype=torch.float64, device=dev)
    sstep.block_gram(L, R, pairs, ref)
    torch.cuda.synchronize()
    G = O.gram(np.array(Lh), np.array(Rh))
    for call in range(2):
        out = torch.full((len(pairs),), float("nan"), dtype=torch.float64, device=dev)
        sstep.block_gram_noalloc(L, R, pairs, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (call, (out - ref).abs().max().item())
        got = out.cpu().numpy()
        for e, (i, j) in enumerate(pairs):
            bound = 1e-14 * np.sqrt(n) * np.linalg.norm(Lh[i]) * np.linalg.norm(Rh[j])
            assert abs(got[e] - G[i, j]) <= bound, (call, e, got[e], G[i, j])


def test_noalloc_takes_nothing_from_the_memory_pool():
    n, nl, nr = 1 << 20, 4, 5
    _, _, L, R, pairs = _inputs(n, nl, nr, 7)
    dev = L[0].device
    out = torch.zeros(len(pairs), dtype=torch.float64, device=dev)
    sstep.block_gram_noalloc(L, R, pairs, out)  # first call on the device: address set-up
    torch.cuda.synchronize()
    pool = _Pool()
    for _ in range(2):
        torch.cuda.synchronize()
        used0 = pool.get(USED_MEM_CURRENT)
        pool.reset_high()
        sstep.block_gram_noalloc(L, R, pairs, out)
        torch.cuda.synchronize()
        assert pool.get(USED_MEM_CURRENT) == used0
        assert pool.get(USED_MEM_HIGH) <= used0, "block_gram_noalloc drew on the memory pool"
    # the allocating entry point, for contrast: its per-call scratch shows in the high mark
    used0 = pool.get(USED_MEM_CURRENT)
    pool.reset_high()
    sstep.block_gram(L, R, pairs, out)
    torch.cuda.synchronize()
    assert pool.get(USED_MEM_HIGH) > used0


def test_noalloc_rejects_too_many_products():
    dev = torch.device("cuda:0")
    v = [torch.ones(1000, dtype=torch.float64, device=dev) for _ in range(17)]
    pairs = [(i, j) for i in range(17) for j in range(17)][:257]
    out = torch.zeros(257, dtype=torch.float64, device=dev)
    with pytest.raises(sstep.SstepError) as e:
        sstep.block_gram_noalloc(v, v, pairs, out)
    assert e.value.status == sstep.ERR_INVALID and "256" in str(e.value)
