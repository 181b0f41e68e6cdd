"""sstep_block_gram_noalloc: block Gram products for callers that cannot allocate device
memory at call time (their framework holds the device's memory in its own pool, or they must
not pay for the allocator).  Checked through the C ABI against sstep_block_gram on the same
inputs, twice in a row so that the second call proves the shared scratch area is re-armed.

The file name sorts last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2603_09790_gb300 import sstep

pytestmark = pytest.mark.gpu


def test_noalloc_matches_block_gram_twice():
    dev = torch.device("cuda:0")
    n = 300007
    rng = np.random.default_rng(42)
    nl, nr = 9, 11
    L = [torch.from_numpy(rng.standard_normal(n)).to(dev) for _ in range(nl)]
    R = [torch.from_numpy(rng.standard_normal(n)).to(dev) for _ in range(nr)]
    pairs = [(i, j) for i in range(nl) for j in range(nr) if (i + 2 * j) % 3 != 1]
    ref = torch.zeros(len(pairs), dtype=torch.float64, device=dev)
    sstep.block_gram(L, R, pairs, ref)
    torch.cuda.synchronize()
    norms = [(float(L[i].norm()), float(R[j].norm())) for i, j in pairs]
    for call in range(2):
        out = torch.full((len(pairs),), float("nan"), dtype=torch.float64, device=dev)
        sstep.block_gram_noalloc(L, R, pairs, out)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        for e, (nli, nrj) in enumerate(norms):
            bound = 1e-14 * np.sqrt(n) * nli * nrj
            assert abs(got[e] - want[e]) <= bound, (call, e, got[e], want[e])


def test_noalloc_rejects_too_many_products():
    dev = torch.device("cuda:0")
    v = [torch.ones(1000, dtype=torch.float64, device=dev) for _ in range(17)]
    pairs = [(i, j) for i in range(17) for j in range(17)][:257]
    out = torch.zeros(257, dtype=torch.float64, device=dev)
    with pytest.raises(sstep.SstepError) as e:
        sstep.block_gram_noalloc(v, v, pairs, out)
    assert e.value.status == sstep.ERR_INVALID and "256" in str(e.value)
