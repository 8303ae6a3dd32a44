"""qcd_norm2_noalloc against qcd_spinor_norm2, through the C ABI.

qcd_norm2_noalloc is for callers that cannot allocate device memory (a
framework that owns all of it, or a path that cannot afford cudaMalloc's
device synchronisation): its reduction scratch is a static device array
inside the library.  Here it must agree with the allocating entry point on
the same field, on two calls in a row (the second call reuses the scratch
the first one left behind).  This file is collected last on purpose.
"""

import numpy as np
import pytest

from paper_1411_5219_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return qcd


@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (24, 24, 24, 8)])
def test_norm2_noalloc_matches_norm2(q, dims):
    import torch
    lat = q.Lattice(dims, -1)
    s = q.Spinor(lat, "full", "f64", torch_alloc=True)
    psi = syn.gaussian_spinor(dims, 4242)
    s.upload(psi)
    want = s.norm2()  # the allocating entry point (lattice reduction scratch)
    data = s._buffers[0]
    n = data.numel() // 8  # doubles, padding sites are zero
    res = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for k in range(2):
        q.norm2_noalloc(data.data_ptr(), n, res[k:].data_ptr())
    q.stream_sync()
    got = res.cpu().numpy()
    ref = float(np.vdot(psi, psi).real)
    for v in got:
        assert abs(v - want) <= 1e-12 * want
        assert abs(v - ref) <= 1e-12 * ref
    assert got[0] == got[1]  # same inputs, fixed summation order


def test_norm2_noalloc_edges(q):
    import torch
    res = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    x = torch.arange(1, 4, dtype=torch.float64, device="cuda")
    q.norm2_noalloc(x.data_ptr(), 3, res.data_ptr())
    q.stream_sync()
    assert res.item() == 14.0
    q.norm2_noalloc(x.data_ptr(), 0, res.data_ptr())
    q.stream_sync()
    assert res.item() == 0.0
    with pytest.raises(q.QcdError) as e:
        q.norm2_noalloc(x.data_ptr(), q.NORM2_NOALLOC_MAX + 1, res.data_ptr())
    assert e.value.status == 1 and "exceeds the maximum" in str(e.value)


def test_norm2_noalloc_at_the_limit_and_block_edges(q):
    """The largest accepted size (every partial-sum slot in use, the ticket
    counter right after the last one) and sizes one element either side of a
    block boundary, against a sum of squares in FP64 on the device; around
    repeated calls the free device memory does not change."""
    import torch
    per_block = 256 * 8
    res = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    n_max = q.NORM2_NOALLOC_MAX
    gen = torch.Generator(device="cuda")
    gen.manual_seed(99)
    x = torch.rand(n_max, dtype=torch.float64, device="cuda", generator=gen) - 0.5
    sizes = (n_max, n_max - 1, 3 * per_block - 1, 3 * per_block, 3 * per_block + 1, 1)
    wants = [float(torch.dot(x[:n], x[:n]).item()) for n in sizes]
    q.norm2_noalloc(x.data_ptr(), n_max, res.data_ptr())  # first use of the entry point (module set-up)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n, want in zip(sizes, wants):
        for _ in range(2):
            q.norm2_noalloc(x.data_ptr(), n, res.data_ptr())
            q.stream_sync()
            assert abs(res.item() - want) <= 1e-12 * want, n
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
