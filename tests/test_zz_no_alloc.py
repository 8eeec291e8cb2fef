"""The allocation-free Omega draw (ckinv_omega_noalloc) against the context-based one.

Some callers cannot let a library allocate device memory (a program whose own pool owns
all device memory, or code that must not take an allocation's implicit synchronisation);
the no-allocation entry point serves them from a fixed device array.  It must give the
same signs and columns as ckinv_omega, call after call, since every call reuses that array.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1312_1869_gb300 import ckinv
    return ckinv


@pytest.mark.parametrize("n,d,seed", [(262144, 512, 7), (1000, 48, 3), (1 << 28, 512, 5)])
def test_noalloc_draw_matches_the_context_draw_twice(ck, n, d, seed):
    ctx = ck.Context(0)
    try:
        for call in range(2):
            s = seed + call
            bits_ref, cols_ref = ck.omega(ctx, n, d, s)
            bits, cols = ck.omega_noalloc(n, d, s)
            torch.cuda.synchronize()
            assert np.array_equal(bits.cpu().numpy(), bits_ref.cpu().numpy())
            assert np.array_equal(cols.cpu().numpy(), cols_ref.cpu().numpy())
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(ck):
    with pytest.raises(ck.CKInvError) as e:
        ck.omega_noalloc(4096, 600, 1)
    assert e.value.status == ck.EINVAL
    assert "scratch" in str(e.value)
