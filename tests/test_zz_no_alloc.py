"""sf_rotate_noalloc: the rotation for callers that cannot allocate device
memory (fixed scratch compiled into the library).  Checked against sf_rotate
through the C ABI on two calls in a row, bit for bit (integer residues), and
for its size limit.  Collected last so that a failure here does not hide the
rest of the suite."""
import numpy as np
import pytest
import torch

import paper_2509_01253_gb300 as sf
from paper_2509_01253_gb300 import workloads as wl

from _gpu import Session, dev_zeros, from_dev

pytestmark = pytest.mark.gpu


def test_rotate_noalloc_matches_rotate_twice():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    ps = wl.PARAMS["conv16"]
    s = Session.from_set(ps, sk_seed=71, rk_seed=72, rot_d=[3, 9, 16385])
    try:
        rng = np.random.default_rng(73)
        for call, (d, count) in enumerate([(3, 3), (16385, 2)]):
            msg = rng.integers(-2 ** 40, 2 ** 40, count * s.n)
            d_ct = s.encrypt(msg, 74 + call, count)
            want = dev_zeros(count, 2, s.L, s.n)
            got = dev_zeros(count, 2, s.L, s.n)
            sf.sf_rotate(s.ctx, s.rk, d, d_ct, want, count)
            sf.sf_rotate_noalloc(s.ctx, s.rk, d, d_ct, got, count)
            sf.sf_sync(s.ctx)
            assert (from_dev(got) == from_dev(want)).all(), (call, d)
        # more ciphertexts than the context's launch batch: both calls split the
        # key switches into the same launch batches
        sf.sf_ctx_set_option(s.ctx, "ks_batch", 1)
        msg = rng.integers(-2 ** 40, 2 ** 40, 3 * s.n)
        d_ct = s.encrypt(msg, 80, 3)
        want = dev_zeros(3, 2, s.L, s.n)
        got = dev_zeros(3, 2, s.L, s.n)
        sf.sf_rotate(s.ctx, s.rk, 9, d_ct, want, 3)
        sf.sf_rotate_noalloc(s.ctx, s.rk, 9, d_ct, got, 3)
        sf.sf_sync(s.ctx)
        assert (from_dev(got) == from_dev(want)).all()
        sf.sf_ctx_set_option(s.ctx, "ks_batch", 512)
        # the property the entry point exists for: with the array's address
        # looked up (first call above), a call changes the device's free memory
        # by nothing, even with per-launch timing switched on (which the call
        # suspends rather than creating events), and leaves that option as it was
        sf.sf_ctx_set_option(s.ctx, "kernel_timing", 1)
        out7 = dev_zeros(7, 2, s.L, s.n)
        in7 = s.encrypt(rng.integers(-2 ** 40, 2 ** 40, 7 * s.n), 81, 7)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        sf.sf_rotate_noalloc(s.ctx, s.rk, 3, in7, out7, 7)
        sf.sf_sync(s.ctx)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert sf.sf_ctx_get_option(s.ctx, "kernel_timing") == 1
        sf.sf_ctx_set_option(s.ctx, "kernel_timing", 0)
        # beyond the fixed scratch: rejected with a clear error, nothing launched
        big = dev_zeros(8, 2, s.L, s.n)
        with pytest.raises(sf.SafhireError) as e:
            sf.sf_rotate_noalloc(s.ctx, s.rk, 3, big, big.clone(), 8)
        assert e.value.status == sf.SF_EINVAL and "fixed maximum" in e.value.message
        sf.sf_sync(s.ctx)
    finally:
        s.close()
