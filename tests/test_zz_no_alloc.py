"""Resampling without allocation, for callers that cannot allocate device
memory while they run (for example a control loop that must not block in the
CUDA allocator, or an application whose device memory belongs to another
allocator).  Its output must equal the allocating entry point's, call after
call, although every call reuses the same library-owned scratch array.

This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import scenarios as S
from gpu_helpers import cuda

pytestmark = pytest.mark.gpu


def test_noalloc_resample_matches_workspace_entry_point_on_consecutive_calls():
    torch = cuda()
    import paper_1506_02869_gb300 as pkg

    rng = np.random.default_rng(4242)
    # call 1: large, with an all-zero segment (degenerate status);
    # call 2: smaller and clean -- it must not see call 1's flag or partial sums
    cases = [(8, 65536, 31, 2, 5, True), (3, 5000, 77, 9, 1, False)]
    for nseg, L, seed, J, mpc, degenerate in cases:
        w = S.random_wtilde(nseg, L, rng)
        if degenerate:
            w[2] = 0.0
        wt = torch.from_numpy(w).cuda()
        ref, st_ref = pkg.resample(wt, seed, 0, J, mpc)
        got = torch.full((nseg, L), -7, dtype=torch.int32, device="cuda")
        st = pkg.tma_resample_noalloc(wt, seed, 0, J, mpc, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        assert st == st_ref == (pkg.TMA_WARN_DEGENERATE if degenerate else pkg.TMA_OK)


def test_noalloc_resample_rejects_sizes_beyond_its_scratch():
    torch = cuda()
    import paper_1506_02869_gb300 as pkg

    lib = pkg.lib()
    dummy = C.c_void_p(16)      # never dereferenced: the size check comes first
    st = lib.tma_resample_noalloc(dummy, 33, 1 << 22, 1, 0, 0, 0, dummy, None)
    assert st == pkg.TMA_ERR_INVALID_ARG
    # the largest allowed shape (32 x 2048 chunks = 65536 partial sums) works
    w = torch.rand((32, 1 << 22), dtype=torch.float64, device="cuda")
    anc = torch.empty((32, 1 << 22), dtype=torch.int32, device="cuda")
    ref, _ = pkg.resample(w, 5, 0, 0, 0)
    assert pkg.tma_resample_noalloc(w, 5, 0, 0, 0, anc) == pkg.TMA_OK
    assert torch.equal(anc, ref)
