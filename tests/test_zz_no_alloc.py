"""The allocation-free norm (jfnk_norm2_noalloc) against the context's norm
(jfnk_norm2), through the C ABI.  It exists for callers that must not allocate
device memory: code running during a CUDA graph capture, allocator callbacks,
services with a device-memory budget fixed at start-up.  Collected last so a
run that stops at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

import synth
from tests._common import gpu_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_norm2_noalloc_matches_context_norm_on_consecutive_calls():
    from paper_2505_24504_gb300 import jfnk
    ctx = gpu_context(synth.scaled(synth.BUBBLE_Q2_20x10, 10, 5))
    sizes = (0, 1, 255, 8192, 8193, 819_200, 3_000_001)
    for call in range(2):           # the shared scratch keeps the last call's contents
        for n, seed in zip(sizes, range(10, 20)):
            x = torch.from_numpy(synth.random_vector(max(n, 1), seed + 7 * call)).cuda()
            got = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            ref = torch.full((1,), -2.0, dtype=torch.float64, device="cuda")
            jfnk.norm2_noalloc(x, got, n=n)
            ctx.norm2(x, ref, n=n)
            torch.cuda.synchronize()
            r = ref.item()
            assert abs(got.item() - r) <= 1e-14 * max(r, 1.0), (call, n, got.item(), r)


def test_norm2_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2505_24504_gb300 import jfnk
    lib = jfnk.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_big = 4096 * 8192 + 1
    rc = lib.jfnk_norm2_noalloc(ctypes.c_void_p(x.data_ptr()), too_big, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert np.isfinite(out.item())
