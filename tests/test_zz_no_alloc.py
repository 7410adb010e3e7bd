"""cng_entry_noalloc: the navigating node computed with a fixed device array instead of
allocations, for callers that cannot allocate device memory (memory owned by another
allocator or budgeted at start-up, latency-bound loops).  Its result must equal the navigating node cng_build
reports for the same points; consecutive calls on different inputs check that no state of an
earlier call leaks into the next.  Kept in a file collected last."""
import numpy as np
import pytest
import torch

from paper_2510_05975_gb300 import synth

from gpu_util import lib, need_gpu, tensor

pytestmark = pytest.mark.gpu


def _reference_entry(cng, X):
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=8, L=16, connect_L=-1)
    _, _, _, entry = cng.cng_graph(idx)
    cng.cng_free(idx)
    assert entry == st["entry"]
    return entry


def test_entry_noalloc_matches_build_on_consecutive_calls():
    need_gpu()
    cng = lib()
    A = synth.generate("gauss", 20000, 48, seed=31)
    B = synth.generate("sift", 9000, 128, seed=32)
    ref_a, ref_b = _reference_entry(cng, A), _reference_entry(cng, B)
    assert ref_a != ref_b
    out = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    for X, ref in ((A, ref_a), (B, ref_b), (A, ref_a)):
        out.fill_(-7)
        cng.cng_entry_noalloc(tensor(X), out)
        torch.cuda.synchronize()
        assert int(out.item()) == ref


def test_entry_noalloc_fp16_and_limits():
    need_gpu()
    cng = lib()
    H = synth.generate("bigann16", 5000, 64, seed=33, dtype="float16")
    assert H.dtype == np.float16
    ref = _reference_entry(cng, H)
    out = torch.empty((1,), dtype=torch.int32, device="cuda")
    cng.cng_entry_noalloc(tensor(H), out)
    torch.cuda.synchronize()
    assert int(out.item()) == ref
    # a shape needing more scratch than the fixed array is rejected before any device access
    rc = cng.lib().cng_entry_noalloc(out.data_ptr(), cng.CNG_F32, 4096 * 5000, 128, out.data_ptr(), None)
    assert rc == cng.CNG_E_INVAL
    assert "exceeds the fixed scratch" in cng.cng_last_error()
