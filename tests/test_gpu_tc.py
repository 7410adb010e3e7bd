"""The tensor-core screen (tcgen05 MMA + TMA + TMEM epilogue) computes, for every (row x,
column y), s = ||y_b||^2 - 2 <x_b, y_b> with x_b, y_b the bf16-rounded vectors.  Compared here
with the same arithmetic in FP64 on the host: equal within the FP32 accumulation bound, and
exactly equal for small integers (every product and partial sum is an exact FP32 integer)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_05975_gb300 import synth

from gpu_util import lib, need_gpu, tensor

pytestmark = pytest.mark.gpu


def _bf16(x):
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def _scores(cng, R, C):
    L = cng.lib()
    L.cngx_tc_scores.restype = ctypes.c_int
    L.cngx_tc_scores.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    rd, cd = tensor(R), tensor(C)
    out = torch.full((R.shape[0], C.shape[0]), float("nan"), device="cuda")
    rc = L.cngx_tc_scores(rd.data_ptr(), R.shape[0], cd.data_ptr(), C.shape[0], R.shape[1],
                          out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, cng.cng_last_error()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,n,d", [(256, 128, 64), (300, 517, 100), (513, 1000, 128), (64, 300, 32),
                                   (257, 129, 192),
                                   # wider rows: A and B streamed together in 64-wide K chunks
                                   (300, 517, 200), (257, 389, 960), (40, 1000, 4000)])
def test_tc_scores_match_reference(m, n, d):
    need_gpu()
    cng = lib()
    R = synth.generate("gauss", m, d, seed=1)
    C = synth.generate("gauss", n, d, seed=2)
    got = _scores(cng, R, C)
    rb, cb = _bf16(R), _bf16(C)
    ref = (cb * cb).sum(1)[None, :] - 2.0 * rb @ cb.T
    bound = (d + 16) * 2.0 ** -22 * ((np.abs(rb) @ np.abs(cb).T) * 2 + (cb * cb).sum(1)[None, :])
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound + 1e-6), float((err / (bound + 1e-30)).max())


def test_tc_scores_exact_on_integers():
    need_gpu()
    cng = lib()
    R = synth.generate("sift", 300, 128, seed=3)
    C = synth.generate("sift", 700, 128, seed=4)
    got = _scores(cng, R, C)
    ref = (C.astype(np.float64) ** 2).sum(1)[None, :] - 2.0 * R.astype(np.float64) @ C.astype(np.float64).T
    assert np.array_equal(got, ref)


def _scores_f16(cng, R, C, scale):
    L = cng.lib()
    L.cngx_tc_scores_f16.restype = ctypes.c_int
    L.cngx_tc_scores_f16.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int32, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
    rd, cd = tensor(R), tensor(C)
    out = torch.full((R.shape[0], C.shape[0]), float("nan"), device="cuda")
    rc = L.cngx_tc_scores_f16(rd.data_ptr(), R.shape[0], cd.data_ptr(), C.shape[0], R.shape[1], scale,
                              out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, cng.cng_last_error()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("kind,m,n,d,scale", [("deep", 300, 517, 96, 8192.0), ("gauss", 257, 129, 192, 2048.0),
                                              ("gist", 200, 300, 160, 1024.0), ("gist", 300, 700, 960, 1024.0)])
def test_tc_scores_fp16_scaled(kind, m, n, d, scale):
    """FP16 operands fp16(scale x) as the build uses them for float data: scores equal the FP64
    arithmetic on the same rounded operands within the FP32 accumulation bound."""
    need_gpu()
    cng = lib()
    R = synth.generate(kind, m, d, seed=1)
    C = synth.generate(kind, n, d, seed=2)
    got = _scores_f16(cng, R, C, scale)
    rh = (R.astype(np.float32) * np.float32(scale)).astype(np.float16).astype(np.float64)
    ch = (C.astype(np.float32) * np.float32(scale)).astype(np.float16).astype(np.float64)
    ref = (ch * ch).sum(1)[None, :] - 2.0 * rh @ ch.T
    bound = (d + 16) * 2.0 ** -22 * ((np.abs(rh) @ np.abs(ch).T) * 2 + (ch * ch).sum(1)[None, :])
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= bound + 1e-6)
    # the scaled FP16 operands are 8x closer to the data than BF16 ones
    rb = _bf16(R) * scale
    assert np.abs(rh - R * scale).max() < np.abs(rb - R * scale).max()


def test_bounded_waits_expire_without_fault():
    """The screen's bounded waits (an mbarrier nothing arrives on, a flag nothing sets) run out,
    record the timeout bit and return; the context stays usable for a screen afterwards."""
    need_gpu()
    cng = lib()
    st = cng.cngx_wait_probe()
    assert st & 1 and not st & 8
    import oracle
    A = synth.generate("sift", 600, 64, seed=31)
    ids, _, _ = cng.cng_knn(tensor(A), 5)
    gt, _ = oracle.knn(A, 5)
    assert np.array_equal(ids.cpu().numpy(), gt)
