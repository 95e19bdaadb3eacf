"""Tensor-core GEMM (tcgen05, BF16 x BF16 -> FP32) against numpy on the same
BF16-rounded operands (the accumulation order differs only in FP32 rounding)."""
import numpy as np
import pytest

import oracle.precond_net as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as B
    return torch, B


@pytest.mark.parametrize("M,K,Ncol,ta,tb,acc", [
    (128, 16, 32, False, False, False),
    (300, 48, 64, False, False, False),
    (128, 128, 128, False, False, False),
    (1000, 300, 32, False, False, False),   # K split over three CTAs, atomic epilogue
    (257, 64, 96, True, False, False),      # A read transposed
    (200, 64, 64, False, True, False),      # B read transposed
    (130, 40, 64, True, True, True),        # both transposed, accumulate into C
])
def test_tc_gemm_matches_numpy(env, M, K, Ncol, ta, tb, acc):
    torch, B = env
    rng = np.random.default_rng(M + K + Ncol)
    A = rng.normal(size=(M, K)).astype(np.float32)
    Bm = rng.normal(size=(K, Ncol)).astype(np.float32)
    C0 = rng.normal(size=(M, Ncol)).astype(np.float32) if acc else np.zeros((M, Ncol), np.float32)
    ref = N.bf16_round(A) @ N.bf16_round(Bm) + (C0.astype(np.float64) if acc else 0.0)
    dev = torch.device("cuda")
    if ta:
        dA = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)   # stored K x M
        a_rs, a_cs = 1, M
    else:
        dA = torch.from_numpy(A).to(dev)
        a_rs, a_cs = K, 1
    if tb:
        dB = torch.from_numpy(np.ascontiguousarray(Bm.T)).to(dev)  # stored N x K
        b_rs, b_cs = 1, K
    else:
        dB = torch.from_numpy(Bm).to(dev)
        b_rs, b_cs = Ncol, 1
    dC = torch.from_numpy(C0.copy()).to(dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    B.ba_tc_gemm(M, Ncol, K, dA.data_ptr(), a_rs, a_cs, dB.data_ptr(), b_rs, b_cs, dC.data_ptr(), Ncol, 1,
                 accumulate=acc, err=err.data_ptr(), stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = dC.cpu().numpy().astype(np.float64)
    scale = np.abs(N.bf16_round(A)) @ np.abs(N.bf16_round(Bm))
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-5 * np.abs(ref) + 1e-6), np.abs(got - ref).max()
