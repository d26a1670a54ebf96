"""tcgen05 BF16 GEMM (hh_gemm_bf16 via the C ABI) against float64 matmul of
the same bf16 values: tails in M, N and K, leading dimensions larger than K,
split-K partial products, and the bounded-wait status word."""
import numpy as np
import pytest

from paper_2601_21407_gb300 import hh, inputs as inp

pytestmark = pytest.mark.gpu


def _case(M, N, K, lda, ldb, splits, seed):
    import torch
    rng = np.random.default_rng(seed)
    A = inp.to_bf16_exact(rng.normal(0, 1, (M, K)))
    B = inp.to_bf16_exact(rng.normal(0, 1, (K, N)))
    Ad = torch.zeros((M, lda), dtype=torch.bfloat16, device="cuda")
    Ad[:, :K] = torch.as_tensor(A, device="cuda").to(torch.bfloat16)
    Btd = torch.zeros((N, ldb), dtype=torch.bfloat16, device="cuda")
    Btd[:, :K] = torch.as_tensor(B.T.copy(), device="cuda").to(torch.bfloat16)
    C = torch.full((splits, M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hh.hh_gemm_bf16(Ad, Btd, C, M, N, K, splits=splits, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = C.sum(0).double().cpu().numpy()
    ref = A.astype(np.float64) @ B.astype(np.float64)
    tol = 2e-6 * np.sqrt(K) * 4.0 * 4.0 + 1e-6 * np.abs(ref)
    return got, ref, tol


@pytest.mark.parametrize("M,N,K,lda,ldb,splits", [
    (128, 256, 64, 64, 64, 1),
    (256, 512, 1024, 1024, 1024, 1),
    (200, 96, 700, 704, 704, 1),       # tails in M, N (< one tile) and K (zero-filled)
    (128, 1024, 1024, 1024, 1024, 8),  # the recurrent projection shape, split-K
    (1000, 288, 130, 136, 144, 3),     # uneven splits, padded leading dimensions
])
def test_gemm_matches_float64(M, N, K, lda, ldb, splits):
    got, ref, tol = _case(M, N, K, lda, ldb, splits, seed=M + N + K)
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()


def test_gemm_rejects_bad_shapes():
    import torch
    A = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((1, 128, 40), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(hh.HHError) as e:
        hh.hh_gemm_bf16(A, A, C, 128, 40, 64, status=st)   # N not a multiple of 32
    assert e.value.status == hh.HH_EINVAL


def test_gemm_wait_expiry_reports_status():
    """The pipeline's bounded mbarrier waits, made to run out: with the poll
    limit at 0 every wait gives up at once, the kernel ORs a nonzero code into
    the status word and returns (no TMA copy or MMA in flight, TMEM freed);
    the context stays usable, and with the default limit restored the same
    product is correct."""
    import torch
    M, N, K = 256, 256, 256
    rng = np.random.default_rng(1)
    A = inp.to_bf16_exact(rng.normal(0, 1, (M, K)))
    B = inp.to_bf16_exact(rng.normal(0, 1, (K, N)))
    Ad = torch.as_tensor(A, device="cuda").to(torch.bfloat16)
    Btd = torch.as_tensor(B.T.copy(), device="cuda").to(torch.bfloat16)
    C = torch.zeros((1, M, N), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    try:
        hh.hh_set_wait_limits(mbarrier_polls=0)
        hh.hh_gemm_bf16(Ad, Btd, C, M, N, K, status=st)
        torch.cuda.synchronize()
        code = int(st.item())
    finally:
        hh.hh_set_wait_limits()
    assert code != 0 and (code & 16) == 0, code  # the drain of its own copies did not time out
    st.zero_()
    hh.hh_gemm_bf16(Ad, Btd, C, M, N, K, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = A.astype(np.float64) @ B.astype(np.float64)
    assert np.abs(C[0].double().cpu().numpy() - ref).max() <= 2e-6 * np.sqrt(K) * 16.0 + 1e-6 * np.abs(ref).max()
