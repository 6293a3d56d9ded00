"""The MLP field's tensor-core building block (tcgen05.mma, BF16 x BF16 ->
FP32 in tensor memory, core-matrix operand layout) against a plain FP32
product of the same BF16 values."""
import ctypes as C

import pytest
import torch

from paper_2210_12375_b300 import _abi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K", [(16, 16), (32, 48), (128, 48), (128, 128), (32, 128),
                                 (256, 64), (64, 256)])
def test_tc_gemm_matches_fp32_product(N, K):
    lib = _abi.load()
    g = torch.Generator(device="cpu").manual_seed(N * 1000 + K)
    A = torch.randn(128, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    Cm = torch.full((128, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.tode_tc_gemm(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                          C.c_void_p(Cm.data_ptr()), 128, N, K, 0, C.c_void_p(err.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    ref = A.double() @ B.double().T
    assert torch.isfinite(Cm).all()
    assert (Cm.double() - ref).abs().max().item() <= 1e-5 * max(1.0, ref.abs().max().item())


def test_tc_gemm_rejects_bad_shapes():
    lib = _abi.load()
    p = C.c_void_p(0x1000)
    for (M, N, K) in [(32, 16, 16), (128, 8, 16), (128, 16, 8), (128, 272, 16)]:
        assert lib.tode_tc_gemm(p, p, p, M, N, K, 0, p, None) == _abi.TODE_EINVAL
    assert lib.tode_tc_gemm(p, p, p, 128, 16, 16, 8, p, None) == _abi.TODE_EINVAL


@pytest.mark.parametrize("flags", [5, 6, 7])
@pytest.mark.parametrize("N", [32, 48, 128, 144])
def test_tc_gemm_mn_major_operands(flags, N):
    """Transposed (MN-major) operands, as the adjoint's weight-gradient GEMMs
    use them: A given as [K][M] (flags bit 0) and/or B as [K][N] (bit 1),
    with the stride fields the primitives use (bit 2)."""
    lib = _abi.load()
    K = 128
    g = torch.Generator(device="cpu").manual_seed(flags * 100 + N)
    A = torch.randn(128, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    Ain = (A.T.contiguous() if flags & 1 else A).cuda()
    Bin = (B.T.contiguous() if flags & 2 else B).cuda()
    Cm = torch.full((128, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.tode_tc_gemm(C.c_void_p(Ain.data_ptr()), C.c_void_p(Bin.data_ptr()),
                          C.c_void_p(Cm.data_ptr()), 128, N, K, flags, C.c_void_p(err.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    ref = (A.double() @ B.double().T).cuda()
    assert (Cm.double() - ref).abs().max().item() <= 1e-5 * max(1.0, ref.abs().max().item())


@pytest.mark.parametrize("N", [64, 128, 256])
def test_tc_gemm_m64_accumulator_lanes(N):
    """M = 64 tiles: every one of the 64 result rows appears exactly in one
    tensor-memory lane; the lane of row m is (m // 16) * 32 + m % 16 (16 rows
    in each warp's lane quarter), the map the 64-row MLP tile relies on."""
    lib = _abi.load()
    K = 64
    g = torch.Generator(device="cpu").manual_seed(64 + N)
    A = torch.randn(64, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    Cm = torch.full((128, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.tode_tc_gemm(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                          C.c_void_p(Cm.data_ptr()), 64, N, K, 0, C.c_void_p(err.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    ref = (A.double() @ B.double().T).cpu()
    dump = Cm.double().cpu()
    tol = 1e-5 * max(1.0, ref.abs().max().item())
    lanes = {}
    for m in range(64):
        hit = [ln for ln in range(128) if (dump[ln] - ref[m]).abs().max().item() <= tol]
        lanes[m] = hit
    assert all(len(v) == 1 for v in lanes.values()), lanes
    assert [lanes[m][0] for m in range(64)] == [(m // 16) * 32 + m % 16 for m in range(64)]


def test_tc_gemm_m64_half_split_load():
    """The 16x32bx2 load on an M = 64 accumulator: thread t < 16 of warp w gets
    row 16w + t at columns [0, 16), thread t >= 16 row 16w + t - 16 at
    columns [32, 48) -- every thread of the warp carries a useful row."""
    lib = _abi.load()
    N, K = 64, 64
    g = torch.Generator(device="cpu").manual_seed(4242)
    A = torch.randn(64, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    Cm = torch.full((128, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.tode_tc_gemm(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                          C.c_void_p(Cm.data_ptr()), 64, N, K, 8, C.c_void_p(err.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    ref = (A.double() @ B.double().T).cpu()
    got = Cm.double().cpu()[:, :16]
    exp = torch.empty(128, 16, dtype=torch.float64)
    for w in range(4):
        for t in range(32):
            row = 16 * w + (t % 16)
            c0 = 0 if t < 16 else 32
            exp[32 * w + t] = ref[row, c0:c0 + 16]
    assert (got - exp).abs().max().item() <= 1e-5 * max(1.0, ref.abs().max().item())


@pytest.mark.parametrize("N", [80, 128, 144])
def test_tc_gemm_m64_mn_major_b(N):
    """M = 64 tiles with an MN-major B operand ([K][N] tile), the shape of the
    wide adjoint's transposed-weight products."""
    lib = _abi.load()
    K = 64
    g = torch.Generator(device="cpu").manual_seed(6400 + N)
    A = torch.randn(64, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    Cm = torch.full((128, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ad, Bd = A.cuda(), B.T.contiguous().cuda()
    rc = lib.tode_tc_gemm(C.c_void_p(Ad.data_ptr()), C.c_void_p(Bd.data_ptr()),
                          C.c_void_p(Cm.data_ptr()), 64, N, K, 6, C.c_void_p(err.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    ref = (A.double() @ B.double().T)
    rows = [(m // 16) * 32 + m % 16 for m in range(64)]
    got = Cm.double().cpu()[rows]
    assert (got - ref).abs().max().item() <= 1e-5 * max(1.0, ref.abs().max().item())
