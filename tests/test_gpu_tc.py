"""The tcgen05 dense-layer kernel as a plain GEMM (BF16 operands, FP32 accumulation in
tensor memory) against float64 products of the same BF16 values."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14051_gb300 import build, nis
    build.build()
    c = nis.Context(0)
    yield c
    c.close()


# (m, n, k, lda pad): ragged rows, partial K tiles, N from 3 (MMA N 16) to 208
SHAPES = [(128, 208, 64, 0), (1000, 200, 240, 0), (300, 3, 200, 8), (4096, 200, 200, 0),
          (257, 16, 80, 16), (130, 200, 600, 0), (20000, 200, 232, 0)]


@pytest.mark.parametrize("m,n,k,pad", SHAPES)
def test_tc_gemm_matches_float64(ctx, m, n, k, pad):
    g = torch.Generator(device="cpu").manual_seed(m * 7 + n + k)
    a = torch.randn((m, k + pad), generator=g).to(torch.bfloat16)
    b = torch.randn((n, k), generator=g).to(torch.bfloat16)
    ref = a[:, :k].double() @ b.double().T
    mag = a[:, :k].double().abs() @ b.double().abs().T
    out = ctx.debug_tc_gemm(a.cuda()[:, :k], b.cuda())
    ctx.sync(timeout_ms=30000)
    err = (out.cpu().double() - ref).abs()
    # FP32 accumulation of exact BF16 products: <= k * 2^-24 of the magnitude sum
    assert torch.all(err <= 2 * k * 2.0 ** -24 * mag + 1e-30), f"max err {err.max():.3g}"


# FP32 shapes: K slabs of 32 with ragged tails (225, 80, 13), N down to 3, rows spanning
# several persistent rounds
SHAPES_F32 = [(128, 208, 32, 0), (1000, 200, 225, 7), (300, 3, 200, 0), (257, 16, 80, 0),
              (130, 200, 600, 0), (40000, 200, 232, 0), (5, 200, 13, 3)]


@pytest.mark.parametrize("m,n,k,pad", SHAPES_F32)
def test_tc_gemm_f32_split_matches_float64(ctx, m, n, k, pad):
    g = torch.Generator(device="cpu").manual_seed(m * 5 + n + k)
    a = torch.randn((m, k + pad), generator=g) * torch.exp(torch.randn((m, k + pad), generator=g))
    b = torch.randn((n, k), generator=g)
    ref = a[:, :k].double() @ b.double().T
    mag = a[:, :k].double().abs() @ b.double().abs().T
    out = ctx.debug_tc_gemm_f32(a.cuda()[:, :k], b.cuda())
    ctx.sync(timeout_ms=30000)
    err = (out.cpu().double() - ref).abs()
    # split residual below 2^-24 |x| per operand (three 8-bit parts), FP32 accumulation of
    # 6 ceil(k / 16) MMA results: a few k 2^-24 of the magnitude sum bounds both
    assert torch.all(err <= 4 * k * 2.0 ** -24 * mag + 1e-30), f"max err {err.max():.3g}"
    # and it is far more accurate than one BF16 product (whose error is ~2^-9 of mag)
    assert (err / (mag + 1e-30)).max() < 2.0 ** -18
