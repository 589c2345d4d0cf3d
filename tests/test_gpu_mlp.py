"""The hand-written tensor-core contraction of the PPO networks (sg_mlp_gemm)
against FP64 products of the same FP32 inputs.

With the split-precision (3xTF32) products the result must carry FP32
accuracy: max |C - C64| <= 2e-6 * sum_k |A(m,k) B(n,k)| (about twenty FP32
roundings of the sum of magnitudes; one TF32 product would miss this by
three orders of magnitude), widened by sqrt(K / 1024) for sums of more than
1024 terms (FP32 accumulation error grows like the square root of the number
of terms), for the three operand layouts of a layer -- forward (X W^T),
input gradient (dY W) and weight gradient (dY^T X, K split over CTAs) -- at
the networks' widths (28-wide inputs, 256, 128, 64 hidden, 8 and 1 outputs),
with ragged M, N and K, bias and ELU -- both with B split into its TF32 parts
by every CTA and with B split once beforehand (a work buffer that holds its
parts: the path of the PPO networks' forward and input-gradient products).
The single-product TF32 mode must land within TF32 rounding (2^-9 relative
to the magnitudes) and be measurably coarser than the split mode.  The
narrow products of the networks (8- and 1-wide output layers and the input
gradients below them) in the mode that runs them as FP32 FMA loops meet the
same bound (exact FP32 products, fixed-order FP32 sums); in that mode the
other shapes take the tensor-core path unchanged.
"""
import pytest
import torch

from paper_2310_04676_gb300 import sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def _rand(shape, seed):
    g = torch.Generator().manual_seed(seed)
    return (torch.rand(shape, generator=g, dtype=torch.float64) * 2 - 1).float()


def _check(C, A64, B64, bias=None, elu=False, tol=2e-6):
    tol = tol * max(1.0, (A64.shape[1] / 1024) ** 0.5)
    ref = A64 @ B64.T
    mag = A64.abs() @ B64.abs().T
    if bias is not None:
        ref = ref + bias.double()[None, :]
        mag = mag + bias.double().abs()[None, :]
    if elu:
        ref = torch.where(ref > 0, ref, torch.expm1(ref))
    err = (C.double().cpu() - ref).abs()
    # the ELU is e^x - 1 from the hardware exponential (at most 2 ulp of e^x
    # <= 1 for x <= 0 with |x| < 0.85, fewer beyond) and one rounding of the
    # difference: an absolute error of at most 3e-7 on top of the product's
    absolute = 5e-7 if elu else 0.0
    assert (err <= tol * mag + absolute + 1e-30).all(), (err / mag.clamp_min(1e-30)).max().item()
    return (err / mag.clamp_min(1e-30)).max().item()


def _presplit_floats(N, K):
    """Floats of B's pre-split TF32 parts: ceil(K/16) chunks x 2 parts x N
    rounded up to 128 rows x 16."""
    return -(-K // 16) * 2 * (-(-N // 128) * 128) * 16


@pytest.mark.parametrize("presplit", [False, True])
@pytest.mark.parametrize("rows,inp,out", [(300, 28, 256), (257, 256, 128), (129, 128, 64),
                                          (200, 64, 8), (131, 64, 1), (1000, 256, 256)])
def test_forward_layer(rows, inp, out, presplit):
    X, W, b = _rand((rows, inp), 1), _rand((out, inp), 2), _rand((out,), 3)
    Xd, Wd, bd = X.cuda(), W.cuda(), b.cuda()
    work = torch.empty(_presplit_floats(out, inp), device="cuda") if presplit else None
    for elu in (False, True):
        Y = torch.empty(rows, out, device="cuda")
        sg.mlp_gemm(Xd, (inp, 1), Wd, (inp, 1), rows, out, inp, Y, out, bias=bd, elu=elu,
                    work=work)
        torch.cuda.synchronize()
        _check(Y, X.double(), W.double(), b, elu)
    # ELU without a bias
    Y = torch.empty(rows, out, device="cuda")
    sg.mlp_gemm(Xd, (inp, 1), Wd, (inp, 1), rows, out, inp, Y, out, elu=True, work=work)
    torch.cuda.synchronize()
    _check(Y, X.double(), W.double(), None, True)


@pytest.mark.parametrize("rows,inp,out", [(70001, 28, 256), (65537, 256, 128), (40000, 128, 64),
                                          (50001, 40, 64), (45000, 33, 128)])
def test_forward_persistent_tiles(rows, inp, out):
    """More output tiles than persistent CTAs (pre-split weights): each CTA
    takes several tiles in turn, the next tile's first chunks copied during
    the current tile's epilogue (the two-chunk lookahead crosses each tile
    boundary; K = 33 and 40 end in a ragged K chunk); a sample of rows, the
    first and the last (ragged) tile against FP64."""
    X, W, b = _rand((rows, inp), 21), _rand((out, inp), 22), _rand((out,), 23)
    Y = torch.empty(rows, out, device="cuda")
    work = torch.empty(_presplit_floats(out, inp), device="cuda")
    sg.mlp_gemm(X.cuda(), (inp, 1), W.cuda(), (inp, 1), rows, out, inp, Y, out, bias=b.cuda(),
                elu=True, work=work)
    torch.cuda.synchronize()
    g = torch.Generator().manual_seed(24)
    idx = torch.cat([torch.randperm(rows, generator=g)[:3000], torch.arange(128),
                     torch.arange(rows - 200, rows)])
    _check(Y.cpu()[idx], X.double()[idx], W.double(), b, True)


@pytest.mark.parametrize("rows,inp,out", [(40000, 256, 128), (39000, 64, 8), (38913, 128, 64)])
def test_input_gradient_presplit(rows, inp, out):
    """Enough row tiles that the library splits B = W^T once into the work
    buffer (no K split), as the PPO update's input gradients do; a sample of
    rows is checked against FP64."""
    dY, W = _rand((rows, out), 10), _rand((out, inp), 11)
    dX = torch.empty(rows, inp, device="cuda")
    work = torch.empty(_presplit_floats(inp, out), device="cuda")
    sg.mlp_gemm(dY.cuda(), (out, 1), W.cuda(), (1, inp), rows, inp, out, dX, inp, work=work)
    torch.cuda.synchronize()
    g = torch.Generator().manual_seed(12)
    idx = torch.cat([torch.randperm(rows, generator=g)[:2000], torch.tensor([0, rows - 1])])
    _check(dX.cpu()[idx], dY.double()[idx], W.double().T)


@pytest.mark.parametrize("rows,inp,out", [(300, 256, 128), (257, 128, 64), (190, 64, 8),
                                          (140, 256, 256)])
def test_input_gradient(rows, inp, out):
    dY, W = _rand((rows, out), 4), _rand((out, inp), 5)
    dX = torch.empty(rows, inp, device="cuda")
    # dX[r][i] = sum_o dY[r][o] W[o][i]: B(n = i, k = o) = W[o * inp + i]
    sg.mlp_gemm(dY.cuda(), (out, 1), W.cuda(), (1, inp), rows, inp, out, dX, inp)
    torch.cuda.synchronize()
    _check(dX, dY.double(), W.double().T)


@pytest.mark.parametrize("rows,inp,out", [(5000, 28, 256), (4099, 256, 128), (3000, 128, 64),
                                          (2500, 64, 8), (777, 64, 1)])
def test_weight_gradient_split(rows, inp, out):
    dY, X = _rand((rows, out), 6), _rand((rows, inp), 7)
    dW = torch.empty(out, inp, device="cuda")
    work = torch.empty(400 * out * inp, device="cuda")
    # dW[o][i] = sum_r dY[r][o] X[r][i]: A(m = o, k = r) = dY[r * out + o], B(n = i, k = r)
    sg.mlp_gemm(dY.cuda(), (1, out), X.cuda(), (1, inp), out, inp, rows, dW, inp, work=work)
    torch.cuda.synchronize()
    _check(dW, dY.double().T, X.double().T)
    # the same without a work buffer (one CTA per output tile) agrees to rounding
    dW1 = torch.empty_like(dW)
    sg.mlp_gemm(dY.cuda(), (1, out), X.cuda(), (1, inp), out, inp, rows, dW1, inp)
    torch.cuda.synchronize()
    _check(dW1, dY.double().T, X.double().T)


@pytest.mark.parametrize("presplit", [False, True])
def test_single_tf32_product_is_coarser(presplit):
    X, W, b = _rand((256, 256), 8), _rand((128, 256), 9), _rand((128,), 13)
    work = torch.empty(_presplit_floats(128, 256), device="cuda") if presplit else None
    Y3, Y1 = (torch.empty(256, 128, device="cuda") for _ in range(2))
    bd = b.cuda()
    sg.mlp_gemm(X.cuda(), (256, 1), W.cuda(), (256, 1), 256, 128, 256, Y3, 128, bias=bd,
                work=work, split=True)
    sg.mlp_gemm(X.cuda(), (256, 1), W.cuda(), (256, 1), 256, 128, 256, Y1, 128, bias=bd,
                work=work, split=False)
    torch.cuda.synchronize()
    e3 = _check(Y3, X.double(), W.double(), b)
    e1 = _check(Y1, X.double(), W.double(), b, tol=2.0 ** -9)
    assert e1 > 20 * e3


@pytest.mark.parametrize("rows,inp,out,elu", [(1000, 28, 256, True), (777, 28, 256, False),
                                              (1000, 64, 8, False), (515, 64, 1, False),
                                              (300, 64, 8, True), (129, 8, 64, False),
                                              (200, 1, 64, True)])
def test_narrow_forward_fp32(rows, inp, out, elu):
    X, W, b = _rand((rows, inp), 14), _rand((out, inp), 15), _rand((out,), 16)
    Y = torch.empty(rows, out, device="cuda")
    sg.mlp_gemm(X.cuda(), (inp, 1), W.cuda(), (inp, 1), rows, out, inp, Y, out, bias=b.cuda(),
                elu=elu, split=2)
    torch.cuda.synchronize()
    _check(Y, X.double(), W.double(), b, elu)


@pytest.mark.parametrize("rows,inp,out", [(999, 64, 8), (1000, 64, 1), (257, 128, 16)])
def test_narrow_input_gradient_fp32(rows, inp, out):
    dY, W = _rand((rows, out), 17), _rand((out, inp), 18)
    dX = torch.empty(rows, inp, device="cuda")
    sg.mlp_gemm(dY.cuda(), (out, 1), W.cuda(), (1, inp), rows, inp, out, dX, inp, split=2)
    torch.cuda.synchronize()
    _check(dX, dY.double(), W.double().T)


@pytest.mark.parametrize("rows,inp,out", [(98304, 64, 8), (98304, 64, 1), (4111, 28, 256)])
def test_weight_gradient_in_narrow_mode(rows, inp, out):
    """Weight gradients take the tensor-core split-K path in that mode too."""
    dY, X = _rand((rows, out), 19), _rand((rows, inp), 20)
    dW = torch.empty(out, inp, device="cuda")
    work = torch.empty(400 * out * inp, device="cuda")
    sg.mlp_gemm(dY.cuda(), (1, out), X.cuda(), (1, inp), out, inp, rows, dW, inp, work=work,
                split=2)
    torch.cuda.synchronize()
    _check(dW, dY.double().T, X.double().T)
