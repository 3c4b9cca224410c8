"""GPU checks of the warm-start network's tensor-core kernels
(include/fil_mlp.h) against the FP64 reference in oracle/mlp.py.

GEMM: C = A B^T with BF16 inputs and FP32 accumulation; every entry within
2^-22 * K * max|a_k b_k| of the FP64 product of the same BF16 values.
Network: the reference emulates the BF16 roundings of the tensor-core path,
so the remaining differences are FP32 accumulation order (and the rare BF16
rounding it flips): outputs within 2e-3 of their scale, the loss within 1e-4
relative, and every gradient entry within K_GRAD * 2^-8 of its magnitude sum
(the backward pass with absolute values, oracle/mlp.py grad_magnitudes: each
term of the entry can carry one flipped BF16 rounding of a factor, 2^-8
relative, and upstream flips reach it through the same absolute-value chain),
as well as within 1e-2 normwise per weight or bias block.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as om  # noqa: E402

NIN = om.DIMS[0][0]
K_GRAD = 4.0

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


def _bf16_dev(a):
    return torch.from_numpy(om.bf16_bits(a).view(np.int16)).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 192, 448), (448, 256, 4096),
                                   (1, 32, 64), (513, 512, 128)])
def test_tc_gemm_matches_fp64(fil, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    Ad, Bd = _bf16_dev(A), _bf16_dev(B)
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    fil.fil_tc_gemm_bf16(Ad, K, Bd, K, C, N, M, N, K)
    Ab, Bb = om.bf16_round(A), om.bf16_round(B)
    ref = Ab @ Bb.T
    bound = 2.0 ** -22 * K * (np.abs(Ab).max(axis=1)[:, None] * np.abs(Bb).max(axis=1)[None, :])
    err = np.abs(C.cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_tc_gemm_rejects_bad_shapes(fil):
    A = torch.zeros((128, 64), dtype=torch.int16, device="cuda")
    C = torch.zeros((128, 48), dtype=torch.float32, device="cuda")
    with pytest.raises(fil.FilError):
        fil.fil_tc_gemm_bf16(A, 64, A, 64, C, 48, 128, 48, 64)       # N not a multiple of 32
    with pytest.raises(fil.FilError):
        fil.fil_tc_gemm_bf16(A, 64, A, 64, C, 48, 128, 32, 48)       # K not a multiple of 64


def _setup(fil, rng, B):
    p = np.zeros(om.NPARAM, dtype=np.float32)
    off = 0
    for i, o in om.DIMS:
        p[off:off + i * o] = rng.standard_normal(i * o) * np.sqrt(2.0 / i)
        off += i * o
        p[off:off + o] = 0.1 * rng.standard_normal(o)
        off += o
    norm = [rng.standard_normal(NIN).astype(np.float32), rng.uniform(0.5, 2, NIN).astype(np.float32),
            rng.standard_normal(192).astype(np.float32), rng.uniform(0.5, 2, 192).astype(np.float32)]
    m = fil.fil_mlp_create(4096)
    fil.fil_mlp_set_params(m, p)
    fil.fil_mlp_set_norm(m, *norm)
    x = (norm[0] + norm[1] * rng.standard_normal((B, NIN))).astype(np.float32)
    t = (norm[2] + norm[3] * rng.standard_normal((B, 192))).astype(np.float32)
    return m, p, norm, x, t


def test_forward_matches_reference(fil):
    rng = np.random.default_rng(3)
    B = 300
    m, p, norm, x, _ = _setup(fil, rng, B)
    y = torch.zeros((B, 192), dtype=torch.float32, device="cuda")
    fil.fil_mlp_forward(m, torch.from_numpy(x).cuda(), y, B)
    fil.fil_mlp_destroy(m)
    ref, _ = om.forward(p, x, norm)
    scale = np.abs(ref - norm[2]).max()
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=0, atol=2e-3 * scale)


@pytest.mark.parametrize("B", [64, 300, 1000])
def test_gradients_match_reference(fil, B):
    rng = np.random.default_rng(B)
    m, p, norm, x, t = _setup(fil, rng, B)
    g = torch.zeros(om.NPARAM, dtype=torch.float32, device="cuda")
    loss = fil.fil_mlp_gradients(m, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), B, g)
    fil.fil_mlp_destroy(m)
    ref_loss, ref = om.loss_and_grad(p, x, t, norm)
    mag = om.grad_magnitudes(p, x, t, norm)
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    g = g.cpu().numpy()
    # every entry: within K_GRAD BF16 roundings (2^-8) of its magnitude sum
    ratio = np.abs(g - ref) / (2.0 ** -8 * mag + 1e-30)
    assert np.all(ratio <= K_GRAD), "max ratio %.3f at %d" % (ratio.max(), int(ratio.argmax()))
    off = 0
    for i, o in om.DIMS:
        for n in (i * o, o):
            a, r = g[off:off + n], ref[off:off + n]
            assert np.linalg.norm(a - r) <= 1e-2 * np.linalg.norm(r), (off, n)
            off += n


def test_training_reduces_the_loss(fil):
    """Adam on a smooth synthetic regression (targets a fixed random linear
    map of the inputs): the loss falls by more than 5x in 300 steps."""
    rng = np.random.default_rng(7)
    B = 1024
    m, p, norm, x, _ = _setup(fil, rng, B)
    Wt = rng.standard_normal((NIN, 192)) / np.sqrt(NIN)
    xn = (x - norm[0]) / norm[1]
    t = (norm[2] + norm[3] * (xn @ Wt)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = fil.fil_mlp_train_step(m, xd, td, B, 1e-3)
    for _ in range(299):
        last = fil.fil_mlp_train_step(m, xd, td, B, 1e-3)
    fil.fil_mlp_destroy(m)
    assert last < first / 5, (first, last)
