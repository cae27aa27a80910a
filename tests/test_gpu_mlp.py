"""GPU checks of the learned warm start's tensor-core (tcgen05) kernels
against plain CPU references of the same operation in float64 on the same
bf16-rounded inputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_12866_gb300 import build, qfs
    build.build()
    c = qfs.Context(0)
    yield c
    c.close()


def _bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (512, 1024, 1024)])
def test_gemm_bf16_matches_reference(ctx, M, N, K):
    import torch
    rng = np.random.default_rng(M + N + K)
    A = _bf16(rng.standard_normal((M, K)))
    B = _bf16(rng.standard_normal((N, K)))
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32))
    dev = torch.device("cuda:0")
    C32, C16 = ctx.gemm_bf16(A.to(dev), B.to(dev), bias=bias.to(dev), gelu=True, want_bf16=True)
    ref = A.double().numpy() @ B.double().numpy().T + bias.double().numpy()
    got = C32.cpu().double().numpy()
    assert np.max(np.abs(got - ref)) < 1e-4 * max(1.0, np.max(np.abs(ref)))
    gelu = 0.5 * ref * (1 + np.tanh(0.7978845608028654 * (ref + 0.044715 * ref ** 3)))
    assert np.max(np.abs(C16.cpu().double().numpy() - gelu)) < 1e-2 * max(1.0, np.max(np.abs(gelu)))
