"""Phi_L = U Psi (Section 3's A tensor) on the GPU: the FP64 kernel and the
FP32 pair-arithmetic kernel of the mixed-precision runs, against a plain
FP64 matrix product on the host."""
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


@pytest.mark.parametrize("n,M", [(2, 1), (3, 8), (5, 3), (6, 33), (8, 16), (10, 64), (12, 32), (12, 1)])
def test_target_product_matches_fp64(ctx, n, M):
    import torch
    from paper_2405_12866_gb300 import qfs
    N = 1 << n
    g = torch.Generator(device="cuda").manual_seed(1000 * n + M)
    U = torch.randn((N, N), dtype=torch.complex128, device="cuda", generator=g) / np.sqrt(N)
    P = torch.randn((N, M), dtype=torch.complex128, device="cuda", generator=g) / np.sqrt(N)
    want = U.cpu().numpy() @ P.cpu().numpy()
    scale = np.abs(want).max()
    got64 = ctx.target_product(n, U, P, qfs.QFS_FP64).cpu().numpy()
    assert np.abs(got64 - want).max() <= 1e-14 * np.sqrt(N) * scale
    pair = ctx.target_product(n, U, P, qfs.QFS_MIXED).cpu().numpy()
    err = np.abs(pair - want).max()
    # ~48-bit pair arithmetic: far below FP32 (6e-8), within 2^-40 of the scale
    assert err <= 1e-12 * scale, err


def test_target_product_rejects_bad_sizes(ctx):
    import torch
    from paper_2405_12866_gb300 import qfs
    U = torch.zeros((8, 8), dtype=torch.complex128, device="cuda")
    P = torch.zeros((8, 9), dtype=torch.complex128, device="cuda")
    with pytest.raises(qfs.QfsError):
        ctx.target_product(3, U, P, qfs.QFS_MIXED)
    with pytest.raises(qfs.QfsError):
        ctx.target_product(3, U, P[:, :2].contiguous(), 7)
