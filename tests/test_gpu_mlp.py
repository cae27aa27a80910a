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


@pytest.mark.parametrize("M,N,K", [(128, 256, 4096), (256, 128, 2048), (1024, 1024, 512)])
def test_gemm_bf16_fp32_only_split_k(ctx, M, N, K):
    """C32-only products (the weight gradients) take the split-K path when
    their tiles alone would leave SMs idle."""
    import torch
    rng = np.random.default_rng(7 * M + N + K)
    A = _bf16(rng.standard_normal((M, K)))
    B = _bf16(rng.standard_normal((N, K)))
    dev = torch.device("cuda:0")
    C32, _ = ctx.gemm_bf16(A.to(dev), B.to(dev))
    ref = A.double().numpy() @ B.double().numpy().T
    got = C32.cpu().double().numpy()
    assert np.max(np.abs(got - ref)) < 2e-4 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("M,N,K", [(4096, 256, 1024), (1024, 256, 2048)])
def test_gemm_bf16_bias_only_split_k(ctx, M, N, K):
    """A C32 output with a bias and no bf16 copy (the network's last layer)
    also splits K; the first split adds the bias, the others only their
    partial products."""
    import torch
    rng = np.random.default_rng(11 * M + N + K)
    A = _bf16(rng.standard_normal((M, K)))
    B = _bf16(rng.standard_normal((N, K)))
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32))
    dev = torch.device("cuda:0")
    C32, _ = ctx.gemm_bf16(A.to(dev), B.to(dev), bias=bias.to(dev))
    ref = A.double().numpy() @ B.double().numpy().T + bias.double().numpy()[None, :]
    got = C32.cpu().double().numpy()
    assert np.max(np.abs(got - ref)) < 2e-4 * max(1.0, np.max(np.abs(ref)))


def test_gemm_bf16_m_valid_rows(ctx):
    import torch
    rng = np.random.default_rng(11)
    A = _bf16(rng.standard_normal((256, 128)))
    B = _bf16(rng.standard_normal((256, 128)))
    dev = torch.device("cuda:0")
    C32, _ = ctx.gemm_bf16(A.to(dev), B.to(dev), M_valid=200)
    ref = A.double().numpy() @ B.double().numpy().T
    got = C32.cpu().double().numpy()
    assert np.max(np.abs(got[:200] - ref[:200])) < 1e-4 * max(1.0, np.max(np.abs(ref)))


def _learned_targets(count, seed):
    from paper_2405_12866_gb300 import workloads as w
    gs = w.haar_gates(seed, w.STREAM_TARGET_GATES, 6 * count).reshape(count, 6, 4, 4)
    return np.stack([w.target_unitary(g, w.LEARNED_PAIRS, 4) for g in gs]), gs


def test_warm_start_gradients_match_oracle(ctx):
    from oracle import mlp_oracle as mo
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    seed = 3
    model = qfs.WarmStart(ctx, seed=seed, batch_cap=256)
    U, gs = _learned_targets(200, 17)
    labels = np.stack([np.stack([gs[i].reshape(-1).real, gs[i].reshape(-1).imag], axis=-1).reshape(-1)
                       for i in range(200)])
    loss, g = model.loss_grad(U, labels)
    params = qfs.WarmStart.unflatten(model.get_params().astype(np.float64))
    phif = w.sample_states(seed ^ 0x5EEDF1C5, 4, 8)
    F = 4.0 * np.einsum("tij,jk->tik", U, phif)
    X = np.stack([F.real, F.imag], axis=-1).reshape(200, 256)
    want_loss, want, mags = mo.loss_and_grads(params, X, labels, 192, round_bf16=True, magnitudes=True)
    assert abs(loss - want_loss) < 1e-3 * want_loss
    got = qfs.WarmStart.unflatten(g.astype(np.float64))
    # Element by element.  Both sides round the same tensors to bf16 at the
    # same points; an FP32-computed value that lies within its FP32 error of
    # a bf16 rounding boundary can round the other way, which moves that one
    # term of a sum by at most one bf16 step (2^-7 of its size, relative;
    # bf16 keeps 8 significant bits).  Each entry may therefore differ by
    # 2^-7 of the summed magnitude of its terms (|g|^T |H| for weights,
    # sum |g| for biases, from the oracle), which also covers the FP32
    # accumulation error; nothing else.  A wrong row, column or slice moves
    # entries by their own size, far outside this bound.
    for li, ((gw, gb), (ww, wb), (mw, mb)) in enumerate(zip(got, want, mags)):
        for name, a, b, m in (("W", gw, ww, mw), ("b", gb, wb, mb)):
            bound = 2.0 ** -7 * m + 1e-6 * np.max(m)
            bad = np.abs(a - b) > bound
            assert not np.any(bad), (f"layer {li} {name}: {int(bad.sum())} of {bad.size} entries outside the "
                                     f"bf16 rounding bound; worst excess "
                                     f"{float(np.max((np.abs(a - b) - bound) / np.maximum(m, 1e-30)))}")
        # and most entries agree far more closely than the bound (2^-7 = 7.8e-3)
        rel = np.abs(gw - ww) / np.maximum(mw, 1e-30)
        assert np.median(rel) < 1e-3, (li, float(np.median(rel)))
    model.close()


def test_warm_start_trains_and_predicts_unitaries(ctx):
    from paper_2405_12866_gb300 import qfs
    model = qfs.WarmStart(ctx, seed=5, batch_cap=512)
    U, gs = _learned_targets(1024, 23)
    labels = np.stack([np.stack([gs[i].reshape(-1).real, gs[i].reshape(-1).imag], axis=-1).reshape(-1)
                       for i in range(1024)])
    losses = model.train(U, labels, epochs=30, batch=256, lr=1e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0]
    pred = model.predict(U[:64])
    for g in pred.reshape(-1, 4, 4):
        assert np.max(np.abs(g.conj().T @ g - np.eye(4))) < 1e-12
    model.close()
