"""The learned cost model's kernels: forward, loss gradient and Adam on the GPU
against the FP64 CPU reference MLP (oracle/mlp_ref.py), whose analytic
gradient is itself pinned by finite differences."""
import numpy as np
import pytest

from oracle import mlp_ref


def data(D=12, H=32, n=300, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 1, size=mlp_ref.num_params(D, H)) / np.sqrt(D)
    X = rng.uniform(-1, 1, size=(n, D))
    y = np.sin(X @ rng.normal(size=D)) + 0.1 * rng.normal(size=n)
    return p, X, y


@pytest.mark.parametrize("H", [16, 32])
def test_reference_gradient_matches_finite_differences(H):
    p, X, y = data(D=5, H=H, n=40)
    l, g = mlp_ref.loss_grad(p, X, y, 5, H)
    fd = mlp_ref.fd_grad(p, X, y, 5, H)
    assert abs(l - mlp_ref.loss(p, X, y, 5, H)) < 1e-14
    assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(g).max())


@pytest.mark.gpu
@pytest.mark.parametrize("H", [16, 32, 64])
def test_gpu_forward_and_gradient_match_reference(fea, H):
    import torch
    D = 12
    p, X, y = data(D=D, H=H, n=517, seed=H)
    assert fea.mlp_num_params(D, H) == p.size
    tp = torch.tensor(p, dtype=torch.float32, device="cuda")
    tX = torch.tensor(X, dtype=torch.float32, device="cuda")
    ty = torch.tensor(y, dtype=torch.float32, device="cuda")
    yh = fea.mlp_forward(tp, tX, H).cpu().numpy()
    ref = mlp_ref.forward(p.astype(np.float32), X.astype(np.float32), D, H)
    assert np.abs(yh - ref).max() < 1e-4 * max(1.0, np.abs(ref).max())
    loss, grad = fea.mlp_loss_grad(tp, tX, ty, H)
    l_ref, g_ref = mlp_ref.loss_grad(p.astype(np.float32), X.astype(np.float32), y.astype(np.float32), D, H)
    assert abs(loss.item() - l_ref) < 1e-4 * l_ref
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-4
    # deterministic: a second evaluation is bit-identical
    _, grad2 = fea.mlp_loss_grad(tp, tX, ty, H)
    assert torch.equal(grad, grad2)


@pytest.mark.gpu
def test_gpu_adam_matches_reference_and_training_converges(fea):
    import torch
    D, H = 8, 32
    p, X, y = data(D=D, H=H, n=256, seed=3)
    tp = torch.tensor(p, dtype=torch.float32, device="cuda")
    tX = torch.tensor(X, dtype=torch.float32, device="cuda")
    ty = torch.tensor(y, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(tp)
    v = torch.zeros_like(tp)
    pr, mr, vr = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    loss0 = None
    for step in range(1, 301):
        loss, grad = fea.mlp_loss_grad(tp, tX, ty, H)
        if step <= 3:  # one-step agreement of the update with the reference Adam
            _, gr = mlp_ref.loss_grad(tp.cpu().numpy().astype(np.float64), X, y, D, H)
            pr, mr, vr = mlp_ref.adam(tp.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64),
                                      m.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64),
                                      step, 1e-2)
        fea.mlp_adam(tp, grad, m, v, step, lr=1e-2)
        if step <= 3:
            assert np.abs(tp.cpu().numpy() - pr).max() < 1e-5
        if step == 1:
            loss0 = loss.item()
    final = fea.mlp_loss_grad(tp, tX, ty, H)[0].item()
    assert final < 0.25 * loss0
