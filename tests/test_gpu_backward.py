"""Backward of the inversion: grad_A = -sym(X G X) through the C-ABI kernel
and the autograd Function, against the FP64 oracle gradient and FP64 finite
differences."""
import numpy as np
import pytest

import oracle
import spd_inputs as si

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 8, 16, 32, 63, 64, 65, 200])
@pytest.mark.parametrize("dtype_name,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_backward_kernel_vs_oracle(gpu, n, dtype_name, tol):
    import torch
    from paper_1002_4057_gb300 import _lib as L
    dtype = getattr(torch, dtype_name)
    A = si.wishart_spd(n, 1.0, seed=n)
    X = np.linalg.inv(A)
    X = 0.5 * (X + X.T)
    Gm = np.random.default_rng(n).standard_normal((n, n))  # not symmetric: sym() is part of the op
    ref = oracle.backward(X, 0.5 * (Gm + Gm.T))
    dX = torch.from_numpy(X).to(gpu, dtype)
    dG = torch.from_numpy(np.asfortranarray(Gm)).to(gpu, dtype)  # column-major
    out = torch.empty((n, n), dtype=dtype, device=gpu).t()
    fn = L.spdinv_potri_backward if dtype == torch.float64 else L.spdinv_spotri_backward
    st = fn(1, n, dX.data_ptr(), n, n * n, dG.data_ptr(), n, n * n, out.data_ptr(), n, n * n,
            torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    assert np.array_equal(got, got.T)  # exactly symmetric
    assert oracle.rel_frobenius(got, ref) <= tol


@pytest.mark.parametrize("n", [8, 16, 32])
def test_autograd_finite_differences_fp64(gpu, n):
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    A = si.wishart_spd(n, 1.0, seed=500 + n)
    G = si.symmetric_gaussian(n, seed=600 + n)
    E = si.symmetric_gaussian(n, seed=700 + n)
    dA = torch.from_numpy(A).to(gpu).requires_grad_(True)
    X = T.spd_inverse(dA)
    loss = (X * torch.from_numpy(G).to(gpu)).sum()
    loss.backward()
    an = float((dA.grad.cpu().numpy() * E).sum())

    def f(M):
        R, info = oracle.potri(M)
        assert info == 0
        return float(np.sum(G * oracle.symmetrize_lower(R)))

    h = 1e-5 * np.linalg.norm(A, 2)
    fd = (f(A + h * E) - f(A - h * E)) / (2 * h)
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    Xo = oracle.symmetrize_lower(oracle.potri(A)[0])
    assert oracle.rel_frobenius(dA.grad.cpu().numpy(), oracle.backward(Xo, G)) <= 1e-10


@pytest.mark.parametrize("dtype_name,tol_x,tol_g", [("float64", 1e-10, 1e-10), ("float32", 1e-4, 1e-4)])
def test_autograd_batch_config(gpu, dtype_name, tol_x, tol_g):
    """A batch of n=512 matrices, A = B B^T/n + I (the differentiable
    workload's shape; 8 of its 256 matrices checked against the oracle)."""
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    dtype = getattr(torch, dtype_name)
    n, b = 512, 8
    As = [si.wishart_spd(n, 1.0, seed=si.SEED_BASE + 4 * 1000 + k) for k in range(b)]
    Gs = [si.symmetric_gaussian(n, seed=si.SEED_BASE + 4 * 2000 + k) for k in range(b)]
    dA = torch.from_numpy(np.stack(As)).to(gpu, dtype).requires_grad_(True)
    dG = torch.from_numpy(np.stack(Gs)).to(gpu, dtype)
    X = T.spd_inverse(dA)
    X.backward(dG)
    torch.cuda.synchronize()
    Xh = X.detach().double().cpu().numpy()
    gh = dA.grad.double().cpu().numpy()
    for k in range(b):
        assert np.array_equal(Xh[k], Xh[k].T)
        Xo = oracle.symmetrize_lower(oracle.potri(As[k])[0])
        assert oracle.rel_frobenius(Xh[k], Xo) <= tol_x
        assert oracle.rel_frobenius(gh[k], oracle.backward(Xo, Gs[k])) <= tol_g
