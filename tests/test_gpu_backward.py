"""Backward kernel of the eigendecomposition layer against the FP64 oracle and finite differences (GPU)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2604_27325_gb300 import binding as B
from paper_2604_27325_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

U32 = 2.0**-24


def _bwd_gpu(W, V, gW, gV, gap_eps=0.0):
    b, n = W.shape
    Wd, Vd = torch.from_numpy(W).cuda(), torch.from_numpy(V).cuda()
    gWd = torch.from_numpy(gW).cuda() if gW is not None else None
    gVd = torch.from_numpy(gV).cuda() if gV is not None else None
    gA = torch.empty(b, n, n, device="cuda")
    st = B.bed_eigh_backward_f32(Wd.data_ptr(), Vd.data_ptr(), gWd.data_ptr() if gWd is not None else None,
                                 gVd.data_ptr() if gVd is not None else None, gA.data_ptr(), b, n, gap_eps,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == B.BED_OK
    torch.cuda.synchronize()
    return gA.cpu().numpy()


@pytest.mark.parametrize("n", [3, 16, 32, 47, 64])
@pytest.mark.parametrize("which", ["both", "gW_only", "gV_only"])
def test_backward_kernel_matches_oracle_on_identical_inputs(n, which):
    """Same FP32 (W, V, gW, gV) into both: the FP32 GEMMs stay within 8 n^2 u |K|_F of the FP64 result,
    K = diag(gW) + F o (V^T gV) (three chained n-term FP32 products)."""
    A = wl.covariance(24, n, seed=800 + n)
    W, V = B.batched_eigh(torch.from_numpy(A).cuda())
    W, V = W.cpu().numpy(), V.cpu().numpy()
    rng = np.random.default_rng(n)
    gW = rng.standard_normal(W.shape).astype(np.float32) if which != "gV_only" else None
    gV = rng.standard_normal(V.shape).astype(np.float32) if which != "gW_only" else None
    gA = _bwd_gpu(W, V, gW, gV)
    for k in range(W.shape[0]):
        ref = oracle.eigh_backward(W[k], V[k], None if gW is None else gW[k], None if gV is None else gV[k])
        Kf = np.diag(gW[k]).astype(np.float64) if gW is not None else np.zeros((n, n))
        if gV is not None:
            M = V[k].T.astype(np.float64) @ gV[k]
            D = W[k][None, :].astype(np.float64) - W[k][:, None]
            np.fill_diagonal(D, 1.0)
            F = 1.0 / D
            np.fill_diagonal(F, 0.0)
            Kf = Kf + F * M
        assert np.linalg.norm(gA[k] - ref) <= 8 * n * n * U32 * np.linalg.norm(Kf) + 1e-30
        assert np.array_equal(gA[k], gA[k].T)


def test_backward_masks_close_pairs():
    n = 12
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(-1, 1, n)
    lam[5] = lam[4] + 1e-7
    A = ((Q * lam) @ Q.T).astype(np.float32)[None]
    A = 0.5 * (A + np.swapaxes(A, 1, 2))
    W, V = B.batched_eigh(torch.from_numpy(A).cuda())
    W, V = W.cpu().numpy(), V.cpu().numpy()
    gV = rng.standard_normal(V.shape).astype(np.float32)
    gA = _bwd_gpu(W, V, None, gV, gap_eps=1e-5)
    ref = oracle.eigh_backward(W[0], V[0], None, gV[0], gap_eps=1e-5)
    assert np.all(np.isfinite(gA))
    assert np.linalg.norm(gA[0] - ref) <= 1e-4 * np.linalg.norm(ref)


def _loss_oracle(M, w, G):
    W, V, _ = oracle.eigh(M)
    return float(w @ W + np.sum(G * V))


def test_differentiation_workload_autograd_against_oracle_and_finite_differences():
    """1024 covariances of size 32 with min eigen-gap >= 1e-3, L = sum w_i lambda_i + <G, V>.
    Per matrix the relative gradient error is held to n u |A|_2 / gap_min (the FP32 forward's eigenvector
    error kappa u, kappa = |A|_2/gap_min, with a factor n)."""
    A, w, G = wl.differentiation()
    b, n, _ = A.shape
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    W, V = B.eigh(At)
    loss = (torch.from_numpy(w).cuda() * W).sum() + (torch.from_numpy(G).cuda() * V).sum()
    loss.backward()
    gA = At.grad.cpu().numpy()
    Wo, Vo, _, _ = oracle.eigh_batch_f32(A, nthreads=os.cpu_count() or 1)
    worst = 0.0
    for k in range(b):
        ref = oracle.eigh_backward(Wo[k], Vo[k], w[k], G[k])
        gap = np.diff(Wo[k]).min()
        tol = n * U32 * np.abs(Wo[k]).max() / gap
        rel = np.linalg.norm(gA[k] - ref) / np.linalg.norm(ref)
        worst = max(worst, rel / tol)
        assert rel <= tol, (k, rel, tol)
    # FP64 central differences of the oracle's loss (h = 1e-6) on a sample, along symmetric directions
    rng = np.random.default_rng(44)
    h = 1e-6
    for k in rng.choice(b, 6, replace=False):
        M = A[k].astype(np.float64)
        gap = np.diff(Wo[k]).min()
        tol = n * U32 * np.abs(Wo[k]).max() / gap
        for _ in range(2):
            E = rng.standard_normal((n, n))
            E = 0.5 * (E + E.T)
            fd = (_loss_oracle(M + h * E, w[k], G[k]) - _loss_oracle(M - h * E, w[k], G[k])) / (2 * h)
            an = float(np.sum(gA[k] * E))
            assert abs(an - fd) <= tol * np.linalg.norm(gA[k]) * np.linalg.norm(E), (k, an, fd)
