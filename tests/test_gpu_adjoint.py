"""Adjoint kernel (tdc_eig_backward / tdc_eig_backward_batched) against the oracle's
adjoint formula on the same (lam, Q), the Hellmann-Feynman closed form, and
central finite differences through the full GPU eigensolver (autograd)."""
import numpy as np
import pytest
import torch

from oracle.adjoint import adjoint
from paper_2008_01990_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def tdc():
    from paper_2008_01990_gb300 import build, tdc as t
    build.build()
    t.lib()
    return t


def test_backward_matches_oracle_formula(tdc):
    ds, es, ws, Gs, gaps, _ = inputs.backward_problems(1, 200, 55, min_gap_rel=1e-4)
    d, e = torch.tensor(ds[0], device=DEV), torch.tensor(es[0], device=DEV)
    lam, Q = tdc.eig(d, e, tdc.default_opts(leaf=32), check=True)
    w = torch.tensor(ws[0], device=DEV)
    G = torch.tensor(Gs[0], device=DEV)
    db, eb = tdc.eig_backward(lam, Q, w, G)
    db_o, eb_o = adjoint(lam.cpu().numpy(), Q.cpu().numpy(), ws[0], Gs[0])
    scale = max(np.abs(db_o).max(), np.abs(eb_o).max())
    assert np.max(np.abs(db.cpu().numpy() - db_o)) <= 1e-11 * scale
    assert np.max(np.abs(eb.cpu().numpy() - eb_o)) <= 1e-11 * scale


def test_backward_hellmann_feynman(tdc):
    d, e = inputs.uniform_tridiag(150, 3)
    lam, Q = tdc.eig(torch.tensor(d, device=DEV), torch.tensor(e, device=DEV), tdc.default_opts(leaf=32), check=True)
    w = torch.tensor(inputs.SplitMix64(4).normal(150), device=DEV)
    db, eb = tdc.eig_backward(lam, Q, w, None)
    Qn = Q.cpu().numpy()
    wn = w.cpu().numpy()
    assert np.allclose(db.cpu().numpy(), (Qn ** 2) @ wn, atol=1e-13)
    assert np.allclose(eb.cpu().numpy(), 2 * (Qn[:-1] * Qn[1:]) @ wn, atol=1e-13)


def test_backward_batched_c5_shape(tdc):
    # the backward workload's problems (n = 512, minimum gap >= 1e-5 ||T||), 8 of them
    B, n = 8, 512
    ds, es, ws, Gs, gaps, _ = inputs.backward_problems(B, n, 5)
    d = torch.tensor(ds, device=DEV)
    e = torch.tensor(es, device=DEV)
    dd = d.clone().requires_grad_(True)
    ee = e.clone().requires_grad_(True)
    lam, Q = tdc.eigh_tridiagonal(dd, ee, tdc.default_opts(leaf=32))
    w = torch.tensor(ws, device=DEV)
    G = torch.tensor(Gs, device=DEV)
    loss = (w * lam).sum() + (G * Q).sum()
    loss.backward()
    for b in range(B):
        db_o, eb_o = adjoint(lam[b].detach().cpu().numpy(), Q[b].detach().cpu().numpy(), ws[b], Gs[b])
        scale = max(np.abs(db_o).max(), np.abs(eb_o).max())
        assert np.max(np.abs(dd.grad[b].cpu().numpy() - db_o)) <= 1e-10 * scale
        assert np.max(np.abs(ee.grad[b].cpu().numpy() - eb_o)) <= 1e-10 * scale


def test_autograd_vs_central_differences(tdc):
    n = 48
    ds, es, ws, Gs, gaps, _ = inputs.backward_problems(1, n, 21, min_gap_rel=1e-3)
    d0, e0, w, G = ds[0], es[0], ws[0], Gs[0]
    o = tdc.default_opts(leaf=16)
    dd = torch.tensor(d0, device=DEV, requires_grad=True)
    ee = torch.tensor(e0, device=DEV, requires_grad=True)
    lam, Q = tdc.eigh_tridiagonal(dd, ee, o)
    wt = torch.tensor(w, device=DEV)
    Gt = torch.tensor(G, device=DEV)
    ((wt * lam).sum() + (Gt * Q).sum()).backward()
    Q0 = Q.detach()

    def loss(dv, ev):
        l2, Q2 = tdc.eig(torch.tensor(dv, device=DEV), torch.tensor(ev, device=DEV), o)
        sgn = torch.sign((Q2 * Q0).sum(dim=0))  # align eigenvector signs with the base point
        return float((wt * l2).sum() + (Gt * (Q2 * sgn)).sum())

    h = 1e-6
    fd_d = np.array([(loss(d0 + h * np.eye(n)[i], e0) - loss(d0 - h * np.eye(n)[i], e0)) / (2 * h) for i in range(n)])
    fd_e = np.array([(loss(d0, e0 + h * np.eye(n - 1)[i]) - loss(d0, e0 - h * np.eye(n - 1)[i])) / (2 * h)
                     for i in range(n - 1)])
    scale = max(1.0, np.abs(fd_d).max(), np.abs(fd_e).max())
    assert np.max(np.abs(dd.grad.cpu().numpy() - fd_d)) <= 1e-5 * scale
    assert np.max(np.abs(ee.grad.cpu().numpy() - fd_e)) <= 1e-5 * scale
