"""Differentiation form on the GPU: L = sum over the inside eigenvalues of
|lambda|^2 and its gradients with respect to A and B, from a GFEAST run on
(A, B), a run on (A^H, B^H) over the conjugated contour (left vectors) and
the library's adjoint kernels.  Checked against the oracle's gradient (own
QZ of the whole pencil), against the closed form of the prescribed-spectrum
pencil, and against central differences of L through torch.autograd."""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu


def _runs(fg, p, m0, prec, eps):
    import torch
    A = torch.from_numpy(p.A).cuda()
    B = torch.from_numpy(p.B).cuda()
    rng = np.random.default_rng(1)
    Y = torch.from_numpy(inputs.complex_normal(rng, (p.n, m0))).cuda()
    kw = dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0, eps=eps, prec=prec, refine_tol=1e-13,
              max_refine=4)
    right = fg.Feast(A, B, Y, **kw)
    right.run()
    left = fg.Feast(A.conj().t().resolve_conj(), B.conj().t().resolve_conj(), Y, **kw)
    left.run()
    return right, left


@pytest.mark.parametrize("prec", [0, 1])
def test_grad_matches_oracle(prec):
    import paper_1404_1768_gb300 as fg
    p = inputs.prescribed_pencil(100, 8, seed=3)
    right, left = _runs(fg, p, 48, prec, 1e-12 if prec == 0 else 1e-10)
    L, gA, gB, cnt = right.grad_abs2(left)
    Lr, gAr, gBr, lin = oracle.eig_grad_abs2(p.A, p.B, 0, 0j, 1.0)
    assert cnt == len(lin)
    assert abs(L - Lr) < 1e-8 * max(1.0, Lr)
    gA = gA.cpu().numpy()
    gB = gB.cpu().numpy()
    assert np.max(np.abs(gA - gAr)) < 1e-6 * np.max(np.abs(gAr))
    assert np.max(np.abs(gB - gBr)) < 1e-6 * np.max(np.abs(gBr))
    right.close()
    left.close()


def test_grad_closed_form_n200():
    import paper_1404_1768_gb300 as fg
    p = inputs.prescribed_pencil(200, 8, seed=0)
    right, left = _runs(fg, p, 64, 0, 1e-12)
    L, gA, gB, cnt = right.grad_abs2(left)
    inside = np.abs(p.lam) < 1.0
    d = np.where(inside, p.lam, 0.0)
    Pih = np.linalg.inv(p.P).conj().T
    Qih = np.linalg.inv(p.Q).conj().T
    refA = 2.0 * Pih @ np.diag(d) @ Qih
    refB = -2.0 * Pih @ np.diag(np.abs(d) ** 2) @ Qih
    assert cnt == int(inside.sum())
    assert np.max(np.abs(gA.cpu().numpy() - refA)) < 1e-6 * np.max(np.abs(refA))
    assert np.max(np.abs(gB.cpu().numpy() - refB)) < 1e-6 * np.max(np.abs(refB))
    right.close()
    left.close()


def test_autograd_central_differences():
    import torch
    import paper_1404_1768_gb300 as fg
    p = inputs.prescribed_pencil(80, 8, seed=4)
    A = torch.from_numpy(p.A).cuda().requires_grad_(True)
    B = torch.from_numpy(p.B).cuda().requires_grad_(True)
    rng = np.random.default_rng(2)
    Y = torch.from_numpy(inputs.complex_normal(rng, (80, 40))).cuda()
    kw = dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0, eps=1e-12)
    L = fg.eig_sum_abs2(A, B, Y, **kw)
    L.backward()
    gA, gB = A.grad.cpu().numpy(), B.grad.cpu().numpy()
    h = 1e-5
    for t in range(4):
        E = inputs.complex_normal(np.random.default_rng(20 + t), (80, 80))
        Et = torch.from_numpy(E).cuda()
        with torch.no_grad():
            for which, g in (("A", gA), ("B", gB)):
                if which == "A":
                    lp = fg.eig_sum_abs2(A.detach() + h * Et, B.detach(), Y, **kw)
                    lm = fg.eig_sum_abs2(A.detach() - h * Et, B.detach(), Y, **kw)
                else:
                    lp = fg.eig_sum_abs2(A.detach(), B.detach() + h * Et, Y, **kw)
                    lm = fg.eig_sum_abs2(A.detach(), B.detach() - h * Et, Y, **kw)
                fd = (float(lp) - float(lm)) / (2 * h)
                an = float(np.real(np.vdot(g, E)))
                assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (which, fd, an)
