"""Pins of the oracle's derivative of L = sum_{lambda inside} |lambda|^2.

* Closed form: for A = P diag(lam) Q, B = P Q the left / right eigenvectors
  are P^{-H} e_i and Q^{-1} e_i with v_i^H B x_i = 1, so
  G_A = 2 P^{-H} diag(lam_in) Q^{-H} and G_B = -2 P^{-H} diag(|lam_in|^2) Q^{-H}
  (lam_in: lam where inside, 0 elsewhere).
* Central differences of L itself (eigenvalues by the oracle's QZ) along
  random complex directions: (L(A + hE) - L(A - hE)) / 2h = Re <G_A, E>."""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs


def _pencil(n, seed):
    return inputs.prescribed_pencil(n, 8, seed=seed)


def test_grad_closed_form_prescribed_pencil():
    p = _pencil(40, 3)
    L, gA, gB, lin = oracle.eig_grad_abs2(p.A, p.B, 0, 0j, 1.0)
    inside = np.abs(p.lam) < 1.0
    d = np.where(inside, p.lam, 0.0)
    Pih = np.linalg.inv(p.P).conj().T
    Qih = np.linalg.inv(p.Q).conj().T
    refA = 2.0 * Pih @ np.diag(d) @ Qih
    refB = -2.0 * Pih @ np.diag(np.abs(d) ** 2) @ Qih
    assert abs(L - np.sum(np.abs(p.lam[inside]) ** 2)) < 1e-12 * max(1.0, L)
    assert np.max(np.abs(gA - refA)) < 1e-10 * np.max(np.abs(refA))
    assert np.max(np.abs(gB - refB)) < 1e-10 * np.max(np.abs(refB))


def _L(A, B):
    al, be, _ = oracle.ggev(A, B)
    lam = al / be
    return float(np.sum(np.abs(lam[np.abs(lam) < 1.0]) ** 2))


@pytest.mark.parametrize("which", ["A", "B"])
def test_grad_central_differences(which):
    p = _pencil(24, 7)
    L, gA, gB, _ = oracle.eig_grad_abs2(p.A, p.B, 0, 0j, 1.0)
    g = gA if which == "A" else gB
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(4):
        E = inputs.complex_normal(rng, (24, 24))
        if which == "A":
            fd = (_L(p.A + h * E, p.B) - _L(p.A - h * E, p.B)) / (2 * h)
        else:
            fd = (_L(p.A, p.B + h * E) - _L(p.A, p.B - h * E)) / (2 * h)
        an = float(np.real(np.vdot(g, E)))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)
