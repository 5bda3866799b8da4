"""Conjugate gradient on the normal equations (CGNE), plain numpy (test
infrastructure only).

Sec. 4 foresees switching SAP-GCR to CG for the most difficult cases; CG
needs a Hermitian positive definite operator, so it runs on D^+ D x = D^+ b.
Textbook CG steps on A = D^+ D with caller-supplied callables for D and D^+:

  r = D^+ (b - D x);  p = r
  repeat:  t = D p;  alpha = |r|^2 / |t|^2;  x += alpha p;  r -= alpha D^+ t;
           beta = |r_new|^2 / |r|^2;  p = r_new + beta p
  until |b - D x| <= tol |b| (checked with the true residual).
"""
from __future__ import annotations

import numpy as np


def cgne(D, Dh, b, x0=None, tol=1e-12, max_iter=10000, check_every=1):
    """Solve D x = b through D^+ D x = D^+ b.  Returns (x, info) with
    info = {"iterations", "converged", "true_rel_res", "normal_res" (|r| per
    iteration), "residuals" (the normal-equation residual vectors of the
    first 8 iterations, for the orthogonality check)}."""
    b = np.asarray(b, np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, np.complex128).ravel().copy()
    bn = np.linalg.norm(b)
    res_true = b - D(x)
    info = {"iterations": 0, "converged": False, "true_rel_res": np.linalg.norm(res_true) / bn,
            "normal_res": [], "residuals": []}
    if info["true_rel_res"] <= tol:
        info["converged"] = True
        return x, info
    r = Dh(res_true)
    p = r.copy()
    rr = np.vdot(r, r).real
    for it in range(1, max_iter + 1):
        t = D(p)
        alpha = rr / np.vdot(t, t).real
        x = x + alpha * p
        r = r - alpha * Dh(t)
        if len(info["residuals"]) < 8:
            info["residuals"].append(r.copy())
        rr_new = np.vdot(r, r).real
        info["normal_res"].append(np.sqrt(rr_new))
        info["iterations"] = it
        if it % check_every == 0:
            tr = np.linalg.norm(b - D(x)) / bn
            info["true_rel_res"] = tr
            if tr <= tol:
                info["converged"] = True
                break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, info
