"""Eigensolvers for the lowest eigenpair of H_eff, in FP64.

* ``lanczos``: plain Lanczos with full modified-Gram-Schmidt
  reorthogonalisation and the tridiagonal eigenproblem solved by
  ``numpy.linalg.eigh`` (the fixed-iteration eigensolver of the 6x6 m=4096
  workload).
* ``davidson``: Algorithm 1 (Davidson routine without preconditioning).
  Readings of the printed algorithm: the projected matrix after i+1 vectors
  is the leading (i+1)x(i+1) block (the loop fills m_ij for j = 0..i); the
  basis vectors are normalised after orthogonalisation so that M is the
  projection of A; convergence is ||q|| < tol * max(1, |lambda|); when the
  orthogonalised q keeps less than 1e-12 of its norm, it is replaced by a
  seeded Gaussian vector and orthogonalised twice (the paper's
  "randomization to alleviate failed reorthogonalization").

Vectors are flat float64 arrays; ``matvec`` maps one to another.
"""
import numpy as np


def _mgs(q, basis, passes=2):
    for _ in range(passes):
        for v in basis:
            q = q - np.dot(v, q) * v
    return q


def lanczos(matvec, v0, n_iter, tol=1e-14):
    """Lowest Ritz pair after ``n_iter`` Lanczos steps (full reorthogonalisation).

    Returns ``(theta, x, info)`` with ``x`` normalised; ``info`` holds the
    tridiagonal coefficients ``alpha``, ``beta`` and the basis size.
    """
    v = v0 / np.linalg.norm(v0)
    V = [v]
    alpha, beta = [], []
    for k in range(n_iter):
        w = matvec(V[k])
        a = float(np.dot(V[k], w))
        alpha.append(a)
        w = w - a * V[k]
        if k > 0:
            w = w - beta[-1] * V[k - 1]
        w = _mgs(w, V)
        b = float(np.linalg.norm(w))
        if k == n_iter - 1 or b < tol * max(1.0, abs(a)):
            break
        beta.append(b)
        V.append(w / b)
    n = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:n - 1], 1) + np.diag(beta[:n - 1], -1)
    evals, evecs = np.linalg.eigh(T)
    s = evecs[:, 0]
    x = sum(si * vi for si, vi in zip(s, V[:n]))
    x = x / np.linalg.norm(x)
    return float(evals[0]), x, {"alpha": alpha, "beta": beta[:n - 1], "n": n}


def davidson(matvec, x0, max_vecs, tol=1e-10, seed=0):
    """Algorithm 1: lowest eigenpair of the operator ``matvec``."""
    rng = np.random.default_rng(seed)
    v0 = x0 / np.linalg.norm(x0)
    V = [v0]
    VA = [matvec(v0)]
    M = np.zeros((max_vecs, max_vecs))
    lam, x = None, v0
    for i in range(max_vecs):
        for j in range(i + 1):
            M[i, j] = M[j, i] = float(np.dot(VA[j], V[i]))
        evals, evecs = np.linalg.eigh(M[:i + 1, :i + 1])
        lam, s = float(evals[0]), evecs[:, 0]
        x = sum(sj * vj for sj, vj in zip(s, V))
        q = sum(sj * vaj for sj, vaj in zip(s, VA))
        q = q - lam * x
        if np.linalg.norm(q) < tol * max(1.0, abs(lam)) or i + 1 == max_vecs:
            break
        qn = np.linalg.norm(q)
        q = _mgs(q, V)
        if np.linalg.norm(q) < 1e-12 * qn:
            q = _mgs(rng.standard_normal(q.shape), V)
        q = q / np.linalg.norm(q)
        V.append(q)
        VA.append(matvec(q))
    return lam, x / np.linalg.norm(x)
