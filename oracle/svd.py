"""Block SVD split of the two-site tensor with truncation (Section IV, Fig. 1e).

The two-site tensor x[a, s1, s2, b] is wrapped into a matrix with rows (a, s1)
and columns (s2, b).  Rows and columns sharing one charge Q = q(a) + q(s1) =
q(b) - q(s2) form one dense block, decomposed by SVD.  The new bond index
carries one sector per Q with as many states as singular values kept.

Readings of the truncation rule (Section II-C "removes all singular values
below 1e-12"; Section VI SVD cutoffs): on x / ||x||, singular values below
``cutoff`` are dropped, then at most ``m_max`` of the largest are kept;
when values tie within 1e-12 * s_max at the cut, the order is decided by
(|Q|, Q, index inside the block).  Singular values are absorbed into the
right factor for a left-to-right sweep and into the left factor otherwise.
"""
import numpy as np

from .blocks import BlockTensor, Index


def svd_split(x, m_max, cutoff=1e-12, absorb="right"):
    """Return (A[a,s1,c], B[c,s2,b], kept singular values, discarded weight)."""
    alpha, phys1, phys2, beta = x.indices
    nrm = x.norm()
    groups = {}
    for (i, s1, s2, j), blk in x.blocks.items():
        Q = tuple(alpha.charges[i] + phys1.charges[s1])
        g = groups.setdefault(Q, {"rows": set(), "cols": set()})
        g["rows"].add((i, s1))
        g["cols"].add((s2, j))
    cand = []
    dec = {}
    for Q, g in groups.items():
        rows = sorted(g["rows"])
        cols = sorted(g["cols"])
        roff, o = {}, 0
        for r in rows:
            roff[r] = o
            o += int(alpha.dims[r[0]])
        nr = o
        coff, o = {}, 0
        for c in cols:
            coff[c] = o
            o += int(beta.dims[c[1]])
        nc = o
        M = np.zeros((nr, nc))
        for (i, s1) in rows:
            for (s2, j) in cols:
                key = (i, s1, s2, j)
                if key in x.blocks:
                    M[roff[(i, s1)]:roff[(i, s1)] + alpha.dims[i],
                      coff[(s2, j)]:coff[(s2, j)] + beta.dims[j]] = x.blocks[key][:, 0, 0, :]
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        dec[Q] = (rows, roff, cols, coff, U, S, Vt)
        for n, s in enumerate(S):
            cand.append((s / nrm if nrm > 0 else 0.0, Q, n))
    smax = max((c[0] for c in cand), default=0.0)
    cand.sort(key=lambda c: (-round(c[0] / max(smax, 1e-300) / 1e-12), sum(abs(v) for v in c[1]),
                             c[1], c[2]))
    kept = [c for c in cand if c[0] >= cutoff][:m_max]
    disc = float(sum(c[0] ** 2 for c in cand) - sum(c[0] ** 2 for c in kept))
    keep_by_Q = {}
    for s, Q, n in kept:
        keep_by_Q.setdefault(Q, []).append(n)
    Qs = sorted(keep_by_Q)
    nq = alpha.charges.shape[1]
    bond = Index(np.array(Qs, dtype=np.int64).reshape(-1, nq), [len(keep_by_Q[Q]) for Q in Qs])
    A = BlockTensor([alpha, phys1, bond], (1, 1, -1), np.zeros(nq, dtype=np.int64))
    B = BlockTensor([bond, phys2, beta], (1, 1, -1), np.zeros(nq, dtype=np.int64))
    svals = []
    for c, Q in enumerate(Qs):
        rows, roff, cols, coff, U, S, Vt = dec[Q]
        sel = sorted(keep_by_Q[Q])
        Us, Ss, Vs = U[:, sel], S[sel], Vt[sel, :]
        svals.extend(Ss.tolist())
        if absorb == "right":
            Vs = Ss[:, None] * Vs
        else:
            Us = Us * Ss[None, :]
        for (i, s1) in rows:
            A.blocks[(i, s1, c)] = Us[roff[(i, s1)]:roff[(i, s1)] + alpha.dims[i]][:, None, :].copy()
        for (s2, j) in cols:
            B.blocks[(c, s2, j)] = Vs[:, coff[(s2, j)]:coff[(s2, j)] + beta.dims[j]][:, None, :].copy()
    return A, B, np.array(svals), disc
