"""Two-site effective-Hamiltonian matvec, y = K x (the DMRG eigensolver's hot loop).

Definition (Section II-C, equation for K, in its two-site form of Section III
with the two-site tensor x^(j,j+1); tensor diagram Fig. 1d):

    y[a', t1, t2, b'] = sum  L[a', wl, a] W1[wl, t1, s1, wm] W2[wm, t2, s2, wr]
                             R[b', wr, b] x[a, s1, s2, b]

with the left environment L (the paper's A), the right environment R (the
paper's B) and the MPO site tensors W1 = H^(j), W2 = H^(j+1).

Index flows: x and y are ``(a, s1, s2, b)`` with flows (+1, +1, +1, -1);
L is ``(a', wl, a)`` and R is ``(b', wr, b)``, both with flows (-1, +1, +1),
i.e. q(a') = q(a) + q(wl) and q(b') = q(b) + q(wr); W obeys
q(wl) + q(t) - q(s) = q(wr).  MPO channels are sectors of dimension 1.

``heff_apply`` evaluates the definition block by block in the order of the
list algorithm (Algorithm 2 applied twice): contract each L block with each x
block sharing the ket sector a (step 1), combine the results with the MPO
coefficients W12 = W1 W2 summed over wm (step 2), contract with each R block
sharing the sector b (step 3).  ``heff_apply_dense`` is the same definition as
one einsum over dense embeddings, for small sizes.
"""
import numpy as np

from .blocks import BlockTensor, Index


def mpo_index(charges):
    """MPO bond index with one dimension-1 sector per channel."""
    q = np.asarray(charges).reshape(len(charges), -1)
    return Index(q, np.ones(len(q), dtype=np.int64))


def w12_pattern(W1, W2):
    """Structural nonzeros of sum_wm W1[wl,t1,s1,wm] W2[wm,t2,s2,wr].

    An entry is structurally nonzero when some wm has both W1 and W2 entries
    nonzero (no credit for numerical cancellation).  Axis order:
    [wl, t1, t2, s1, s2, wr].
    """
    b1 = (W1 != 0).astype(np.int64)
    b2 = (W2 != 0).astype(np.int64)
    return np.einsum("atsm,muvr->atusvr", b1, b2) > 0


def heff_apply(L, W1, W2, R, x, count=None, left_sectors=None):
    """y = K x by blocks.  ``count`` (a dict) receives the matmul flop counts.

    ``left_sectors``: if given, only output blocks whose first (a') sector is in this
    set are computed (the others stay zero); an output block depends only on the
    step-1 products with that a', so this is a restriction, not an approximation.

    ``count['gemm1']``: sum of 2*M*N*K over the step-1 products L-block @ x-block
    that feed a structurally nonzero W12 entry; ``count['gemm2']``: the same
    over the step-3 products Z-block @ R-block^T.
    """
    alpha, phys1, phys2, beta = x.indices
    W12 = np.einsum("atsm,muvr->atusvr", W1, W2)
    pat = w12_pattern(W1, W2)
    # which (wl, s1, s2) feed anything, and which (t1, t2, wr) they feed
    feeds = {}
    for wl, t1, t2, s1, s2, wr in zip(*np.nonzero(pat)):
        feeds.setdefault((int(wl), int(s1), int(s2)), []).append(
            (int(t1), int(t2), int(wr), float(W12[wl, t1, t2, s1, s2, wr])))
    L_by_ket = {}
    for (ip, wl, i), blk in L.blocks.items():
        L_by_ket.setdefault(i, []).append((ip, wl, blk[:, 0, :]))
    R_by_ket = {}
    for (jp, wr, j), blk in R.blocks.items():
        R_by_ket.setdefault((wr, j), []).append((jp, blk[:, 0, :]))
    g1 = 0
    g2 = 0
    # steps 1 and 2: T1 = L x, then Z = W12 . T1
    Z = {}
    for (i, s1, s2, j), xb in x.blocks.items():
        xm = xb[:, 0, 0, :]
        for ip, wl, Lm in L_by_ket.get(i, ()):
            if left_sectors is not None and ip not in left_sectors:
                continue
            f = feeds.get((wl, s1, s2))
            if not f:
                continue
            T1 = Lm @ xm
            g1 += 2 * Lm.shape[0] * Lm.shape[1] * xm.shape[1]
            for t1, t2, wr, c in f:
                key = (ip, t1, t2, wr, j)
                if key in Z:
                    Z[key] += c * T1
                else:
                    Z[key] = c * T1
    # step 3: y[ip, t1, t2, jp] += Z[ip, t1, t2, wr, j] @ R[jp, wr, j]^T
    y = BlockTensor.zeros(x.indices, x.flows, x.target)
    for (ip, t1, t2, wr, j), Zm in Z.items():
        for jp, Rm in R_by_ket.get((wr, j), ()):
            key = (ip, t1, t2, jp)
            if key not in y.blocks:
                raise AssertionError(f"output block {key} violates the charge rule")
            y.blocks[key][:, 0, 0, :] += Zm @ Rm.T
            g2 += 2 * Zm.shape[0] * Zm.shape[1] * Rm.shape[0]
    if count is not None:
        count["gemm1"] = g1
        count["gemm2"] = g2
    return y


def canonical_flops(L, W1, W2, R, x):
    """Matmul flops of ``heff_apply`` without doing the arithmetic."""
    alpha, phys1, phys2, beta = x.indices
    pat = w12_pattern(W1, W2)
    feeds = {}
    for wl, t1, t2, s1, s2, wr in zip(*np.nonzero(pat)):
        feeds.setdefault((int(wl), int(s1), int(s2)), set()).add((int(t1), int(t2), int(wr)))
    L_by_ket = {}
    for (ip, wl, i) in L.keys():
        L_by_ket.setdefault(i, []).append((ip, wl))
    R_by_ket = {}
    for (jp, wr, j) in R.keys():
        R_by_ket.setdefault((wr, j), []).append(jp)
    ad, bd = alpha.dims, beta.dims
    g1 = 0
    zkeys = set()
    for (i, s1, s2, j) in x.keys():
        for ip, wl in L_by_ket.get(i, ()):
            f = feeds.get((wl, s1, s2))
            if not f:
                continue
            g1 += 2 * int(ad[ip]) * int(ad[i]) * int(bd[j])
            for t1, t2, wr in f:
                zkeys.add((ip, t1, t2, wr, j))
    g2 = 0
    for (ip, t1, t2, wr, j) in zkeys:
        for jp in R_by_ket.get((wr, j), ()):
            g2 += 2 * int(ad[ip]) * int(bd[j]) * int(bd[jp])
    return {"gemm1": g1, "gemm2": g2, "total": g1 + g2}


def heff_apply_dense(Ld, W1, W2, Rd, xd):
    """The definition over dense arrays, one index contraction at a time.

    Equal to einsum("pwa,wtsm,muvr,qrb,asvb->ptuq"): sum over a, then wl and
    s1, then wm and s2, then wr and b.
    """
    T = np.einsum("pwa,asvb->pwsvb", Ld, xd)
    T = np.einsum("pwsvb,wtsm->ptmvb", T, W1)
    T = np.einsum("ptmvb,muvr->ptubr", T, W2)
    return np.einsum("ptubr,qrb->ptuq", T, Rd)


def heff_matrix_dense(Ld, W1, W2, Rd):
    """K as a dense matrix over (a, s1, s2, b) for tiny sizes."""
    K = np.einsum("pwa,wtsm,muvr,qrb->ptuqasvb", Ld, W1, W2, Rd, optimize=True)
    n = K.shape[0] * K.shape[1] * K.shape[2] * K.shape[3]
    return K.reshape(n, n)


def problem_from_workload(w, batch=0):
    """Oracle block tensors (L, W1, W2, R, x) for a ``workloads`` problem."""
    alpha = Index(w.alpha_q, w.alpha_d)
    beta = Index(w.beta_q, w.beta_d)
    phys = Index(w.phys, np.ones(len(w.phys), dtype=np.int64))
    wl, wr = mpo_index(w.ql), mpo_index(w.qr)
    nq = alpha.charges.shape[1]
    zero = np.zeros(nq, dtype=np.int64)
    L = BlockTensor.from_fill([alpha, wl, alpha], (-1, 1, 1), zero, w.L_block)
    R = BlockTensor.from_fill([beta, wr, beta], (-1, 1, 1), zero, w.R_block)
    x = BlockTensor.from_fill([alpha, phys, phys, beta], (1, 1, 1, -1), zero,
                              lambda k: w.x_block(k, batch))
    return L, np.array(w.W1, dtype=np.float64), np.array(w.W2, dtype=np.float64), R, x
