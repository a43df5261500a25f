"""Gradients of the Rayleigh quotient rho = <x|K|x> / <x|x> of H_eff.

K is the two-site effective Hamiltonian of ``heff`` (Section II-C).  With
y = K x and n = <x|x> (real tensors, K symmetric):

* d rho / d x  = 2 (K x - rho x) / n;
* rho is linear in each of L, W1, W2, R, so every other gradient is the
  contraction of the bra x, the ket x and the remaining three operators:

    d rho / d L[a', wl, a]  = sum x[a',t1,t2,b'] W1 W2 R[b',wr,b] x[a,s1,s2,b] / n
    d rho / d R[b', wr, b]  = sum x[a',t1,t2,b'] L[a',wl,a] W1 W2 x[a,s1,s2,b] / n
    G[wl,t1,t2,s1,s2,wr]    = sum x[a',t1,t2,b'] L[a',wl,a] R[b',wr,b] x[a,s1,s2,b] / n
    d rho / d W1[wl,t1,s1,wm] = sum_{t2,s2,wr} G W2[wm,t2,s2,wr]
    d rho / d W2[wm,t2,s2,wr] = sum_{wl,t1,s1} G W1[wl,t1,s1,wm]

  The gradient with respect to a coupling J that the MPO tensors depend on
  is sum dW1 * dW1/dJ + sum dW2 * dW2/dJ (through W1 and W2 only; L and R are
  independent inputs).
"""
import numpy as np

from .blocks import BlockTensor
from .heff import heff_apply


def rayleigh(L, W1, W2, R, x):
    y = heff_apply(L, W1, W2, R, x)
    return x.vdot(y) / x.vdot(x), y


def grad_x(L, W1, W2, R, x):
    rho, y = rayleigh(L, W1, W2, R, x)
    n = x.vdot(x)
    g = y.copy().axpy(-rho, x).scale(2.0 / n)
    return rho, g


def _L_by_ket(L):
    d = {}
    for (ip, wl, i), blk in L.blocks.items():
        d.setdefault(i, []).append((ip, wl, blk[:, 0, :]))
    return d


def grad_all(L, W1, W2, R, x):
    """rho and its gradients (dx, dL, dR, dW1, dW2) by blocks."""
    n = x.vdot(x)
    rho, dx = grad_x(L, W1, W2, R, x)
    W12 = np.einsum("atsm,muvr->atusvr", W1, W2)
    kl, d1, d2 = W1.shape[0], W1.shape[1], W2.shape[1]
    kr = W2.shape[3]
    G = np.zeros((kl, d1, d2, d1, d2, kr))
    dL = BlockTensor.zeros(L.indices, L.flows, L.target)
    dR = BlockTensor.zeros(R.indices, R.flows, R.target)
    R_by_ket = {}
    for (jp, wr, j), blk in R.blocks.items():
        R_by_ket.setdefault(j, []).append((jp, wr, blk[:, 0, :]))
    Lk = _L_by_ket(L)
    for (i, s1, s2, j), xb in x.blocks.items():
        xk = xb[:, 0, 0, :]
        for ip, wl, Lm in Lk.get(i, ()):
            T1 = Lm @ xk                               # [a', b]
            for jp, wr, Rm in R_by_ket.get(j, ()):
                for t1 in range(d1):
                    for t2 in range(d2):
                        bra = x.blocks.get((ip, t1, t2, jp))
                        if bra is None:
                            continue
                        xb_ = bra[:, 0, 0, :]            # [a', b']
                        c = W12[wl, t1, t2, s1, s2, wr]
                        G[wl, t1, t2, s1, s2, wr] += float(np.sum(xb_ * (T1 @ Rm.T)))
                        if c == 0.0:
                            continue
                        # dL[a', wl, a] += c * xb_ R x^T
                        dL.blocks[(ip, wl, i)][:, 0, :] += c * (xb_ @ Rm @ xk.T) / n
                        # dR[b', wr, b] += c * xb_^T L x
                        dR.blocks[(jp, wr, j)][:, 0, :] += c * (xb_.T @ T1) / n
    G /= n
    dW1 = np.einsum("atusvr,muvr->atsm", G, W2)
    dW2 = np.einsum("atusvr,atsm->muvr", G, W1)
    return {"rho": rho, "dx": dx, "dL": dL, "dR": dR, "dW1": dW1, "dW2": dW2, "G": G}
