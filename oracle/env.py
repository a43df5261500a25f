"""Environment extension (Section II-C: the left environment A and right
environment B, built by contracting the canonical MPS sites with the MPO).

Growing the left environment by one site n with left-canonical tensor
A[a, s, b] (flows +1, +1, -1) and MPO tensor W[w, t, s, w']:

    Lnew[c, w', d] = sum  A[a, t, c] L[a, w, b] W[w, t, s, w'] A[b, s, d]

Growing the right environment by one site with right-canonical B[a, s, b]:

    Rnew[c, w, d] = sum  B[c, t, a] R[a, w', b] W[w, t, s, w'] B[d, s, b]

Both results keep the environment layout (bra, channel, ket) with flows
(-1, +1, +1).  Boundaries: the environment left of site 0 is the 1x1x1 block
on the ``start`` channel and the one right of the last site is the 1x1x1
block on the ``done`` channel.
"""
import numpy as np

from .blocks import BlockTensor, Index
from .heff import mpo_index


def left_boundary(nq):
    one = Index(np.zeros((1, nq), dtype=np.int64), [1])
    ch = Index(np.zeros((1, nq), dtype=np.int64), [1])
    t = BlockTensor([one, ch, one], (-1, 1, 1))
    t.blocks[(0, 0, 0)] = np.ones((1, 1, 1))
    return t


def right_boundary(total_charge, done_channel_charges, done_index):
    nq = len(total_charge)
    one = Index(np.asarray(total_charge).reshape(1, nq), [1])
    ch = mpo_index(done_channel_charges)
    t = BlockTensor([one, ch, one], (-1, 1, 1))
    t.blocks[(0, done_index, 0)] = np.ones((1, 1, 1))
    return t


def extend_left(L, A, W, channel_charges):
    """Lnew = A^T L W A over one site (block form)."""
    bond_out = A.indices[2]
    ch_out = mpo_index(channel_charges)
    out = BlockTensor.zeros([bond_out, ch_out, bond_out], (-1, 1, 1), L.target)
    A_by_left = {}
    for (i, s, j), blk in A.blocks.items():
        A_by_left.setdefault(i, []).append((s, j, blk[:, 0, :]))
    nz = np.argwhere(W != 0)
    W_by_ws = {}
    for w, t, s, wp in nz:
        W_by_ws.setdefault((int(w), int(t), int(s)), []).append((int(wp), float(W[w, t, s, wp])))
    for (ip, w, i), Lb in L.blocks.items():
        Lm = Lb[:, 0, :]
        for s, j, Aket in A_by_left.get(i, ()):
            LA = Lm @ Aket                      # [m_ip x m_j]
            for t, jpp, Abra in A_by_left.get(ip, ()):
                terms = W_by_ws.get((w, t, s))
                if not terms:
                    continue
                blk = Abra.T @ LA                # [m_jpp x m_j]
                for wp, c in terms:
                    out.blocks[(jpp, wp, j)][:, 0, :] += c * blk
    return out


def extend_right(R, B, W, channel_charges):
    """Rnew = B R W B^T over one site (block form)."""
    bond_out = B.indices[0]
    ch_out = mpo_index(channel_charges)
    out = BlockTensor.zeros([bond_out, ch_out, bond_out], (-1, 1, 1), R.target)
    B_by_right = {}
    for (i, s, j), blk in B.blocks.items():
        B_by_right.setdefault(j, []).append((i, s, blk[:, 0, :]))
    nz = np.argwhere(W != 0)
    W_by_ts = {}
    for w, t, s, wp in nz:
        W_by_ts.setdefault((int(t), int(s), int(wp)), []).append((int(w), float(W[w, t, s, wp])))
    for (jp, wp, j), Rb in R.blocks.items():
        Rm = Rb[:, 0, :]
        for i, s, Bket in B_by_right.get(j, ()):
            RB = Rm @ Bket.T                     # [m_jp x m_i]
            for ipp, t, Bbra in B_by_right.get(jp, ()):
                terms = W_by_ts.get((t, s, wp))
                if not terms:
                    continue
                blk = Bbra @ RB                  # [m_ipp x m_i]
                for w, c in terms:
                    out.blocks[(ipp, w, i)][:, 0, :] += c * blk
    return out


def extend_left_dense(Ld, Ad, W):
    return np.einsum("atc,awb,wtsv,bsd->cvd", Ad, Ld, W, Ad, optimize=True)


def extend_right_dense(Rd, Bd, W):
    return np.einsum("cta,avb,wtsv,dsb->cwd", Bd, Rd, W, Bd, optimize=True)
