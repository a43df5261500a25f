"""Bond sector lists (charge tuple, dimension) for the synthetic workloads.

A bond index is given as ``(charges, dims)``: ``charges`` is an int32 array of
shape ``[nsec, nq]`` (one U(1) charge per column) and ``dims`` an int32 array of
shape ``[nsec]``, every entry at least 1.

Charges use integer units: ``2 Sz`` for spin-1/2 chains (a site carries +1 or
-1) and ``(N, 2 Sz)`` for electrons (a site carries (0,0), (1,1), (1,-1) or
(2,0)).  These are the U(1) and U(1)xU(1) labels of the paper's Section II-D
and Section V (spin models conserve Sz; the Hubbard model conserves particle
number and Sz).
"""
import numpy as np
from scipy.stats import binom


def _multinomial_at_least_one(rng, m, p):
    """Draw sector dimensions summing to ``m`` with every sector at least 1."""
    n = len(p)
    if m < n:
        raise ValueError("bond dimension smaller than the number of sectors")
    p = np.asarray(p, dtype=np.float64)
    p = p / p.sum()
    return (rng.multinomial(m - n, p) + 1).astype(np.int32)


def binomial_sectors(m, nsec, seed, parity=1):
    """Spin bond with ``nsec`` sectors of charge 2Sz in steps of 2.

    Charges run over ``-(nsec-1) .. nsec-1`` when ``parity`` is 1 (odd values
    for an even ``nsec``); dimensions are multinomial(m, Binom(nsec-1, 1/2)) with
    each sector at least 1, drawn from ``seed``.
    """
    q = 2 * np.arange(nsec, dtype=np.int32) - (nsec - 1)
    if (q[0] % 2 != 0) != bool(parity % 2):
        q = q + 1
    rng = np.random.default_rng(seed)
    dims = _multinomial_at_least_one(rng, m, binom.pmf(np.arange(nsec), nsec - 1, 0.5))
    return q.reshape(-1, 1).astype(np.int32), dims


def paper_model_sectors(m, q=4.0, r=0.6):
    """Block-size model of the paper's Table II: b_l = floor((m/q) r^|l|).

    Sectors with b_l >= 1 are kept; charges are 2l (even 2Sz values).
    """
    dims = []
    ls = []
    lmax = 0
    while int(np.floor((m / q) * r ** (lmax + 1))) >= 1:
        lmax += 1
    for l in range(-lmax, lmax + 1):
        ls.append(2 * l)
        dims.append(int(np.floor((m / q) * r ** abs(l))))
    return (np.array(ls, dtype=np.int32).reshape(-1, 1),
            np.array(dims, dtype=np.int32))


def electron_sectors(m, seed, n_center, nspan=5, sspan=5, max_block=256):
    """Electron bond on a 2-D (N, 2Sz) charge grid.

    Cells are ``N = n_center + n`` for ``|n| <= nspan`` and ``2Sz = s`` for
    ``|s| <= sspan`` with ``s`` of the same parity as ``N``.  Weights are the
    product of Binom(2 nspan, 1/2) and Binom(2 sspan, 1/2) probabilities;
    dimensions are multinomial(m) with each at least 1, then clipped to
    ``max_block`` with the excess handed to unclipped cells in proportion to
    their weight (repeated until nothing exceeds the cap).
    """
    cells = []
    w = []
    pn = binom.pmf(np.arange(2 * nspan + 1), 2 * nspan, 0.5)
    ps = binom.pmf(np.arange(2 * sspan + 1), 2 * sspan, 0.5)
    for n in range(-nspan, nspan + 1):
        N = n_center + n
        for s in range(-sspan, sspan + 1):
            if (s - N) % 2 != 0:
                continue
            cells.append((N, s))
            w.append(pn[n + nspan] * ps[s + sspan])
    w = np.array(w)
    rng = np.random.default_rng(seed)
    dims = _multinomial_at_least_one(rng, m, w).astype(np.int64)
    for _ in range(64):
        over = dims > max_block
        if not over.any():
            break
        excess = int((dims[over] - max_block).sum())
        dims[over] = max_block
        free = ~over & (dims < max_block)
        if not free.any():
            break
        extra = rng.multinomial(excess, w[free] / w[free].sum())
        dims[free] += extra
    dims = np.minimum(dims, max_block)
    return np.array(cells, dtype=np.int32), dims.astype(np.int32)


def spin_phys():
    """Spin-1/2 site: state 0 = up (2Sz=+1), state 1 = down (2Sz=-1)."""
    return np.array([[1], [-1]], dtype=np.int32)


def electron_phys():
    """Hubbard site: |0>, |up>, |dn>, |up dn> with charges (N, 2Sz)."""
    return np.array([[0, 0], [1, 1], [1, -1], [2, 0]], dtype=np.int32)
