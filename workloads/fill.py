"""Seeded block values and the named synthetic H_eff workloads.

Every block is drawn from its own NumPy generator seeded by
``(seed, tag, *sector_key)``, so a block's values depend only on its key and
not on the order in which a caller enumerates blocks.  Environment blocks are
made symmetric under transposition combined with the MPO channel map
``w -> conj(w)`` (the relation ``L[a', w, a] = L[a, conj(w), a']`` that the
environments of a real MPS satisfy, Section II-C), and the identity channel of
an environment (``start`` on the left, ``done`` on the right) is the block
identity, as it is for a canonical MPS.
"""
from dataclasses import dataclass
import numpy as np

from .sectors import (binomial_sectors, paper_model_sectors, electron_sectors,
                      spin_phys, electron_phys)
from .mpo import (heisenberg_mpo, hubbard_mpo, chain_pairs, cylinder_pairs, cylinder_hops, triangular_hops,
                  bulk_window, compress_mpo)

TAG_L, TAG_R, TAG_X, TAG_SITE = 1, 2, 3, 4


def site_block(seed, key, shape):
    """Gaussian block of an MPS site tensor T[a, s, b] (key = (a, s, b) sectors)."""
    return gaussian_block(seed, TAG_SITE, key, shape)


def gaussian_block(seed, tag, key, shape):
    """Standard-normal block drawn from a generator keyed by (seed, tag, key)."""
    ss = np.random.SeedSequence([int(seed), int(tag)] + [int(k) for k in key])
    return np.random.default_rng(ss).standard_normal(shape)


def env_block(seed, tag, key, shape_fn, conj, ident, scale):
    """Symmetrised Gaussian environment block for ``key = (row, w, col)``.

    ``shape_fn(row, col)`` gives the block shape, ``conj`` maps MPO channels
    to their transpose partner and ``ident`` is the identity channel.
    Returns ``scale * (X[row,w,col] + X[col,conj(w),row]^T) / 2``, or the
    identity on the identity channel.
    """
    r, w, c = key
    shape = shape_fn(r, c)
    if w == ident:
        if r != c:
            return np.zeros(shape)
        return np.eye(shape[0])
    X = gaussian_block(seed, tag, (r, w, c), shape)
    wc = int(conj[w])
    if wc < 0:
        return scale * X
    Y = gaussian_block(seed, tag, (c, wc, r), (shape[1], shape[0]))
    return scale * 0.5 * (X + Y.T)


def assemble_flat(blocks, fill, total, dtype=np.float64):
    """Write ``fill(key)`` for each ``(key, offset, size)`` into a flat array."""
    out = np.zeros(int(total), dtype=dtype)
    for key, off, size in blocks:
        v = np.asarray(fill(tuple(int(k) for k in key)), dtype=np.float64).reshape(-1)
        if v.size != size:
            raise ValueError(f"block {key}: fill gave {v.size} values, layout wants {size}")
        out[int(off):int(off) + int(size)] = v
    return out


@dataclass
class HeffWorkload:
    """Inputs of one two-site effective-Hamiltonian problem.

    Bonds: ``alpha`` (left, charges ``[n,nq]`` and dims), ``beta`` (right);
    physical charges ``phys``; MPO site tensors ``W1[wl,t1,s1,wm]`` and
    ``W2[wm,t2,s2,wr]`` with channel charges ``ql, qm, qr``; transposition
    maps ``conj_l, conj_r`` of the environment channels; identity channels
    ``start_l`` (left) and ``done_r`` (right).  The two-site tensor has
    indices ``(a, s1, s2, b)`` and total charge ``target``.
    """
    name: str
    alpha_q: np.ndarray
    alpha_d: np.ndarray
    beta_q: np.ndarray
    beta_d: np.ndarray
    phys: np.ndarray
    W1: np.ndarray
    W2: np.ndarray
    ql: np.ndarray
    qm: np.ndarray
    qr: np.ndarray
    conj_l: np.ndarray
    conj_r: np.ndarray
    start_l: int
    done_r: int
    seed: int
    env_scale: float
    labels_m: tuple = ()

    @property
    def nq(self):
        return self.alpha_q.shape[1]

    @property
    def target(self):
        return np.zeros(self.nq, dtype=np.int32)

    @property
    def m(self):
        return int(self.alpha_d.sum())

    def L_block(self, key):
        """Block ``L[a' in key[0], wl = key[1], a in key[2]]`` as a matrix."""
        d = self.alpha_d
        return env_block(self.seed, TAG_L, key, lambda r, c: (int(d[r]), int(d[c])),
                         self.conj_l, self.start_l, self.env_scale)

    def R_block(self, key):
        """Block ``R[b' in key[0], wr = key[1], b in key[2]]`` as a matrix."""
        d = self.beta_d
        return env_block(self.seed, TAG_R, key, lambda r, c: (int(d[r]), int(d[c])),
                         self.conj_r, self.done_r, self.env_scale)

    def x_block(self, key, batch=0):
        """Block ``x[a in key[0], s1, s2, b in key[3]]`` as a matrix."""
        i, s1, s2, j = key
        return gaussian_block(self.seed + 1000 * batch, TAG_X, key,
                              (int(self.alpha_d[i]), int(self.beta_d[j])))

    def W1_entry(self, key):
        return self.W1[key]

    def W2_entry(self, key):
        return self.W2[key]


SPIN_COUPLINGS = (1.0, 0.5, 0.2, 0.1)   # J_1 (nearest), J_2 (tagged "J2"), J_3, J_4


def spin_window(couplings=SPIN_COUPLINGS):
    """Bulk two-site window of the range-R spin chain MPO (k = 2 + 3R)."""
    R = len(couplings)
    n = 2 * R + 4
    mpo = heisenberg_mpo(n, chain_pairs(n, list(couplings)))
    return bulk_window(mpo, R + 1)


def _compressed(mpo, compress):
    """compress: False (the automaton), True or "svd" (the SVD basis), "interpolative" (a
    subset of the automaton's channels; the same channel counts with a sparser W)."""
    if not compress:
        return mpo
    return compress_mpo(mpo, method="svd" if compress is True else compress)


def _widest_window(mpo):
    """The two-site window at the first bond triple with the largest total channel count."""
    n = mpo.n_sites
    best = max(range(n - 1), key=lambda s: (mpo.bond_dim(s) + mpo.bond_dim(s + 1) + mpo.bond_dim(s + 2), -s))
    return bulk_window(mpo, best)


def lattice_window(Lx=6, Ly=6, J1=1.0, J2=0.5, compress=False):
    """Two-site window of the snake-ordered Lx x Ly J1-J2 Heisenberg cylinder MPO (the
    paper's spin lattice, Section V), at the first bond triple with the largest total
    channel count (the MPO's k there: 26 on all three bonds for 6 x 6).  compress=True
    takes the window of the MPO compressed at the paper's SVD cutoff of 1e-13 (Section VI-B;
    k = 20 for 6 x 6, 32 for 20 x 10)."""
    n = Lx * Ly
    mpo = heisenberg_mpo(n, cylinder_pairs(Lx, Ly, J1, J2))
    return _widest_window(_compressed(mpo, compress))


def electron_window(t=1.0, U=8.0, R=5):
    """Bulk two-site window of the range-R Hubbard chain MPO (k = 2 + 4R).

    Hopping ``t`` acts between sites at every distance ``r <= R`` with
    amplitude ``t / r`` (a stand-in for the longer-range hops a snake-ordered
    cylinder produces), plus the on-site ``U n_up n_dn``.
    """
    n = 2 * R + 4
    hops = []
    for r in range(1, R + 1):
        for i in range(n - r):
            hops.append((i, i + r, t / r))
    mpo = hubbard_mpo(n, hops, U)
    return bulk_window(mpo, R + 1)


def hubbard_lattice_window(Lx=8, Ly=4, t=1.0, U=8.0):
    """Two-site window of the snake-ordered Lx x Ly Hubbard cylinder MPO (nearest-neighbour
    hopping t, on-site U; the electron lattice of Section V, here 4 x 8 as a 32-site MPS), at
    the first bond triple with the largest total channel count."""
    n = Lx * Ly
    mpo = hubbard_mpo(n, cylinder_hops(Lx, Ly, t), U)
    best = max(range(n - 1), key=lambda s: (mpo.bond_dim(s) + mpo.bond_dim(s + 1) + mpo.bond_dim(s + 2), -s))
    return bulk_window(mpo, best)


def triangular_hubbard_window(Lx=6, Ly=6, t=1.0, U=8.5, compress=False):
    """Two-site window of the snake-ordered Lx x Ly triangular Hubbard cylinder MPO (the
    paper's electron lattice of Section V, 6 x 6 with U = 8.5), at the first bond triple
    with the largest total channel count.  compress=True: of the MPO compressed at the SVD
    cutoff 1e-13 (Section VI-B: k = 26, the paper's figure for this lattice)."""
    n = Lx * Ly
    mpo = hubbard_mpo(n, triangular_hops(Lx, Ly, t), U)
    return _widest_window(_compressed(mpo, compress))


def spin_heff_workload(m, nsec, seed=0, model="binomial", couplings=SPIN_COUPLINGS,
                       name=None, window=None):
    """Spin-1/2 two-site H_eff inputs.

    ``model="binomial"``: left/right bonds from ``binomial_sectors`` with
    seeds ``seed`` and ``seed+1``, tensors from ``seed+2``.
    ``model="paper"``: both bonds from the block-size model of Table II.
    """
    if model == "binomial":
        aq, ad = binomial_sectors(m, nsec, seed)
        bq, bd = binomial_sectors(m, nsec, seed + 1)
    elif model == "paper":
        aq, ad = paper_model_sectors(m)
        bq, bd = paper_model_sectors(m)
    else:
        raise ValueError(model)
    win = spin_window(couplings) if window is None else window
    return HeffWorkload(
        name=name or f"spin_{model}_m{m}", alpha_q=aq, alpha_d=ad, beta_q=bq, beta_d=bd,
        phys=spin_phys(), W1=win["W1"], W2=win["W2"], ql=win["ql"], qm=win["qm"],
        qr=win["qr"], conj_l=win["conj_l"], conj_r=win["conj_r"], start_l=win["start_l"],
        done_r=win["done_r"], seed=seed + 2, env_scale=1.0 / np.sqrt(max(m, 1)),
        labels_m=tuple(win["labels_m"]))


def electron_heff_workload(m, seed=0, n_center=16, max_block=256, name=None, span=5, window=None):
    """Hubbard two-site H_eff inputs on (N, 2Sz) charges (d = 4; k = 22 for the default
    range-5 chain window, or the MPO window passed in)."""
    aq, ad = electron_sectors(m, seed, n_center, span, span, max_block=max_block)
    bq, bd = electron_sectors(m, seed + 1, n_center + 2, span, span, max_block=max_block)
    win = electron_window() if window is None else window
    return HeffWorkload(
        name=name or f"electron_m{m}", alpha_q=aq, alpha_d=ad, beta_q=bq, beta_d=bd,
        phys=electron_phys(), W1=win["W1"], W2=win["W2"], ql=win["ql"], qm=win["qm"],
        qr=win["qr"], conj_l=win["conj_l"], conj_r=win["conj_r"], start_l=win["start_l"],
        done_r=win["done_r"], seed=seed + 2, env_scale=1.0 / np.sqrt(max(m, 1)),
        labels_m=tuple(win["labels_m"]))


def workload_by_name(name):
    """Named workloads: the 6x6 J1-J2 stand-ins at m=1024/4096 and the
    electron workload at m=2048, plus small cases used by parity tests."""
    table = {
        "spin_m1024": lambda: spin_heff_workload(1024, 30, 0, name="spin_m1024"),
        "spin_m4096": lambda: spin_heff_workload(4096, 40, 0, name="spin_m4096"),
        "spin_paper_m4096": lambda: spin_heff_workload(4096, 0, 0, model="paper",
                                                       name="spin_paper_m4096"),
        "spin_j1j2_6x6_m1024": lambda: spin_heff_workload(1024, 30, 0, name="spin_j1j2_6x6_m1024",
                                                          window=lattice_window()),
        "spin_j1j2_6x6_m4096": lambda: spin_heff_workload(4096, 40, 0, name="spin_j1j2_6x6_m4096",
                                                          window=lattice_window()),
        "spin_j1j2_6x6_m200": lambda: spin_heff_workload(200, 10, 7, name="spin_j1j2_6x6_m200",
                                                         window=lattice_window()),
        "spin_j1j2_20x10_m4096": lambda: spin_heff_workload(4096, 40, 0, name="spin_j1j2_20x10_m4096",
                                                            window=lattice_window(20, 10)),
        "spin_j1j2_20x10_m200": lambda: spin_heff_workload(200, 10, 7, name="spin_j1j2_20x10_m200",
                                                           window=lattice_window(20, 10)),
        "electron_tri_xc6_m2048": lambda: electron_heff_workload(2048, 0, name="electron_tri_xc6_m2048",
                                                                 window=triangular_hubbard_window()),
        # the paper's lattices with their MPOs compressed at the SVD cutoff 1e-13 (Section VI-B)
        "spin_j1j2_20x10c_m4096": lambda: spin_heff_workload(4096, 40, 0, name="spin_j1j2_20x10c_m4096",
                                                             window=lattice_window(20, 10, compress=True)),
        "spin_j1j2_20x10c_m200": lambda: spin_heff_workload(200, 10, 7, name="spin_j1j2_20x10c_m200",
                                                            window=lattice_window(20, 10, compress=True)),
        "electron_tri_xc6c_m2048": lambda: electron_heff_workload(2048, 0, name="electron_tri_xc6c_m2048",
                                                                  window=triangular_hubbard_window(compress=True)),
        "electron_tri_xc6c_m96": lambda: electron_heff_workload(96, 3, n_center=6, max_block=24,
                                                                name="electron_tri_xc6c_m96",
                                                                window=triangular_hubbard_window(compress=True)),
        # the same compressions keeping a subset of the automaton's channels (a sparser W)
        "spin_j1j2_20x10ci_m4096": lambda: spin_heff_workload(
            4096, 40, 0, name="spin_j1j2_20x10ci_m4096", window=lattice_window(20, 10, compress="interpolative")),
        "spin_j1j2_20x10ci_m200": lambda: spin_heff_workload(
            200, 10, 7, name="spin_j1j2_20x10ci_m200", window=lattice_window(20, 10, compress="interpolative")),
        "electron_tri_xc6ci_m2048": lambda: electron_heff_workload(
            2048, 0, name="electron_tri_xc6ci_m2048", window=triangular_hubbard_window(compress="interpolative")),
        "electron_tri_xc6ci_m96": lambda: electron_heff_workload(
            96, 3, n_center=6, max_block=24, name="electron_tri_xc6ci_m96",
            window=triangular_hubbard_window(compress="interpolative")),
        "electron_tri_xc6_m96": lambda: electron_heff_workload(96, 3, n_center=6, max_block=24,
                                                               name="electron_tri_xc6_m96",
                                                               window=triangular_hubbard_window()),
        "electron_m2048": lambda: electron_heff_workload(2048, 0, name="electron_m2048"),
        "electron_hubbard_4x8_m2048": lambda: electron_heff_workload(2048, 0, name="electron_hubbard_4x8_m2048",
                                                                     window=hubbard_lattice_window()),
        "electron_hubbard_4x8_m96": lambda: electron_heff_workload(96, 3, n_center=6, max_block=24,
                                                                   name="electron_hubbard_4x8_m96",
                                                                   window=hubbard_lattice_window()),
        "spin_m24": lambda: spin_heff_workload(24, 6, 9, name="spin_m24"),
        "spin_m64": lambda: spin_heff_workload(64, 8, 5, name="spin_m64"),
        "spin_m200": lambda: spin_heff_workload(200, 10, 7, name="spin_m200"),
        "spin_m384": lambda: spin_heff_workload(384, 12, 11, name="spin_m384"),
        "electron_m40": lambda: electron_heff_workload(40, 13, n_center=4, max_block=8, span=2,
                                                       name="electron_m40"),
        "electron_m96": lambda: electron_heff_workload(96, 3, n_center=6, max_block=24,
                                                       name="electron_m96"),
        "electron_m256": lambda: electron_heff_workload(256, 5, n_center=8, max_block=48,
                                                        name="electron_m256"),
    }
    return table[name]()
