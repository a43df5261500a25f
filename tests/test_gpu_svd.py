"""GPU block SVD split with truncation (heff_svd_*) against the oracle's svd_split.

The oracle's truncation is pinned by 'squared reconstruction error = discarded weight'
and exact reconstruction without truncation (tests/test_oracle_eig_svd_dmrg_grad.py).
Here, on the same two-site tensor: the new bond (charges, dimensions), the kept singular
values and the discarded weight equal the oracle's, the product of the two factors equals
the oracle's truncated tensor (unique when the cut does not split a degenerate multiplet;
singular vectors themselves carry a sign freedom), and the factor without the singular
values is an isometry.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import heff as oh, svd as osvd, mps as omps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff              # noqa: E402
from tests.helpers import library_problem             # noqa: E402


def _product(A_l, B_l, A, B, x_l):
    """Contract A[a,s1,c] B[c,s2,b] into x's layout (numpy, per block)."""
    Ab = {k: A[o:o + n] for k, o, n in A_l.blocks()}
    Bb = {k: B[o:o + n] for k, o, n in B_l.blocks()}
    ad = A_l.indices[0][1]
    cd = A_l.indices[2][1]
    bd = B_l.indices[2][1]

    def fill(k):
        i, s1, s2, j = k
        acc = np.zeros((ad[i], bd[j]))
        for c in range(len(cd)):
            a = Ab.get((i, s1, c))
            b = Bb.get((c, s2, j))
            if a is not None and b is not None:
                acc += a.reshape(ad[i], cd[c]) @ b.reshape(cd[c], bd[j])
        return acc
    return x_l.assemble(fill)


@pytest.mark.parametrize("name,m_max,cutoff,absorb_right", [
    ("spin_m64", 24, 1e-12, True), ("spin_m64", 10 ** 6, 0.0, False), ("electron_m96", 40, 1e-12, True),
    ("spin_m200", 120, 1e-3, False), ("spin_m1024", 1024, 1e-12, True)])
def test_svd_split_matches_oracle(name, m_max, cutoff, absorb_right):
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    x_l = lays[4]
    L, W1, W2, R, xo = oh.problem_from_workload(w)
    A_o, B_o, s_o, disc_o = osvd.svd_split(xo, m_max, cutoff, "right" if absorb_right else "left")
    s = heff.heff_svd_create(x_l.handle)
    try:
        ws = torch.empty(heff.heff_svd_workspace_size(s), dtype=torch.uint8, device="cuda")
        x = torch.from_numpy(bufs["x"][0]).to("cuda", torch.float64)
        sweeps = heff.heff_svd_compute(s, x, ws)
        q, d, disc, nrm = heff.heff_svd_truncate(s, m_max, cutoff, w.nq, 4096)
        bond_o = A_o.indices[2]
        assert np.array_equal(q, bond_o.charges) and np.array_equal(d, bond_o.dims)
        sv = heff.heff_svd_singular_values(s, int(d.sum()))
        assert np.abs(sv / nrm - s_o / xo.norm()).max() < 1e-12 * (s_o.max() / xo.norm())
        assert abs(disc - disc_o) < 1e-12
        ones = np.ones(len(w.phys), dtype=np.int32)
        A_l = heff.Layout([(w.alpha_q, w.alpha_d, 1), (w.phys, ones, 1), (q, d, -1)])
        B_l = heff.Layout([(q, d, 1), (w.phys, ones, 1), (w.beta_q, w.beta_d, -1)])
        A = torch.full((A_l.nelem,), float("nan"), dtype=torch.float64, device="cuda")
        B = torch.full((B_l.nelem,), float("nan"), dtype=torch.float64, device="cuda")
        heff.heff_svd_write(s, A_l.handle, B_l.handle, A, B, absorb_right, ws)
        A, B = A.cpu().numpy(), B.cpu().numpy()
        assert not np.isnan(A).any() and not np.isnan(B).any()
        y = _product(A_l, B_l, A, B, x_l)
        x_trunc = omps.two_site(A_o, B_o)
        y_o = x_l.assemble(lambda k: x_trunc.blocks[k])
        err = np.linalg.norm(y - y_o) / np.linalg.norm(y_o)
        print(f"{name} m_max={m_max}: kept {int(d.sum())}, sweeps {sweeps}, discarded {disc:.3e}, "
              f"product rel err {err:.2e}")
        assert err < 1e-10
        # the factor without singular values is an isometry per new-bond sector
        iso_l, iso = (A_l, A) if absorb_right else (B_l, B)
        for c in range(len(d)):
            if absorb_right:
                M = np.vstack([iso[o:o + n].reshape(-1, d[c]) for k, o, n in iso_l.blocks() if k[2] == c])
                G = M.T @ M
            else:
                M = np.hstack([iso[o:o + n].reshape(d[c], -1) for k, o, n in iso_l.blocks() if k[0] == c])
                G = M @ M.T
            assert np.abs(G - np.eye(d[c])).max() < 1e-10
    finally:
        heff.heff_svd_destroy(s)


def _gpu_svd(x_l, xflat, m_max, cutoff, nq):
    s = heff.heff_svd_create(x_l.handle)
    try:
        ws = torch.empty(heff.heff_svd_workspace_size(s), dtype=torch.uint8, device="cuda")
        heff.heff_svd_compute(s, torch.from_numpy(xflat).to("cuda", torch.float64), ws)
        q, d, disc, nrm = heff.heff_svd_truncate(s, m_max, cutoff, nq, 4096)
        sv = heff.heff_svd_singular_values(s, max(1, int(d.sum())))[:int(d.sum())]
        return q, d, disc, nrm, sv
    finally:
        heff.heff_svd_destroy(s)


def test_svd_of_rank_one_tensor():
    """Degenerate input: the oracle's rank-1 truncation of a two-site tensor (one singular
    triplet in one charge sector, every other sector exactly zero).  The GPU keeps exactly
    that triplet at the cutoff 1e-12: the same bond, singular value and norm."""
    w = wl.workload_by_name("spin_m200")
    lays, bufs = library_problem(w)
    x_l = lays[4]
    L, W1, W2, R, xo = oh.problem_from_workload(w)
    A1, B1, s1, _ = osvd.svd_split(xo, 1, 0.0, "right")
    x1 = omps.two_site(A1, B1)
    xflat = x_l.assemble(lambda k: x1.blocks[k])
    A_o, B_o, s_o, disc_o = osvd.svd_split(x1, 64, 1e-12, "right")
    q, d, disc, nrm, sv = _gpu_svd(x_l, xflat, 64, 1e-12, w.nq)
    assert int(d.sum()) == 1 and len(s_o) == 1
    assert np.array_equal(q, A_o.indices[2].charges) and np.array_equal(d, A_o.indices[2].dims)
    assert abs(nrm - x1.norm()) < 1e-12 * x1.norm()
    assert abs(sv[0] / nrm - s_o[0] / x1.norm()) < 1e-12
    assert disc < 1e-24


def test_svd_of_zero_tensor():
    """All-zero input: no singular value reaches any positive cutoff (an empty bond, nothing
    discarded, norm 0, nothing NaN); with cutoff 0 every zero singular value up to m_max is
    kept."""
    w = wl.workload_by_name("spin_m64")
    lays, _ = library_problem(w)
    x_l = lays[4]
    xflat = np.zeros(x_l.nelem)
    q, d, disc, nrm, sv = _gpu_svd(x_l, xflat, 16, 1e-12, w.nq)
    assert len(d) == 0 and nrm == 0.0 and disc == 0.0
    q, d, disc, nrm, sv = _gpu_svd(x_l, xflat, 16, 0.0, w.nq)
    assert int(d.sum()) == 16 and np.all(sv == 0.0) and disc == 0.0
