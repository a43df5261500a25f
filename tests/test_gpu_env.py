"""GPU environment extension (heff_env_update) against the oracle (Section II-C).

Inputs come from the shared seeded generators: the workload's environment and MPO
tensors and Gaussian site tensors on a new bond with even 2Sz charges (the bond after
one more spin-1/2 site).  Both sides enumerate blocks on their own; the GPU result must
match the oracle's block-by-block extension to 1e-12 relative (FP64).
"""
import numpy as np
import pytest

import workloads as wl
from workloads.fill import site_block
from oracle import env as oenv
from oracle.blocks import BlockTensor, Index
from oracle.heff import mpo_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff              # noqa: E402


def _dev(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64)).to("cuda")


def _env_case(name, side, new_m, new_nsec, seed=31):
    w = wl.workload_by_name(name)
    ph = w.phys
    ones = lambda n: np.ones(n, dtype=np.int32)
    gq, gd = wl.binomial_sectors(new_m, new_nsec, seed, parity=0)      # even charges
    if side == "left":
        bq, bd = w.alpha_q, w.alpha_d            # env_old bond (site's left bond)
        site_idx = [(bq, bd, 1), (ph, ones(len(ph)), 1), (gq, gd, -1)]
        env_old_fill, ch_old, ch_new, W = w.L_block, w.ql, w.qm, w.W1
        new_q, new_d = gq, gd
    else:
        bq, bd = w.beta_q, w.beta_d              # env_old bond (site's right bond)
        site_idx = [(gq, gd, 1), (ph, ones(len(ph)), 1), (bq, bd, -1)]
        env_old_fill, ch_old, ch_new, W = w.R_block, w.qr, w.qm, w.W2
        new_q, new_d = gq, gd
    # library layouts and buffers
    site_l = heff.Layout(site_idx)
    W_l = heff.Layout([(w.ql if side == "left" else w.qm, ones(W.shape[0]), 1), (ph, ones(len(ph)), 1),
                       (ph, ones(len(ph)), -1), (w.qm if side == "left" else w.qr, ones(W.shape[3]), -1)])
    old_l = heff.Layout([(bq, bd, -1), (ch_old, ones(len(ch_old)), 1), (bq, bd, 1)])
    new_l = heff.Layout([(new_q, new_d, -1), (ch_new, ones(len(ch_new)), 1), (new_q, new_d, 1)])
    site_fill = lambda k: site_block(seed + 5, k, (int(site_idx[0][1][k[0]]), int(site_idx[2][1][k[2]])))
    bufs = {"site": site_l.assemble(site_fill), "W": W_l.assemble(lambda k: W[k]),
            "old": old_l.assemble(lambda k: env_old_fill(k))}
    # oracle tensors built from the same generators
    phys_ix = Index(ph, ones(len(ph)))
    site_o = BlockTensor.from_fill([Index(site_idx[0][0], site_idx[0][1]), phys_ix,
                                    Index(site_idx[2][0], site_idx[2][1])], (1, 1, -1), np.zeros(w.nq),
                                   lambda k: site_fill(k))
    old_o = BlockTensor.from_fill([Index(bq, bd), mpo_index(ch_old), Index(bq, bd)], (-1, 1, 1),
                                  np.zeros(w.nq), env_old_fill)
    if side == "left":
        ref = oenv.extend_left(old_o, site_o, W, ch_new)
    else:
        ref = oenv.extend_right(old_o, site_o, W, ch_new)
    ref_flat = new_l.assemble(lambda k: ref.blocks[k])
    return old_l, site_l, W_l, new_l, bufs, ref_flat


# FP64 block products: 1e-12; tensor-core BF16x3 products (two chained contractions, FP32
# accumulation): the BF16 path's 1e-3 bound of the matvec, norm-wise, and every element
# within 20x of it relative to the largest
TOL = {"fp64": 1e-12, "bf16x3": 1e-3}


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("side", ["left", "right"])
@pytest.mark.parametrize("name,new_m,new_nsec", [("spin_m64", 70, 9), ("spin_m1024", 1100, 31)])
def test_env_update_matches_oracle(name, new_m, new_nsec, side, prec):
    old_l, site_l, W_l, new_l, bufs, ref = _env_case(name, side, new_m, new_nsec)
    plan = heff.heff_env_plan_create(old_l.handle, site_l.handle, W_l.handle, new_l.handle, bufs["W"], side)
    try:
        heff.heff_env_plan_set_precision(plan, prec)
        ws = torch.empty(heff.heff_env_workspace_size(plan), dtype=torch.uint8, device="cuda")
        out = torch.full((new_l.nelem,), float("nan"), dtype=torch.float64, device="cuda")
        heff.heff_env_update(plan, _dev(bufs["old"]), _dev(bufs["site"]), _dev(bufs["W"]), out, ws)
        torch.cuda.synchronize()
        assert heff.heff_env_status(plan, ws) == 0
        y = out.cpu().numpy()
        assert not np.isnan(y).any()
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        merr = np.abs(y - ref).max() / np.abs(ref).max()
        print(f"env {side} {name} {prec}: rel err {err:.2e} (max element {merr:.2e}), "
              f"flops {heff.heff_env_flops(plan):.3e}")
        assert err < TOL[prec] and merr < 20 * TOL[prec]
    finally:
        heff.heff_env_plan_destroy(plan)


def test_env_update_precision_switch_back_to_fp64_is_exact():
    # retiling for the tensor cores and back leaves the FP64 result bitwise unchanged
    old_l, site_l, W_l, new_l, bufs, ref = _env_case("spin_m64", "left", 70, 9)
    plan = heff.heff_env_plan_create(old_l.handle, site_l.handle, W_l.handle, new_l.handle, bufs["W"], "left")
    try:
        ws = torch.empty(heff.heff_env_workspace_size(plan), dtype=torch.uint8, device="cuda")
        outs = []
        for prec in ("fp64", "bf16x3", "fp64"):
            heff.heff_env_plan_set_precision(plan, prec)
            out = torch.empty((new_l.nelem,), dtype=torch.float64, device="cuda")
            heff.heff_env_update(plan, _dev(bufs["old"]), _dev(bufs["site"]), _dev(bufs["W"]), out, ws)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        assert np.array_equal(outs[0], outs[2])
        assert not np.array_equal(outs[0], outs[1])
        with pytest.raises(heff.HeffError):
            heff.heff_env_plan_set_precision(plan, "tf32x3")
    finally:
        heff.heff_env_plan_destroy(plan)
