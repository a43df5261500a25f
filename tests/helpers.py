"""Test helpers: build library inputs from a workload and interpret plan tables on CPU.

``library_problem`` turns a ``workloads`` problem into the library's layouts and
flat buffers (via the library's own block enumeration and the shared seeded fills).
``interpret_plan`` executes a plan's exported schedule tables with numpy, following
the record semantics documented in csrc/internal.h, so the schedule can be checked
against the oracle on a machine without a GPU.
"""
import numpy as np

from paper_2007_05540_gb300 import heff


def library_problem(w, batches=(0,)):
    lays = heff.heff_layouts((w.alpha_q, w.alpha_d), (w.beta_q, w.beta_d), w.phys, w.ql, w.qm, w.qr)
    Ll, W1l, W2l, Rl, xl = lays
    bufs = {
        "L": Ll.assemble(lambda k: w.L_block((k[0], k[1], k[2]))),
        "R": Rl.assemble(lambda k: w.R_block((k[0], k[1], k[2]))),
        "W1": W1l.assemble(lambda k: w.W1[k]),
        "W2": W2l.assemble(lambda k: w.W2[k]),
        "x": [xl.assemble(lambda k, b=b: w.x_block(k, b)) for b in batches],
    }
    return lays, bufs


def oracle_flat(xl, yb):
    """Oracle block tensor -> flat buffer in the library layout of x."""
    return xl.assemble(lambda k: yb.blocks[k])


def interpret_plan(plan, bufs, x_flat):
    """y = K x by executing the plan's tables in float64 numpy."""
    h = plan.handle
    st = plan.stats
    rows_x, ld_x, rows_lw, rows_t, ld_t, rows_rw = st[8], st[9], st[10], st[11], st[12], st[13]
    XT = np.full((rows_x, ld_x), np.nan)
    LW = np.full((rows_lw, ld_x), np.nan)
    T = np.full((rows_t, ld_t), np.nan)
    RW = np.full((rows_rw, ld_t), np.nan)
    for t in heff.heff_plan_export(h, 0):
        for b in range(t["b0"], min(t["b0"] + 32, t["m_b"])):
            for a in range(t["a0"], min(t["a0"] + 32, t["a_pad"])):
                v = x_flat[t["x_off"] + a * t["m_b"] + b] if a < t["m_a"] else 0.0
                XT[t["xt_row0"] + b, t["xt_col0"] + a] = v
    terms = heff.heff_plan_export(h, 2)
    for t in heff.heff_plan_export(h, 1):
        src = bufs["R"] if t["which"] else bufs["L"]
        W = bufs["W2"] if t["which"] else bufs["W1"]
        dst = RW if t["which"] else LW
        for r in range(t["r0"], t["r0"] + t["nrows"]):
            acc = np.zeros(t["cols_pad"])
            for m in terms[t["term_begin"]:t["term_begin"] + t["term_count"]]:
                acc[:t["cols"]] += W[m["w_idx"]] * src[m["src_off"] + r * t["cols"]:
                                                       m["src_off"] + (r + 1) * t["cols"]]
            dst[t["dst_row0"] + r, t["dst_col0"]:t["dst_col0"] + t["cols_pad"]] = acc
    y = np.full(len(x_flat), np.nan)
    Tflat = T.reshape(-1)
    for which, (A, B, out) in ((3, (LW, XT, Tflat)), (5, (T, RW, y))):
        tasks = heff.heff_plan_export(h, which)
        segs = heff.heff_plan_export(h, which + 1)
        for t in tasks:
            m, n = t["m"], t["n"]
            acc = np.zeros((m, n))
            for s in segs[t["seg_begin"]:t["seg_begin"] + t["seg_count"]]:
                k0, k1 = s["k0"], s["k0"] + s["klen"]
                acc += A[t["a_row"]:t["a_row"] + m, k0:k1] @ B[t["b_row"]:t["b_row"] + n, k0:k1].T
            for r in range(m):
                o = t["c_off"] + r * t["ldc"]
                out[o:o + n] = acc[r]
                if t["n_zero"]:
                    out[o + n:o + n + t["n_zero"]] = 0.0
    return y
