"""Shared helpers of the GPU parity tests: seeded inputs, one GEMM through the
C ABI, and the element-wise comparison with the FP64 oracle.

The acceptance bound for every output element is

    |C - C64|_ij <= k * 2^-22 * |alpha| * (|A||B|)_ij + 2^-22 * |beta * C_in|_ij
                    + ulp_out(C64_ij)

where C64 is the oracle's FP64 result on the same (already rounded) inputs and
ulp_out is one unit in the last place of the output format at C64: FP32
accumulation of k products, whose rounding (the tensor core's and the fixup's)
stays within k * 2^-22 relative to sum |a||b|, plus one rounding of the result
into the output format.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from oracle import rounding
from paper_2301_03598_gb300 import inputs
from paper_2301_03598_gb300 import streamk as sk

ACC_REL = 2.0 ** -22


def num_sms() -> int:
    return torch.cuda.get_device_properties(0).multi_processor_count


def hybrid_shape(p: int, waves: int, extra: int, tiles_n: int = 8):
    """tiles_m so that t = tiles_m * tiles_n is waves * p + extra (rounded up
    to a multiple of tiles_n)."""
    return -(-(waves * p + extra) // tiles_n)


def bound(k, alpha, beta, absAB, C64, Cin64, c_type):
    b = k * ACC_REL * abs(alpha) * absAB + rounding.ulp(C64, c_type)
    if beta != 0.0:
        b = b + ACC_REL * np.abs(beta * Cin64)
    return b


def check_bound(C, C64, b, what=""):
    err = np.abs(C.astype(np.float64) - C64)
    bad = ~(err <= b)
    if bad.any():
        idx = np.argwhere(bad)
        i = tuple(idx[0])
        raise AssertionError(
            f"{what}: {bad.sum()} of {bad.size} elements outside the bound; first at {i}: "
            f"got {C[i]!r} want {C64[i]!r} err {err[i]:.3e} bound {b[i]:.3e}; "
            f"max err/bound {np.max(err / np.maximum(b, 1e-300)):.3g}")
    return float(np.max(err / np.maximum(b, 1e-300))) if err.size else 0.0


class Problem:
    """Seeded inputs for C = alpha*A*B + beta*C: A (m x k, row-major), B
    (k x n, column-major, i.e. an n x k row-major tensor), C_in (m x n)."""

    def __init__(self, m, n, k, a_type="bf16", c_type="bf16", dist="normal", seed=0,
                 beta=0.0, lda=None, ldb=None):
        self.m, self.n, self.k = m, n, k
        self.a_type, self.c_type = a_type, c_type
        self.lda = lda or k
        self.ldb = ldb or k
        a_full, _ = inputs.host_matrix(m, self.lda, a_type, dist, seed * 7 + 1)
        b_full, _ = inputs.host_matrix(n, self.ldb, a_type, dist, seed * 7 + 2)
        self.A = a_full             # storage m x lda
        self.B = b_full             # storage n x ldb (B^T rows)
        if beta != 0.0:
            self.Cin, _ = inputs.host_matrix(m, n, c_type, dist, seed * 7 + 3)
        else:
            self.Cin = torch.zeros((m, n), dtype=inputs.DTYPES[c_type])

    def oracle(self, alpha, beta):
        A64 = inputs.widen(self.A)[:, :self.k]
        B64 = inputs.widen(self.B)[:, :self.k].T
        Cin64 = inputs.widen(self.Cin)
        return oracle.gemm(A64, B64, alpha, beta, Cin64 if beta != 0.0 else None)

    def run(self, alpha=1.0, beta=0.0, mode="auto", c_layout="row", plan_attrs=None,
            trace=False, reps=1):
        m, n, k = self.m, self.n, self.k
        plan = sk.sk_plan(m, n, k, self.a_type, self.a_type, self.c_type, "f32", "row", "col",
                          c_layout, mode)
        try:
            for key, v in (plan_attrs or {}).items():
                plan.set(key, v)
            if self.lda != k:
                plan.set("lda", self.lda)
            if self.ldb != k:
                plan.set("ldb", self.ldb)
            A = self.A.cuda()
            B = self.B.cuda()
            outs = []
            tr = None
            for _ in range(reps):
                if c_layout == "row":
                    C = self.Cin.clone().cuda()
                else:
                    C = self.Cin.t().contiguous().cuda()   # n x m storage of column-major C
                if trace:
                    tr = torch.full((plan.get("trace_ints"),), -7, dtype=torch.int32,
                                    device="cuda")
                    sk.sk_gemm_traced(plan, A, B, C, alpha, beta, tr)
                else:
                    sk.sk_gemm(plan, A, B, C, alpha, beta)
                st, dev = sk.sk_last_error(plan)
                assert st == sk.SK_OK, (sk.sk_status_string(st), dev)
                out = C.cpu()
                outs.append(out if c_layout == "row" else out.t().contiguous())
            info = plan.info()
            trace_records = None
            if trace:
                trace_records = sk.decode_trace(tr.cpu().tolist(), info["ctas"],
                                                info["trace_cap"])
            return outs, info, trace_records
        finally:
            plan.destroy()

    def check(self, C, alpha, beta, what=""):
        C64, absAB = self.oracle(alpha, beta)
        b = bound(self.k, alpha, beta, absAB, C64, inputs.widen(self.Cin), self.c_type)
        return check_bound(inputs.widen(C), C64, b, what)
