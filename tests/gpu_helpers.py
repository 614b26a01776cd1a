"""Helpers shared by the GPU tests: device copies of seeded problems and the
error metrics the parity tests use."""
import numpy as np

import oracle

# Tolerance of the floating-point parity tests: the workload asks for a max
# relative error <= 1e-5 against an FP64 reference.  Each output is one FP32
# fmaf chain over fh*fw products of inputs in [0, 1) and non-negative taps,
# so its rounding error is a sum of at most fh*fw relative errors of 2^-24:
# the expected size is ~sqrt(fh*fw) * 2^-24 (1e-6 at 17 x 17), the worst case
# fh*fw * 2^-24 (1.7e-5 at 17 x 17), hence a measured gate, not a bound.
MAX_REL = 1e-5


def max_rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mask = np.abs(ref) > 1e-30
    if not mask.any():
        return float(np.max(np.abs(got - ref))) if got.size else 0.0
    return float(np.max(np.abs(got[mask] - ref[mask]) / np.abs(ref[mask])))


def normwise_err(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref)) if ref.size else 0.0
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / den) if den > 0 else 0.0


def to_device(prob, out_pitch=None, guard_rows=0, guard_val=np.float32(-7.0)):
    """(d_in, d_out_full, d_out_view) on cuda:0; the output has optional
    guard rows / columns filled with guard_val around the written region."""
    import torch
    d_in = torch.from_numpy(prob.inp).cuda()
    pitch = out_pitch or ((prob.out_w + 3) // 4 * 4)
    full = torch.full((prob.out_h + 2 * guard_rows, pitch), float(guard_val), dtype=torch.float32,
                      device="cuda")
    view = full[guard_rows:guard_rows + prob.out_h]
    return d_in, full, view


def oracle_ref(prob):
    return oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w)
