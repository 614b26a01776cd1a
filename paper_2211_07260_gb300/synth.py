"""Seeded synthetic inputs for the convolution workloads.

This module only draws random numbers and lays them out in memory; it holds
none of the method's arithmetic, so both the CUDA path and the CPU oracle can
take their inputs from it.

Recipe (numpy ``default_rng``; the workloads name seeds but no generator):

* one problem: ``rng = default_rng(seed)``; the H x W image is
  ``rng.random((H, W), float32)`` (uniform [0, 1)), then the fh x fw filter is
  ``rng.random((fh, fw), float32)`` divided by its FP64 sum and rounded back to
  float32 (normalised to sum 1);
* the padded input has (fh-1)/2 rows and (fw-1)/2 columns of zeros on each
  side (a "same"-size output), rows of ``pitch`` floats with
  ``pitch = round_up(W + fw - 1, pitch_align)``;
* batched shapes: ``default_rng(seed)`` draws, per image in order, H then W as
  ``round(exp(U[ln 256, ln 2048]))`` and the odd filter size
  ``3 + 2 * integers(0, 8)``; image i takes its values from
  ``default_rng([seed, i])`` with the single-problem recipe;
* served requests: arrival gaps are exponential with mean 1/rate from
  ``default_rng([seed, 0])``; shapes follow the batched law from
  ``default_rng([seed, 1])``; request i takes its values from
  ``default_rng([seed, 2, i])``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def round_up(x: int, a: int) -> int:
    return (int(x) + a - 1) // a * a


@dataclasses.dataclass
class ConvProblem:
    """Host-side padded input, filter and output geometry of one correlation."""
    inp: np.ndarray      # (in_h, in_pitch) float32, zero padded
    in_w: int            # logical input width (<= pitch)
    filt: np.ndarray     # (fh, fw) float32
    out_h: int
    out_w: int

    @property
    def in_h(self) -> int:
        return self.inp.shape[0]

    @property
    def in_pitch(self) -> int:
        return self.inp.shape[1]

    @property
    def fh(self) -> int:
        return self.filt.shape[0]

    @property
    def fw(self) -> int:
        return self.filt.shape[1]


def conv_problem(h: int, w: int, fh: int, fw: int | None = None, seed=0,
                 pitch_align: int = 4, values: str = "uniform") -> ConvProblem:
    """One seeded problem: an h x w image, an fh x fw filter (odd sizes)."""
    fw = fh if fw is None else fw
    if fh < 1 or fw < 1 or fh % 2 == 0 or fw % 2 == 0:
        raise ValueError("filter sides must be odd and positive")
    rng = np.random.default_rng(seed)
    if values == "uniform":
        image = rng.random((h, w), dtype=np.float32)
        filt = rng.random((fh, fw), dtype=np.float32)
        filt = (filt / filt.astype(np.float64).sum()).astype(np.float32)
    elif values == "signed":
        image = (rng.random((h, w), dtype=np.float32) * 2 - 1).astype(np.float32)
        filt = (rng.random((fh, fw), dtype=np.float32) * 2 - 1).astype(np.float32)
    else:
        raise ValueError(values)
    return pad_problem(image, filt, pitch_align)


def pad_problem(image: np.ndarray, filt: np.ndarray, pitch_align: int = 4) -> ConvProblem:
    """Zero-pad an image for a "same"-size correlation with ``filt``."""
    image = np.asarray(image, dtype=np.float32)
    filt = np.ascontiguousarray(filt, dtype=np.float32)
    h, w = image.shape
    fh, fw = filt.shape
    rh, rw = (fh - 1) // 2, (fw - 1) // 2
    in_h, in_w = h + fh - 1, w + fw - 1
    pitch = round_up(in_w, pitch_align)
    inp = np.zeros((in_h, pitch), dtype=np.float32)
    inp[rh:rh + h, rw:rw + w] = image
    return ConvProblem(inp=inp, in_w=in_w, filt=filt, out_h=h, out_w=w)


def batch_shapes(n: int, seed: int, lo: int = 256, hi: int = 2048, kmin: int = 3,
                 kmax: int = 17):
    """Shapes (H, W, k) of a batch of n images drawn by the batched law."""
    rng = np.random.default_rng(seed)
    nk = (kmax - kmin) // 2 + 1
    out = []
    for _ in range(n):
        hh = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        ww = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        k = kmin + 2 * int(rng.integers(0, nk))
        out.append((hh, ww, k))
    return out


def batch_problems(n: int, seed: int, lo: int = 256, hi: int = 2048, pitch_align: int = 4):
    """The n seeded problems of a batch (shapes from ``batch_shapes``)."""
    probs = []
    for i, (hh, ww, k) in enumerate(batch_shapes(n, seed, lo, hi)):
        probs.append(conv_problem(hh, ww, k, seed=[seed, i], pitch_align=pitch_align))
    return probs


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of n requests of a Poisson process of the given rate."""
    rng = np.random.default_rng([seed, 0])
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def request_shapes(n: int, seed: int, lo: int = 256, hi: int = 2048):
    return batch_shapes(n, [seed, 1], lo, hi)


def request_problem(seed: int, i: int, shape, pitch_align: int = 4) -> ConvProblem:
    hh, ww, k = shape
    return conv_problem(hh, ww, k, seed=[seed, 2, i], pitch_align=pitch_align)
