"""Pins of the FP64 correlation oracle against facts outside itself.

The oracle's sum is checked against library routines that compute the same
operation by other means (scipy's direct correlation, an FFT product), and
against closed forms and invariants of the operation, so that a dropped tap,
a flipped or transposed filter, an off-by-one window or a wrong pitch fails at
least one test.
"""
import numpy as np
import pytest
import scipy.signal

import oracle
from paper_2211_07260_gb300 import synth


def _valid(prob):
    return prob.inp[:, :prob.in_w].astype(np.float64)


@pytest.mark.parametrize("h", range(1, 10))
@pytest.mark.parametrize("w", [1, 2, 5, 9])
@pytest.mark.parametrize("fh,fw", [(1, 1), (3, 3), (5, 5), (3, 5), (5, 1)])
def test_matches_scipy_correlate2d(h, w, fh, fw):
    prob = synth.conv_problem(h, w, fh, fw, seed=[h, w, fh, fw], values="signed")
    got = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w)
    want = scipy.signal.correlate2d(_valid(prob), prob.filt.astype(np.float64), mode="valid")
    assert got.shape == (h, w)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("k", [7, 17])
def test_matches_fft_correlation(k):
    prob = synth.conv_problem(61, 47, k, seed=5)
    a = _valid(prob)
    f = prob.filt.astype(np.float64)
    shp = (a.shape[0] + k - 1, a.shape[1] + k - 1)
    # correlation = convolution with the filter rotated by 180 degrees
    full = np.fft.irfft2(np.fft.rfft2(a, shp) * np.fft.rfft2(f[::-1, ::-1], shp), shp)
    want = full[k - 1:a.shape[0], k - 1:a.shape[1]]
    got = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12)


def test_delta_filter_returns_image_exactly():
    for k in (3, 9, 17):
        img = np.random.default_rng(k).random((37, 29), dtype=np.float32)
        filt = np.zeros((k, k), np.float32)
        filt[k // 2, k // 2] = 1.0
        prob = synth.pad_problem(img, filt)
        got = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w)
        assert np.array_equal(got, img.astype(np.float64))


def test_off_centre_delta_shifts():
    img = np.random.default_rng(1).random((20, 24), dtype=np.float32)
    filt = np.zeros((5, 5), np.float32)
    filt[0, 4] = 1.0  # picks in[y][x+4], i.e. image[y-2][x+2]
    prob = synth.pad_problem(img, filt)
    got = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w)
    assert np.array_equal(got[2:, :-2], img[:-2, 2:].astype(np.float64))
    assert np.all(got[:2, :] == 0) and np.all(got[:, -2:] == 0)


def test_constant_image_sum_one_filter_interior():
    c = 0.625
    k = 7
    img = np.full((40, 33), c, np.float32)
    filt = np.full((k, k), 1.0 / 64.0, np.float32)
    filt[0, :] = 0.0
    filt[1, 0] += np.float32(1.0 - filt.astype(np.float64).sum())  # sum exactly 1
    assert filt.astype(np.float64).sum() == 1.0
    prob = synth.pad_problem(img, filt)
    got = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w)
    r = k // 2
    np.testing.assert_allclose(got[r:-r, r:-r], c, rtol=1e-14)
    assert np.all(got[0, :] < c)  # the zero border reaches the first row


def test_ramp_closed_form_all_ones_filter():
    # in[y][x] = a*y + b*x + c on the whole (unpadded) array; an all-ones
    # fh x fw window sums to fh*fw*(a*(y+(fh-1)/2) + b*(x+(fw-1)/2) + c).
    a, b, c = 3.0, -2.0, 5.0
    hh, ww, fh, fw = 23, 31, 5, 3
    yy, xx = np.mgrid[0:hh, 0:ww]
    inp = (a * yy + b * xx + c).astype(np.float32)
    got = oracle.conv2d(inp, np.ones((fh, fw), np.float32))
    oy, ox = np.mgrid[0:hh - fh + 1, 0:ww - fw + 1]
    want = fh * fw * (a * (oy + (fh - 1) / 2) + b * (ox + (fw - 1) / 2) + c)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)


def test_linearity_in_input_and_filter():
    rng = np.random.default_rng(7)
    # dyadic values keep s*x + t*y exact in float32
    x = (rng.integers(-64, 65, (30, 28)) / 16.0).astype(np.float32)
    y = (rng.integers(-64, 65, (30, 28)) / 16.0).astype(np.float32)
    f = (rng.integers(-64, 65, (5, 5)) / 32.0).astype(np.float32)
    g = (rng.integers(-64, 65, (5, 5)) / 32.0).astype(np.float32)
    conv = lambda im, fl: oracle.conv2d(synth.pad_problem(im, fl).inp, fl,
                                        in_w=im.shape[1] + fl.shape[1] - 1)
    s, t = np.float32(2.0), np.float32(-0.5)  # exact in float32
    np.testing.assert_allclose(conv(s * x + t * y, f), 2.0 * conv(x, f) - 0.5 * conv(y, f),
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(conv(x, s * f + t * g), 2.0 * conv(x, f) - 0.5 * conv(x, g),
                               rtol=1e-12, atol=1e-12)


def test_symmetric_filter_correlation_equals_convolution():
    rng = np.random.default_rng(3)
    f = rng.random((7, 7)).astype(np.float32)
    f = (f + f[::-1, ::-1]) / 2  # point-symmetric
    img = rng.random((25, 19), dtype=np.float32)
    prob = synth.pad_problem(img, f)
    got = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w)
    want = scipy.signal.convolve2d(_valid(prob), f.astype(np.float64), mode="valid")
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_asymmetric_filter_is_not_flipped():
    f = np.zeros((3, 3), np.float32)
    f[0, 0] = 1.0
    inp = np.arange(25, dtype=np.float32).reshape(5, 5)
    got = oracle.conv2d(inp, f)
    assert np.array_equal(got, inp[:3, :3].astype(np.float64))  # top-left tap, no flip


def test_shift_equivariance_interior():
    rng = np.random.default_rng(11)
    big = rng.random((50, 50), dtype=np.float32)
    f = rng.random((5, 5)).astype(np.float32)
    o1 = oracle.conv2d(big[0:40, 0:40], f)
    o2 = oracle.conv2d(big[3:43, 2:42], f)
    assert np.array_equal(o1[3:, 2:], o2[:-3, :-2])


def test_pitch_padding_is_ignored():
    prob4 = synth.conv_problem(13, 11, 5, seed=2, pitch_align=4)
    prob32 = synth.conv_problem(13, 11, 5, seed=2, pitch_align=32)
    prob32.inp[:, prob32.in_w:] = 1e30  # garbage beyond the logical width
    a = oracle.conv2d(prob4.inp, prob4.filt, in_w=prob4.in_w)
    b = oracle.conv2d(prob32.inp, prob32.filt, in_w=prob32.in_w)
    assert np.array_equal(a, b)


def test_points_equal_full_and_threads_agree():
    prob = synth.conv_problem(70, 90, 9, seed=4)
    full1 = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w, nthreads=1)
    fulln = oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w, nthreads=4)
    assert np.array_equal(full1, fulln)
    rng = np.random.default_rng(0)
    ys = rng.integers(0, 70, 200)
    xs = rng.integers(0, 90, 200)
    pts = oracle.conv2d_points(prob.inp, prob.filt, ys, xs, in_w=prob.in_w)
    assert np.array_equal(pts, full1[ys, xs])


def test_rejects_bad_geometry():
    with pytest.raises(ValueError):
        oracle.conv2d(np.zeros((3, 3), np.float32), np.ones((5, 5), np.float32))
    with pytest.raises(ValueError):
        oracle.conv2d_points(np.zeros((8, 8), np.float32), np.ones((3, 3), np.float32),
                             [6], [0])
