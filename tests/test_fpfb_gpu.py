"""The fine polyphase filterbank (Section 3.2.1) against the oracle.

The kernel computes in fp32 and the oracle in fp64, so the spectra are
compared with a bound derived from the arithmetic: each output is a sum of
n_taps * 128 products h x (the windowed sums, 12 fp32 multiply-adds per
point) taken through a 128-point FFT (7 radix-2 levels, each adding at most
a few units of rounding per level, twiddles included).  Every rounding error
is at most 2^-24 of a partial sum whose magnitude is bounded by
A = sum_n sum_p |h[p 128 + n]| (|Re x| + |Im x|), so

    |Y_gpu - Y_exact| <= (12 + 3 * 7 + margin) 2^-24 A  ->  64 * 2^-24 * A

per frame and input.  The 4+4-bit codes are the same except where the exact
scaled value lies within that bound of a rounding boundary (a half-integer),
where either neighbour is correct.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1501_05992_gb300 import corr
from synth import coarse

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _bound(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """64 eps A per (frame, channel, input), broadcast over the 128 channels
    of each coarse channel: [M][Q * 128][N]."""
    Q, N, S, _ = x.shape
    taps = h.size // 128
    M = S // 128 - taps + 1
    ax = (np.abs(x[..., 0].astype(np.float64)) + np.abs(x[..., 1])).reshape(Q, N, S // 128, 128)
    ah = np.abs(h).reshape(taps, 128)
    A = np.zeros((Q, N, M))
    for p in range(taps):
        A += np.einsum("qnmk,k->qnm", ax[:, :, p:p + M], ah[p])
    b = 64 * EPS32 * A                                        # [Q][N][M]
    return np.repeat(b.transpose(2, 0, 1), 128, axis=1)       # [M][Q*128][N]


def _run(x, h, scale, spec=True):
    xt = torch.from_numpy(x).cuda()
    ht = torch.from_numpy(h.astype(np.float32)).cuda()
    v, sp = corr.fine_pfb(xt, ht, scale, volt=True, spec=spec)
    torch.cuda.synchronize()
    return v.cpu().numpy(), (None if sp is None else sp.cpu().numpy())


def _check_codes(got, want_spec, bound, scale):
    vals = np.array([v if v < 8 else v - 16 for v in range(16)])
    for part, shift in (("real", 4), ("imaginary", 0)):
        g = vals[(got >> shift) & 15]
        exact = (want_spec.real if shift else want_spec.imag) * scale
        want = np.clip(np.rint(exact), -7, 7)
        near = np.abs(np.abs(exact - np.floor(exact)) - 0.5) <= bound * scale
        ok = (g == want) | (near & (np.abs(g - exact) <= 0.5 + bound * scale))
        assert ok.all(), f"{part} codes differ away from a rounding boundary at {np.argwhere(~ok)[:5]}"
        assert np.mean(g == want) > 0.99


@pytest.mark.parametrize("Q,N,M", [(2, 20, 130), (1, 8, 1), (3, 64, 240), (1, 1, 9), (2, 17, 16)],
                         ids=["ragged_inputs_and_frames", "one_frame", "three_coarse", "one_input",
                              "odd_inputs"])
def test_fine_pfb_12_taps(Q, N, M):
    taps = 12
    S = 128 * (M + taps - 1)
    x = coarse.coarse_samples(100 + Q * N + M, Q, N, S)
    h = coarse.kaiser_sinc_window(taps)
    scale = coarse.output_scale(h, 8.0)
    want_spec, want_volt = oracle.fine_pfb(x, h.astype(np.float32).astype(np.float64), scale)
    got_volt, got_spec = _run(x, h, scale)
    b = _bound(x, h.astype(np.float32).astype(np.float64))
    err = np.abs(got_spec[..., 0] + 1j * got_spec[..., 1] - want_spec)
    assert got_spec.shape[:3] == want_spec.shape
    assert (err <= b).all(), f"max error / bound {np.max(err / b):.3f}"
    _check_codes(got_volt, want_spec, b, scale)


def test_fine_pfb_single_tap_is_dft():
    Q, N, M = 2, 16, 9
    x = coarse.coarse_samples(7, Q, N, 128 * M, sigma=30.0)
    h = np.ones(128)
    want_spec, _ = oracle.fine_pfb(x, h, 0.01)
    _, got = _run(x, h, 0.01)
    err = np.abs(got[..., 0] + 1j * got[..., 1] - want_spec)
    assert (err <= _bound(x, h)).all()


def test_fine_pfb_feeds_the_x_engine():
    """Integer tones at bins 0, +-32 and 64 with the window 1/12 give exact
    spectra (128 A in one channel, 0 elsewhere), so with scale 1/128 every
    code is far from a rounding boundary; the codes go straight into the
    X-engine and the visibilities must match the oracle chain exactly."""
    taps, M, N = 12, 64, 32
    S = 128 * (M + taps - 1)
    s = np.arange(S)
    x = np.zeros((1, N, S, 2), np.int8)
    units = [np.ones(S, complex), 1j ** s, (-1j) ** s, (-1.0) ** s + 0j]
    for n in range(N):
        z = (1 + n % 5) * units[n % 4] * (1j ** (n // 4))
        x[0, n, :, 0] = np.rint(z.real)
        x[0, n, :, 1] = np.rint(z.imag)
    h = np.full(taps * 128, 1.0 / taps)
    want_spec, want_volt = oracle.fine_pfb(x, h, 1.0 / 128)
    got_volt, _ = _run(x, h, 1.0 / 128, spec=False)
    assert np.array_equal(got_volt, want_volt)
    c = corr.Correlator(N, 128, M, path="auto")
    try:
        c.accumulate(torch.from_numpy(got_volt).cuda())
        vis = c.dump().cpu().numpy()
        c.sync()
    finally:
        c.close()
    assert np.array_equal(vis, oracle.to_int32(oracle.xmac(want_volt)))
    # the tones really are in their channels
    assert np.count_nonzero(want_volt) == M * N


def test_fine_pfb_argument_errors():
    x = torch.zeros((1, 8, 128 * 12, 2), dtype=torch.int8, device="cuda")
    h = torch.ones(12 * 128, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        corr.fine_pfb(x[:, :, :1000], h)                      # not a multiple of 128
    with pytest.raises(corr.CorrError) as e:
        corr.fine_pfb(x, torch.ones(5 * 128, dtype=torch.float32, device="cuda"))
    assert e.value.status == corr.CORR_E_UNSUPPORTED
    v, _ = corr.fine_pfb(x, h)
    torch.cuda.synchronize()
    assert v.shape == (1, 128, 8) and int(v.sum()) == 0


@pytest.mark.parametrize("taps", [1, 12])
def test_fine_pfb_output_choices(taps):
    """Spectra only, codes only, and both into caller tensors agree with each
    other and with the oracle; 13 inputs leave a partial group of 8, whose
    codes go out byte by byte."""
    Q, N, M = 2, 13, 9
    S = 128 * (M + taps - 1)
    x = coarse.coarse_samples(900 + taps, Q, N, S, sigma=12.0)
    h = coarse.kaiser_sinc_window(taps) if taps > 1 else np.ones(128)
    scale = coarse.output_scale(h, 12.0)
    xt = torch.from_numpy(x).cuda()
    ht = torch.from_numpy(h.astype(np.float32)).cuda()
    v_only, none = corr.fine_pfb(xt, ht, scale, volt=True, spec=False)
    assert none is None
    none2, s_only = corr.fine_pfb(xt, ht, scale, volt=False, spec=True)
    assert none2 is None
    v_out = torch.full((M, Q * 128, N), 0xAB, dtype=torch.uint8, device="cuda")
    s_out = torch.full((M, Q * 128, N, 2), float("nan"), dtype=torch.float32, device="cuda")
    v_both, s_both = corr.fine_pfb(xt, ht, scale, volt=v_out, spec=s_out)
    torch.cuda.synchronize()
    assert v_both is v_out and s_both is s_out
    assert torch.equal(v_only, v_out) and torch.equal(s_only, s_out)
    h64 = h.astype(np.float32).astype(np.float64)
    want_spec, _ = oracle.fine_pfb(x, h64, scale)
    got = s_out.cpu().numpy()
    err = np.abs(got[..., 0] + 1j * got[..., 1] - want_spec)
    b = _bound(x, h64)
    assert (err <= b).all()
    _check_codes(v_out.cpu().numpy(), want_spec, b, scale)
    with pytest.raises(ValueError):
        corr.fine_pfb(xt, ht, scale, volt=False, spec=False)


def test_fine_pfb_full_scale_inputs():
    """Samples at the ends of the int8 range (random +-127 and -128, and runs of
    a constant full-scale value, whose whole power lands in channel 64): the
    largest spectra the format allows stay within the fp32 bound, and the
    codes saturate at +-7 exactly where the oracle's do."""
    Q, N, M, taps = 1, 16, 40, 12
    S = 128 * (M + taps - 1)
    rng = np.random.default_rng(127)
    x = rng.choice(np.array([-128, -127, 127], np.int8), size=(Q, N, S, 2))
    x[0, 3] = 127                                   # DC at full scale
    x[0, 4, :, 0] = -128
    x[0, 4, :, 1] = 127
    h = coarse.kaiser_sinc_window(taps)
    h64 = h.astype(np.float32).astype(np.float64)
    scale = coarse.output_scale(h, 127.0)
    want_spec, want_volt = oracle.fine_pfb(x, h64, scale)
    got_volt, got_spec = _run(x, h, scale)
    b = _bound(x, h64)
    err = np.abs(got_spec[..., 0] + 1j * got_spec[..., 1] - want_spec)
    assert (err <= b).all(), f"max error / bound {np.max(err / b):.3f}"
    _check_codes(got_volt, want_spec, b, scale)
    # the constant inputs saturate channel 64 and leave the rest near zero
    vals = np.array([v if v < 8 else v - 16 for v in range(16)])
    assert np.all(vals[got_volt[:, 64, 3] >> 4] == 7) and np.all(vals[got_volt[:, 64, 3] & 15] == 7)
    assert np.all(vals[got_volt[:, 64, 4] >> 4] == -7) and np.all(vals[got_volt[:, 64, 4] & 15] == 7)
