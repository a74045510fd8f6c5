"""Seeded synthetic coarse-channel voltages and a prototype window for the
fine polyphase filterbank (input generators only: none of the filterbank's
arithmetic lives here).

The fine filterbank of Section 3.2.1 takes the 1.28 MHz coarse channels of
the receivers and splits each into 128 fine channels with a 12-tap, 128-point
filter.  The paper gives neither the coarse samples' word format nor the
window, so:

``coarse_samples``  int8 ``[Q][N][S][2]`` (real, imaginary): Gaussian noise of
                    standard deviation ``sigma`` per component plus one common
                    complex tone at fine bin ``tone_bin`` of amplitude
                    ``tone_amp`` whose phase at input n is 2 pi n / N, rounded
                    and clipped to [-127, 127] (numpy's PCG64 seeded with
                    ``seed``).
``kaiser_sinc_window``  the usual prototype of a critically sampled
                    filterbank: a sinc of width one channel (``points``
                    samples per lobe) times a Kaiser window of shape ``beta``
                    over ``taps * points`` samples, normalised so that the
                    coefficients sum to ``points``.
``output_scale``    the factor that brings white noise of ``sigma`` per
                    component to a standard deviation of ``target`` codes after
                    the filterbank (the filterbank multiplies the noise power
                    per component by the sum of the squared coefficients).
"""
from __future__ import annotations

import math

import numpy as np


def kaiser_sinc_window(taps: int = 12, points: int = 128, beta: float = 5.0) -> np.ndarray:
    L = taps * points
    t = (np.arange(L) - (L - 1) / 2.0) / points
    h = np.sinc(t) * np.kaiser(L, beta)
    return (h * (points / h.sum())).astype(np.float64)


def output_scale(window: np.ndarray, sigma: float, target: float = 2.5) -> float:
    return float(target / (sigma * math.sqrt(float(np.sum(np.asarray(window, np.float64) ** 2)))))


def coarse_samples(seed: int, Q: int, N: int, S: int, sigma: float = 8.0,
                   tone_bin: int = 17, tone_amp: float = 6.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((Q, N, S, 2)) * sigma
    s = np.arange(S)
    n = np.arange(N)
    ph = 2 * np.pi * (tone_bin * s[None, :] / 128.0 + n[:, None] / N)   # [N][S]
    z[..., 0] += tone_amp * np.cos(ph)[None]
    z[..., 1] += tone_amp * np.sin(ph)[None]
    return np.clip(np.rint(z), -127, 127).astype(np.int8)
