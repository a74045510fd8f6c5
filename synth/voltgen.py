"""Seeded synthetic 4+4-bit channelised voltages shaped like MWA X-engine input.

This module holds input generators only: it contains none of the correlator's
arithmetic and is the one piece of code that both the CPU oracle's tests and
the CUDA path's tests consume.  Every random number is drawn from a
counter-based generator -- the SplitMix64 output function of Steele, Lea &
Flood (OOPSLA 2014) applied to ``key + (index + 1) * GAMMA`` -- so any slice
(t, f, n) of a workload can be regenerated on its own, on the CPU (here, numpy)
or on the GPU (``synth/voltgen.cu``), with identical bytes.  After the hash,
everything is integer fixed-point arithmetic (Q12 voltages, Q14 complex gains),
so the two implementations agree bit for bit.

Layout of the output: uint8 ``[T][F][N]``, one byte per complex sample, real
part in the high nibble, imaginary part in the low nibble, both 4-bit two's
complement (Appendix A, "Data Format"; Appendix C, "GPU Input" order).

Two recipes:

``uniform_tone``  i.i.d. integers uniform on [-7, 7] per component plus one
                  common complex sinusoid of amplitude 3 whose phase at input n
                  is 2*pi*n/N_phase, rounded and clipped to [-7, 7].
``gauss3``        Gaussian-like noise (sum of four 8-bit uniforms, an
                  Irwin-Hall(4) shape) of standard deviation 2.25 per
                  component, plus three point-source-like correlated signals,
                  each of standard deviation 0.63 per component, reaching input
                  n of channel f through the phase factor
                  exp(-2*pi*i*nu_f*tau_{s,n}) for seeded delays tau; the sum
                  (total sigma 2.5) is rounded and clipped to [-7, 7].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
KEY_SALT = 0x6A09E667F3BCC909

# stream tags (per array index a: tag + 16*a)
TAG_NOISE = 1
TAG_SRC0 = 2          # sources use TAG_SRC0 + s, s = 0..2
TAG_UNIFORM = 8

Q_VOLT = 12           # voltages in Q12 fixed point
Q_GAIN = 14           # complex gains in Q14
N_SOURCES = 3
SIGMA_NOISE = 2.25
SIGMA_SOURCE = 0.63
TONE_AMPLITUDE = 3.0
CHANNEL_WIDTH_HZ = 1.0e4      # 10 kHz fine channels (Section 3.2.1)
TAU_MAX_S = 2.0e-6            # seeded delays drawn uniformly in [-TAU_MAX, TAU_MAX]
TONE_CYCLES_PER_SAMPLE = 0.0123

# Irwin-Hall(4) of bytes: sum of four uniforms on 0..255 minus 510 (mean 0)
_IH4_SIGMA = math.sqrt(4.0 * (256.0 ** 2 - 1.0) / 12.0)


def _scale_for_sigma(sigma: float) -> int:
    """Integer K so that (ih4 * K) >> 8 is a Q12 value of standard deviation sigma."""
    return int(round(sigma * (1 << Q_VOLT) * 256.0 / _IH4_SIGMA))


K_NOISE = _scale_for_sigma(SIGMA_NOISE)
K_SOURCE = _scale_for_sigma(SIGMA_SOURCE)


def mix64(z: int) -> int:
    """SplitMix64 output function (scalar Python int)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, tag: int) -> int:
    return mix64((seed & MASK64) ^ ((tag & 0xFFFFFF) << 40) ^ KEY_SALT)


def hash_idx(key: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output at positions idx (uint64 array) of the stream ``key``."""
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def _ih4_pair(h: np.ndarray):
    """Irwin-Hall(4) pair from one hash: (sum of bytes 0..3) - 510 and
    (sum of bytes 4..7) - 510 (zero mean), as int32 arrays (bytes in little-endian order
    of the 64-bit value)."""
    h = np.ascontiguousarray(h, dtype=np.uint64)
    b = h.view(np.uint8).reshape(h.shape + (2, 4))
    if not np.little_endian:          # keep byte k = bits 8k..8k+7
        b = b[..., ::-1, ::-1]
    s = b.sum(axis=-1, dtype=np.int32) - 510
    return s[..., 0], s[..., 1]


def _quantise(xq_re: np.ndarray, xq_im: np.ndarray) -> np.ndarray:
    """Q12 -> nearest integer (halves up), clipped to [-7, 7], packed 4+4 bits."""
    half = 1 << (Q_VOLT - 1)
    r = np.clip((xq_re + half) >> Q_VOLT, -7, 7).astype(np.int32)
    m = np.clip((xq_im + half) >> Q_VOLT, -7, 7).astype(np.int32)
    return (((r & 0xF) << 4) | (m & 0xF)).astype(np.uint8)


@dataclass
class Gauss3Params:
    """Host-side parameters of the gauss3 recipe for one array."""
    seed: int
    array: int
    n_inputs: int
    n_chan: int
    gains: np.ndarray          # int32 [S][F][N][2] Q14 (re, im)
    delays_s: np.ndarray       # float64 [S][N]

    @property
    def key_noise(self) -> int:
        return stream_key(self.seed, TAG_NOISE + 16 * self.array)

    def key_src(self, s: int) -> int:
        return stream_key(self.seed, TAG_SRC0 + s + 16 * self.array)


def gauss3_params(seed: int, n_inputs: int, n_chan: int, array: int = 0) -> Gauss3Params:
    rng = np.random.default_rng([seed, array, 0x5EED])
    tau = rng.uniform(-TAU_MAX_S, TAU_MAX_S, size=(N_SOURCES, n_inputs))
    nu = (np.arange(n_chan, dtype=np.float64) + 0.5) * CHANNEL_WIDTH_HZ
    ph = -2.0 * np.pi * nu[None, :, None] * tau[:, None, :]          # [S][F][N]
    g = np.empty((N_SOURCES, n_chan, n_inputs, 2), np.int32)
    g[..., 0] = np.round(np.cos(ph) * (1 << Q_GAIN)).astype(np.int32)
    g[..., 1] = np.round(np.sin(ph) * (1 << Q_GAIN)).astype(np.int32)
    return Gauss3Params(seed, array, n_inputs, n_chan, np.ascontiguousarray(g), tau)


def gauss3(params: Gauss3Params, t0: int, n_time: int,
           f0: int = 0, n_f: int | None = None) -> np.ndarray:
    """Samples t in [t0, t0+n_time), channels [f0, f0+n_f): uint8 [n_time][n_f][N]."""
    N, F = params.n_inputs, params.n_chan
    n_f = F - f0 if n_f is None else n_f
    out = np.empty((n_time, n_f, N), np.uint8)
    if n_time == 0 or n_f == 0:
        return out
    kn = params.key_noise
    ks = [params.key_src(s) for s in range(N_SOURCES)]
    g = params.gains[:, f0:f0 + n_f, :, :]                           # int32 [S][nf][N][2]
    n_idx = np.arange(N, dtype=np.int64)
    f_idx = np.arange(f0, f0 + n_f, dtype=np.int64)
    step = max(1, (1 << 22) // max(1, n_f * N))
    for ta in range(t0, t0 + n_time, step):
        tb = min(t0 + n_time, ta + step)
        t_idx = np.arange(ta, tb, dtype=np.int64)
        tf = t_idx[:, None] * F + f_idx[None, :]                     # [nt][nf]
        idx = tf[:, :, None] * N + n_idx[None, None, :]              # [nt][nf][N]
        nr, ni = _ih4_pair(hash_idx(kn, idx))
        # every intermediate stays below 2**31 in magnitude (int32 is exact)
        xr = (nr * np.int32(K_NOISE)) >> 8
        xi = (ni * np.int32(K_NOISE)) >> 8
        for s in range(N_SOURCES):
            sr, si = _ih4_pair(hash_idx(ks[s], tf))
            sr = ((sr * np.int32(K_SOURCE)) >> 8)[:, :, None]
            si = ((si * np.int32(K_SOURCE)) >> 8)[:, :, None]
            gr = g[s, :, :, 0][None]
            gi = g[s, :, :, 1][None]
            xr += (gr * sr - gi * si) >> Q_GAIN
            xi += (gr * si + gi * sr) >> Q_GAIN
        out[ta - t0:tb - t0] = _quantise(xr, xi)
    return out


@dataclass
class ToneParams:
    seed: int
    array: int
    n_inputs: int
    n_chan: int
    n_phase: int                 # phase of input n is 2*pi*n/n_phase

    @property
    def key(self) -> int:
        return stream_key(self.seed, TAG_UNIFORM + 16 * self.array)

    def phases(self) -> np.ndarray:
        return 2.0 * np.pi * np.arange(self.n_inputs) / self.n_phase


def tone_params(seed: int, n_inputs: int, n_chan: int, array: int = 0,
                n_phase: int | None = None) -> ToneParams:
    return ToneParams(seed, array, n_inputs, n_chan, n_phase or n_inputs)


def tone_table(params: ToneParams, t0: int, n_time: int) -> np.ndarray:
    """Q12 tone A*exp(i(w t + phi_n)), int32 [n_time][N][2]."""
    t = np.arange(t0, t0 + n_time, dtype=np.float64)
    ph = (2.0 * np.pi * TONE_CYCLES_PER_SAMPLE * t[:, None]) + params.phases()[None, :]
    tab = np.empty((n_time, params.n_inputs, 2), np.int32)
    tab[..., 0] = np.round(TONE_AMPLITUDE * np.cos(ph) * (1 << Q_VOLT)).astype(np.int32)
    tab[..., 1] = np.round(TONE_AMPLITUDE * np.sin(ph) * (1 << Q_VOLT)).astype(np.int32)
    return tab


def uniform_tone(params: ToneParams, t0: int, n_time: int,
                 f0: int = 0, n_f: int | None = None) -> np.ndarray:
    """Samples t in [t0, t0+n_time), channels [f0, f0+n_f): uint8 [n_time][n_f][N]."""
    N, F = params.n_inputs, params.n_chan
    n_f = F - f0 if n_f is None else n_f
    out = np.empty((n_time, n_f, N), np.uint8)
    if n_time == 0 or n_f == 0:
        return out
    tab = tone_table(params, t0, n_time).astype(np.int64)             # [nt][N][2]
    t_idx = np.arange(t0, t0 + n_time, dtype=np.int64)
    f_idx = np.arange(f0, f0 + n_f, dtype=np.int64)
    n_idx = np.arange(N, dtype=np.int64)
    idx = (t_idx[:, None, None] * F + f_idx[None, :, None]) * N + n_idx[None, None, :]
    h = hash_idx(params.key, idx)
    ur = ((h & np.uint64(0xFFFFFFFF)) * np.uint64(15) >> np.uint64(32)).astype(np.int64) - 7
    ui = ((h >> np.uint64(32)) * np.uint64(15) >> np.uint64(32)).astype(np.int64) - 7
    xr = (ur << Q_VOLT) + tab[:, None, :, 0]
    xi = (ui << Q_VOLT) + tab[:, None, :, 1]
    return _quantise(xr, xi)


# ----------------------------------------------------------------------------
# The workloads (shapes and seeds).  seed = 1501 + workload index.
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class ArraySpec:
    n_inputs: int
    n_chan: int
    n_time: int              # samples per integration


WORKLOADS = {
    # name: (recipe, seed, [arrays], integrations)
    "small": ("uniform_tone", 1501, [ArraySpec(16, 32, 1000)], 1),
    "coarse_channel": ("gauss3", 1502, [ArraySpec(256, 128, 5000)], 1),
    "full_band": ("gauss3", 1503, [ArraySpec(256, 3072, 5000)], 16),
    "uneven_batch": ("gauss3", 1504, [ArraySpec(128, 1536, 2000),
                                      ArraySpec(256, 3072, 5000),
                                      ArraySpec(1024, 512, 10000)], 1),
    "streaming": ("gauss3", 1505, [ArraySpec(256, 3072, 5000),
                                   ArraySpec(128, 3072, 5000),
                                   ArraySpec(512, 3072, 5000)], 1),
}


def make_params(recipe: str, seed: int, spec: ArraySpec, array: int = 0):
    if recipe == "gauss3":
        return gauss3_params(seed, spec.n_inputs, spec.n_chan, array)
    if recipe == "uniform_tone":
        return tone_params(seed, spec.n_inputs, spec.n_chan, array)
    raise ValueError(recipe)


def generate(params, t0: int, n_time: int, f0: int = 0, n_f: int | None = None) -> np.ndarray:
    if isinstance(params, Gauss3Params):
        return gauss3(params, t0, n_time, f0, n_f)
    if isinstance(params, ToneParams):
        return uniform_tone(params, t0, n_time, f0, n_f)
    raise TypeError(type(params))
