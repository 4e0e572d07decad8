"""Seeded synthetic inputs for the FNT-CDC / FNT-AEQ path.

This module holds no arithmetic of the method: it only simulates, in float64
numpy, the transmitter and channel that stand in for the paper's lab captures
(40 GBaud PDM-16QAM, RRC roll-off 0.1, standard single-mode fibre, AWGN, a
drifting Jones matrix), quantises the received 2-sample/symbol signal to 5-bit
signed I/Q, and designs 6-bit CD taps.  Both the CPU oracle and the GPU path
consume the int8 arrays it returns, so floating point never touches the
bit-exact comparison.

Seeds: configuration i uses numpy PCG64 seed 2405042530 + i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.signal import oaconvolve

BAUD = 40e9
SPS = 2
FS = BAUD * SPS
LAMBDA = 1550e-9
C_LIGHT = 299792458.0
D_PS_NM_KM = 17.0
ROLLOFF = 0.1
SEED_BASE = 2405042530

# beta2 = -D lambda^2 / (2 pi c)  [s^2/m]
BETA2 = -(D_PS_NM_KM * 1e-6) * LAMBDA ** 2 / (2 * math.pi * C_LIGHT)


def rng_for(config: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + config, sub]))


# ----------------------------------------------------------------- channel -----

def cd_tap_count(fiber_km: float) -> int:
    """CD tap count for a fibre length: L = 2 * round(2 + (z - 10) / 10) + 1
    (5 taps at 10 km, 17 at 75 km, 19 at 80 km; numpy rounds half to even)."""
    return int(2 * np.round(2 + (fiber_km - 10.0) / 10.0) + 1)


def _freq_grid(nfft: int) -> np.ndarray:
    return 2 * math.pi * np.fft.fftfreq(nfft, d=1.0 / FS)


def _raised_cosine(nfft: int) -> np.ndarray:
    f = np.abs(np.fft.fftfreq(nfft, d=1.0 / FS))
    f1 = (1 - ROLLOFF) * BAUD / 2
    f2 = (1 + ROLLOFF) * BAUD / 2
    H = np.zeros(nfft)
    H[f <= f1] = 1.0
    mid = (f > f1) & (f < f2)
    H[mid] = 0.5 * (1 + np.cos(math.pi / (ROLLOFF * BAUD) * (f[mid] - f1)))
    return H


def channel_impulse(fiber_km: float, ntaps: int = 1025, nfft: int = 8192) -> np.ndarray:
    """Tx RRC * fibre CD * Rx matched RRC at 2 sps, centred, ntaps long."""
    w = _freq_grid(nfft)
    H = _raised_cosine(nfft) * np.exp(1j * BETA2 * fiber_km * 1e3 * w ** 2 / 2)
    h = np.fft.ifft(H)
    h = np.roll(h, ntaps // 2)[:ntaps]
    return h


def cd_taps(fiber_km: float, L: int | None = None, nfft: int = 8192) -> np.ndarray:
    """6-bit complex CD-compensation taps, int8 [L, 2] (re, im).

    Frequency-sampled inverse of the fibre's all-pass response, truncated to the
    L centre taps, scaled so the largest component is 31, rounded half to even
    and clipped to [-32, 31]."""
    if L is None:
        L = cd_tap_count(fiber_km)
    w = _freq_grid(nfft)
    h = np.fft.ifft(np.exp(-1j * BETA2 * fiber_km * 1e3 * w ** 2 / 2))
    h = np.roll(h, L // 2)[:L]
    scale = 31.0 / max(np.abs(h.real).max(), np.abs(h.imag).max())
    q = np.stack([np.rint(h.real * scale), np.rint(h.imag * scale)], axis=1)
    return np.clip(q, -32, 31).astype(np.int8)


def qam16(rng: np.random.Generator, n_pol: int, n_sym: int) -> np.ndarray:
    lv = np.array([-3.0, -1.0, 1.0, 3.0])
    return lv[rng.integers(0, 4, (n_pol, n_sym))] + 1j * lv[rng.integers(0, 4, (n_pol, n_sym))]


def haar_unitary(rng: np.random.Generator) -> np.ndarray:
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def quantize5(v: np.ndarray, rms_lsb: float = 5.0) -> np.ndarray:
    """Scale each real component to the given RMS, round half to even, clip to
    the 5-bit signed range [-16, 15]."""
    re, im = v.real, v.imag
    s = rms_lsb / max(np.sqrt(np.mean(re ** 2)), np.sqrt(np.mean(im ** 2)), 1e-30)
    out = np.stack([np.clip(np.rint(re * s), -16, 15), np.clip(np.rint(im * s), -16, 15)], axis=-1)
    return out.astype(np.int8)


def received(rng: np.random.Generator, n_samples: int, n_pol: int, fiber_km: float,
             snr_db: float, drift_rad_per_s: float = 100.0, chunk: int = 1 << 22) -> np.ndarray:
    """Received 2-sps signal, int8 [n_samples, n_pol, 2] after 5-bit quantisation."""
    return transmission(rng, n_samples, n_pol, fiber_km, snr_db, drift_rad_per_s, chunk).x


@dataclass
class Transmission:
    x: np.ndarray          # int8 [n_samples, n_pol, 2]: the received signal after 5-bit quantisation
    symbols: np.ndarray    # complex128 [n_pol, n_sym]: the transmitted 16QAM symbols (levels +-1, +-3)
    analog: np.ndarray     # complex128 [n_pol, n_samples]: the received signal before quantisation


def transmission(rng: np.random.Generator, n_samples: int, n_pol: int, fiber_km: float,
                 snr_db: float, drift_rad_per_s: float = 100.0, chunk: int = 1 << 22) -> Transmission:
    """The transmitted symbols, the received 2-sps signal and its 5-bit
    quantisation (the same draws as received()).  Symbol j is at sample 2 j of
    the received signal."""
    n_sym = (n_samples + 1) // 2
    sym = qam16(rng, n_pol, n_sym)
    h = channel_impulse(fiber_km)
    half = len(h) // 2
    up = np.zeros((n_pol, n_sym * 2), dtype=np.complex128)
    up[:, ::2] = sym
    sig = np.empty((n_pol, n_samples), dtype=np.complex128)
    for p in range(n_pol):
        for c0 in range(0, n_samples, chunk):
            c1 = min(n_samples, c0 + chunk)
            a0, a1 = max(0, c0 - half), min(up.shape[1], c1 + half)
            y = oaconvolve(up[p, a0:a1], h, mode="full")
            off = c0 - a0 + half
            sig[p, c0:c1] = y[off:off + (c1 - c0)]
    if n_pol == 2:
        U = haar_unitary(rng)
        sig = U @ sig
        th = drift_rad_per_s * np.arange(n_samples) / FS
        c, s = np.cos(th), np.sin(th)
        x, y = sig[0].copy(), sig[1].copy()
        sig[0] = c * x - s * y
        sig[1] = s * x + c * y
    p_sig = np.mean(np.abs(sig) ** 2)
    sigma = math.sqrt(p_sig / 10 ** (snr_db / 10) / 2)
    sig = sig + sigma * (rng.standard_normal(sig.shape) + 1j * rng.standard_normal(sig.shape))
    q = quantize5(sig)                         # [n_pol, n_samples, 2]
    return Transmission(np.ascontiguousarray(np.transpose(q, (1, 0, 2))), sym, sig)


# ----------------------------------------------------------------- configs -----

@dataclass
class Frame:
    x: np.ndarray            # int8 [n, n_pol, 2]
    taps: np.ndarray         # int8 [L, 2]
    fiber_km: float
    link: int = 0
    arrival_s: float = 0.0


def config1(n_samples: int = 65536) -> Frame:
    """Single-polarisation CDC: 65,536 samples, 75 km (17 taps), SNR 20 dB."""
    rng = rng_for(1)
    return Frame(received(rng, n_samples, 1, 75.0, 20.0), cd_taps(75.0), 75.0)


def config2(n_sym: int = 1 << 20) -> Frame:
    """PDM CDC + AEQ: 2^20 symbols per pol (2^21 samples), 75 km, SNR 18 dB."""
    rng = rng_for(2)
    return Frame(received(rng, 2 * n_sym, 2, 75.0, 18.0), cd_taps(75.0), 75.0)


def frame_lengths(rng: np.random.Generator, n: int, lo_log2: float, hi_log2: float) -> np.ndarray:
    return np.rint(2.0 ** rng.uniform(lo_log2, hi_log2, n)).astype(np.int64)


class _Pools:
    """One received stream per fibre-length class (5 km classes over 10-80 km);
    frames are slices of their class's stream at seeded offsets.  The frame's
    own CD taps come from its exact fibre length.  Generating one stream per
    class instead of one per frame keeps thousands of frames cheap to make; the
    path's cost does not depend on the sample values."""

    def __init__(self, config: int, pool_len: int, snr_db: float = 18.0):
        self.config, self.pool_len, self.snr_db = config, pool_len, snr_db
        self.cache = {}

    def stream(self, km: float) -> np.ndarray:
        c = int(np.clip(np.rint(km / 5.0) * 5, 10, 80))
        if c not in self.cache:
            self.cache[c] = received(rng_for(self.config, 1000 + c), self.pool_len, 2, float(c), self.snr_db)
        return self.cache[c]

    def frame(self, rng: np.random.Generator, n: int, km: float) -> np.ndarray:
        pool = self.stream(km)
        off = int(rng.integers(0, max(1, pool.shape[0] - n + 1)))
        return np.ascontiguousarray(pool[off:off + n])


def config3(n_frames: int = 4096, lo_log2: float = 12, hi_log2: float = 18) -> list[Frame]:
    """Batched: independent PDM frames, lengths log-uniform in [2^12, 2^18]
    samples, fibre uniform over 10-80 km (5-19 taps), SNR 18 dB."""
    rng = rng_for(3)
    lens = frame_lengths(rng, n_frames, lo_log2, hi_log2)
    kms = rng.uniform(10.0, 80.0, n_frames)
    pools = _Pools(3, int(2 ** hi_log2) + 1)
    return [Frame(pools.frame(rng, int(lens[i]), kms[i]), cd_taps(kms[i]), float(kms[i])) for i in range(n_frames)]


@dataclass
class ServeTrace:
    link_km: np.ndarray
    link_taps: list
    frames: list = field(default_factory=list)


def config4(n_frames: int = 2048, n_links: int = 256, rate_hz: float = 20e3,
            lo_log2: float = 12, hi_log2: float = 16) -> ServeTrace:
    """Served: Poisson arrivals at 20k frames/s over 256 links with fixed fibre,
    frames of 2^12-2^16 PDM samples."""
    rng = rng_for(4)
    kms = rng.uniform(10.0, 80.0, n_links)
    tr = ServeTrace(kms, [cd_taps(k) for k in kms])
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_frames))
    links = rng.integers(0, n_links, n_frames)
    lens = frame_lengths(rng, n_frames, lo_log2, hi_log2)
    pools = _Pools(4, int(2 ** hi_log2) + 1)
    for i in range(n_frames):
        k = int(links[i])
        tr.frames.append(Frame(pools.frame(rng, int(lens[i]), kms[k]), tr.link_taps[k], float(kms[k]), link=k,
                               arrival_s=float(t[i])))
    return tr


def config5(n_samples: int = 1 << 27, period: int = 1 << 23) -> Frame:
    """Bandwidth stress: one PDM stream of 2^27 samples per pol, 80 km (19 taps).
    A generated stretch of `period` samples repeats to the full length."""
    rng = rng_for(5)
    base = received(rng, min(n_samples, period), 2, 80.0, 18.0)
    reps = -(-n_samples // base.shape[0])
    x = np.tile(base, (reps, 1, 1))[:n_samples] if reps > 1 else base
    return Frame(np.ascontiguousarray(x), cd_taps(80.0, 19), 80.0)


def random_frame(rng: np.random.Generator, n: int, n_pol: int, L: int) -> Frame:
    """Uniform 5-bit samples and 6-bit taps: the worst-case-leaning edge inputs."""
    x = rng.integers(-16, 16, (n, n_pol, 2)).astype(np.int8)
    taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
    return Frame(x, taps, 0.0)
