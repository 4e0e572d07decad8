"""Synthetic BER comparison of the FNT-CDC + FNT-AEQ chain with a
floating-point receiver.

The paper's experimental section compares, by BER against received power and
SNR, its integer FNT-CDC + FNT-AEQ scheme with a conventional floating-point
FD-CDC + TD-AEQ scheme, and reads the penalty at the hard-decision FEC limit.
Here the same comparison runs on the synthetic 75 km PDM-16QAM signal of
`synth`, swept over SNR.

The floating-point receiver in this module is the comparison system, not the
method, and shares no code with the oracle or with the CUDA path:
  * FD-CDC: the inverse of the fibre's all-pass response exp(-j beta2 z w^2 / 2)
    applied over the whole frame in the frequency domain (the ideal limit of
    overlap-save FD-CDC);
  * 2:1 decimation at the symbol instants;
  * TD-AEQ: a 4x4 real-valued MIMO equaliser in float64 with K = 16 taps per
    filter, the RDE error of eq. (6) (rings 2 A^2, 10 A^2, 18 A^2 with A = 1,
    decision thresholds 6 A^2 and 14 A^2) and the FNT-AEQ's update schedule (one
    update per block of N - 16 symbols from the gradient summed over the block).
Decisions, Gray bit mapping and the alignment of an equaliser's outputs to the
transmitted symbols are common to every scheme.  The alignment searches the
delay and the polarisation order and fits one complex gain per polarisation on
the known symbols.  The synthetic channel has no carrier phase noise, so that
static phase stands in for the carrier recovery of the paper's receiver.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import synth

HD_FEC_BER = 3.8e-3      # hard-decision FEC limit (7 % overhead)
LEVELS = np.array([-3.0, -1.0, 1.0, 3.0])


# ------------------------------------------------------------ decisions ----

def decide(v: np.ndarray) -> np.ndarray:
    """Nearest 16QAM level of each real component (levels -3, -1, 1, 3)."""
    return np.clip(2.0 * np.floor(v / 2.0) + 1.0, -3.0, 3.0)


def gray_bits(levels: np.ndarray) -> np.ndarray:
    """Two Gray-coded bits per level, [..., 2]: -3 -> 00, -1 -> 01, 1 -> 11,
    3 -> 10 (neighbouring levels differ in one bit)."""
    lv = np.asarray(levels)
    b = np.zeros(lv.shape + (2,), dtype=np.int8)
    b[..., 0] = lv > 0
    b[..., 1] = np.abs(lv) < 2
    return b


@dataclass
class Count:
    errors: int
    bits: int
    per_pol: list          # [(tx polarisation, delay, |gain|, bit errors, bits)] per output

    @property
    def ber(self) -> float:
        return self.errors / self.bits if self.bits else float("nan")


def _delay(z: np.ndarray, s: np.ndarray, skip: int, win: int, max_delay: int) -> int:
    """Delay d (s[t + d] pairs with z[t]) by correlation on a window of z."""
    seg = z[skip:skip + win]
    lo = max(0, skip - max_delay)
    ref = s[lo:skip + win + max_delay]
    c = np.abs(np.correlate(ref, seg, mode="valid"))
    return int(np.argmax(c)) + lo - skip


def count_errors(z: np.ndarray, symbols: np.ndarray, skip: int, max_delay: int = 64) -> Count:
    """Bit errors of the equalised outputs z (complex [2, m] or [1, m]) against
    the transmitted symbols [n_pol, n], counted from output symbol `skip` on
    (the equaliser's convergence is not counted), with the polarisation order,
    delay and complex gain that give the fewest errors."""
    n_pol = z.shape[0]
    orders = [(0,)] if n_pol == 1 else [(0, 1), (1, 0)]
    best = None
    for order in orders:
        tot_e = tot_b = 0
        info = []
        for p in range(n_pol):
            q = order[p]
            d = _delay(z[p], symbols[q], skip, min(8192, z.shape[1] - skip), max_delay)
            t = np.arange(skip, z.shape[1])
            t = t[(t + d >= 0) & (t + d < symbols.shape[1])]
            zs, ss = z[p, t], symbols[q, t + d]
            g = np.vdot(ss, zs) / np.vdot(ss, ss)
            zh = zs / g
            e = int((gray_bits(decide(zh.real)) != gray_bits(ss.real)).sum() +
                    (gray_bits(decide(zh.imag)) != gray_bits(ss.imag)).sum())
            tot_e += e
            tot_b += 4 * len(t)
            info.append((q, d, float(abs(g)), e, 4 * len(t)))
        if best is None or tot_e < best.errors:
            best = Count(tot_e, tot_b, info)
    return best


def snr_at_ber(snrs, bers, target: float = HD_FEC_BER):
    """SNR (dB) at which a BER curve crosses `target`, interpolating log10(BER)
    linearly between the two sweep points around the crossing; None when the
    curve does not cross it inside the sweep."""
    pts = [(s, b) for s, b in zip(snrs, bers) if b > 0]
    for (s0, b0), (s1, b1) in zip(pts, pts[1:]):
        if (b0 - target) * (b1 - target) <= 0 and b0 != b1:
            l0, l1, lt = math.log10(b0), math.log10(b1), math.log10(target)
            return s0 + (lt - l0) * (s1 - s0) / (l1 - l0)
    return None


# ------------------------------------------------ floating-point receiver ----

def fd_cdc(sig: np.ndarray, fiber_km: float) -> np.ndarray:
    """Ideal frequency-domain CD compensation of a 2-sps signal [n_pol, n]:
    the spectrum times exp(-j beta2 z w^2 / 2), the inverse of the fibre's
    all-pass response."""
    n = sig.shape[-1]
    w = 2 * math.pi * np.fft.fftfreq(n, d=1.0 / synth.FS)
    H = np.exp(-1j * synth.BETA2 * fiber_km * 1e3 * w ** 2 / 2)
    return np.fft.ifft(np.fft.fft(sig, axis=-1) * H, axis=-1)


def td_aeq(x: np.ndarray, n_aeq: int = 32, K: int = 16, mu: float = 3e-5, w0: float = 1.0) -> np.ndarray:
    """Float64 4x4 real-valued MIMO equaliser on 1-sps input x [m, 4] (XI, XQ,
    YI, YQ), scaled so that each component has the power of the 16QAM levels
    (5): z_S2(t) = sum_S1 sum_k w[S2][S1][k] x_S1(t - k), the RDE error of each
    polarisation e(t) = R(t) - |z(t)|^2 with R the ring of |z(t)|^2, and the
    update w[S2][S1][k] += mu sum_t e_p(S2)(t) z_S2(t) x_S1(t - k) once per block
    of n_aeq - 16 symbols, over that block (the FNT-AEQ's schedule).  Starts
    from a centre spike w0 on the four diagonal filters."""
    m = x.shape[0]
    SA = n_aeq - K
    W = np.zeros((4, 4, K))
    for s in range(4):
        W[s, s, K // 2] = w0
    X = np.zeros((m + K, 4))
    X[K:] = x
    z = np.zeros((m, 4))
    lags = np.arange(K)
    for b0 in range(0, m, SA):
        b1 = min(m, b0 + SA)
        F = X[np.arange(b0, b1)[:, None] - lags[None, :] + K]          # [n, K, 4]: x(t - k)
        zb = np.einsum("osk,nks->no", W, F)
        z[b0:b1] = zb
        e = np.empty_like(zb)
        for p in range(2):
            r2 = zb[:, 2 * p] ** 2 + zb[:, 2 * p + 1] ** 2
            R = np.where(r2 < 6.0, 2.0, np.where(r2 < 14.0, 10.0, 18.0))
            e[:, 2 * p] = e[:, 2 * p + 1] = R - r2
        W += mu * np.einsum("no,nks->osk", e * zb, F)
    return z


def float_receiver(sig: np.ndarray, fiber_km: float, n_aeq: int = 32, mu: float = 3e-5) -> np.ndarray:
    """The floating-point FD-CDC + TD-AEQ scheme on a 2-sps PDM signal
    [2, n] (complex): equalised outputs, complex [2, n / 2]."""
    c = fd_cdc(sig, fiber_km)[:, 0::2]
    x = np.stack([c[0].real, c[0].imag, c[1].real, c[1].imag], axis=1)
    x = x * math.sqrt(5.0 / np.mean(x ** 2))
    z = td_aeq(x, n_aeq=n_aeq, mu=mu)
    return np.stack([z[:, 0] + 1j * z[:, 1], z[:, 2] + 1j * z[:, 3]])


def int8_to_complex(x: np.ndarray) -> np.ndarray:
    """int8 [n, n_pol, 2] (I, Q) samples as complex [n_pol, n]."""
    return (x[:, :, 0].astype(np.float64) + 1j * x[:, :, 1].astype(np.float64)).T


def chain_to_complex(out: np.ndarray) -> np.ndarray:
    """FNT chain output int16 [n_sym, 4] (XI, XQ, YI, YQ) as complex [2, n_sym]."""
    o = out.astype(np.float64)
    return np.stack([o[:, 0] + 1j * o[:, 1], o[:, 2] + 1j * o[:, 3]])


def td_cdc(sig: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """Float64 time-domain CD compensation with the chain's own integer taps
    (int8 [L, 2], re/im), centred: y[t] = sum_k h[k] x[t + (L - 1) / 2 - k]."""
    h = taps[:, 0].astype(np.float64) + 1j * taps[:, 1].astype(np.float64)
    L = h.shape[0]
    return np.stack([np.convolve(s, h)[(L - 1) // 2:(L - 1) // 2 + s.shape[0]] for s in sig])


def float_receiver_taps(sig: np.ndarray, taps: np.ndarray, n_aeq: int = 32, mu: float = 3e-5) -> np.ndarray:
    """The floating-point TD-AEQ after a float convolution with the chain's
    quantised CD taps: the FNT scheme's filters in float arithmetic."""
    c = td_cdc(sig, taps)[:, 0::2]
    x = np.stack([c[0].real, c[0].imag, c[1].real, c[1].imag], axis=1)
    x = x * math.sqrt(5.0 / np.mean(x ** 2))
    z = td_aeq(x, n_aeq=n_aeq, mu=mu)
    return np.stack([z[:, 0] + 1j * z[:, 1], z[:, 2] + 1j * z[:, 3]])
