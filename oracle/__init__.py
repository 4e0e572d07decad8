"""CPU oracle for the FNT-CDC / FNT-AEQ path (arXiv 2405.04253).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only callers.
The product package never imports this module, and this module never imports the
product package.  The arithmetic lives in plain C (``fnt_oracle.c``), written
from the paper's equations with int64 everywhere and O(N^2) transforms; this file
only builds it with gcc and marshals numpy arrays.

Paper references used below:
  eq. (1)/(2)  forward / inverse transform          (section "Fermat number transform")
  eq. (3)/(4)  modulus / radix conditions
  eq. (5)      overflow constraint, zero padding    (section "Proposed FNT-CDC&AEQ structure")
  eq. (6)      RDE tap update of the 4x4 RV-MIMO AEQ
  eq. (7)/(8)  complex convolution from two real products
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fnt_oracle.c")
_HDR = os.path.join(_HERE, "fnt_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")

F = 65537

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no vectorisation flags tied to a CPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or force or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        ll, i32, vp = ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p
        L.orc_powmod.restype = ll
        L.orc_powmod.argtypes = [ll, ll, ll]
        L.orc_invmod.restype = ll
        L.orc_invmod.argtypes = [ll, ll]
        L.orc_order.restype = ll
        L.orc_order.argtypes = [ll, ll]
        L.orc_check_transform.restype = i32
        L.orc_check_transform.argtypes = [i32, ll, ll]
        L.orc_decode.restype = ll
        L.orc_decode.argtypes = [ll, ll]
        L.orc_fnt.restype = None
        L.orc_fnt.argtypes = [vp, vp, i32, ll, ll]
        L.orc_ifnt.restype = None
        L.orc_ifnt.argtypes = [vp, vp, i32, ll, ll]
        L.orc_cdc.restype = i32
        L.orc_cdc.argtypes = [vp, ll, i32, vp, i32, i32, ll, i32, vp]
        L.orc_cdc_shift.restype = i32
        L.orc_cdc_shift.argtypes = [vp, i32]
        L.orc_decim_phase.restype = i32
        L.orc_decim_phase.argtypes = [i32]
        L.orc_requant_decimate.restype = ll
        L.orc_requant_decimate.argtypes = [vp, ll, i32, i32, vp]
        L.orc_aeq_init_taps.restype = None
        L.orc_aeq_init_taps.argtypes = [i32, i32, vp]
        L.orc_aeq.restype = i32
        L.orc_aeq.argtypes = [vp, ll, i32, ll, i32, i32, i32, vp, vp, i32, i32, i32, i32]
        L.orc_aeq_segmented.restype = i32
        L.orc_aeq_segmented.argtypes = [vp, ll, i32, ll, i32, i32, i32, vp, ll, ll, vp, vp, i32, i32, i32]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ field -----

def powmod(a: int, e: int, mod: int = F) -> int:
    return int(lib().orc_powmod(a, e, mod))


def invmod(a: int, mod: int = F) -> int:
    return int(lib().orc_invmod(a, mod))


def order(alpha: int, mod: int = F) -> int:
    return int(lib().orc_order(alpha, mod))


def check_transform(N: int, alpha: int, mod: int = F) -> int:
    """0 when eq. (4) holds, alpha has order exactly N and N is invertible."""
    return int(lib().orc_check_transform(N, alpha, mod))


def decode(r: int, mod: int = F) -> int:
    return int(lib().orc_decode(r, mod))


# -------------------------------------------------------------- transforms -----

def fnt(x, N: int, alpha: int, mod: int = F) -> np.ndarray:
    """Eq. (1), literal O(N^2) sum."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.int64).reshape(N))
    X = np.zeros(N, dtype=np.int64)
    lib().orc_fnt(_p(x), _p(X), N, alpha, mod)
    return X


def ifnt(X, N: int, alpha: int, mod: int = F) -> np.ndarray:
    """Eq. (2), literal O(N^2) sum including N^-1."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.int64).reshape(N))
    x = np.zeros(N, dtype=np.int64)
    lib().orc_ifnt(_p(X), _p(x), N, alpha, mod)
    return x


# --------------------------------------------------------------------- CDC -----

def cdc(x: np.ndarray, taps: np.ndarray, N: int = 64, alpha: int = 4080, S: int | None = None) -> np.ndarray:
    """FNT-CDC by overlap-save through eqs. (7)-(8).

    x    : int8 [n, n_pol, 2] (I, Q), 5-bit signed
    taps : int8 [L, 2] (re, im), 6-bit signed
    returns int32 [n, n_pol, 2]
    """
    x = np.ascontiguousarray(x, dtype=np.int8)
    taps = np.ascontiguousarray(taps, dtype=np.int8)
    n, n_pol = x.shape[0], x.shape[1]
    L = taps.shape[0]
    if S is None:
        S = N - L + 1
    out = np.zeros((n, n_pol, 2), dtype=np.int32)
    rc = lib().orc_cdc(_p(x), n, n_pol, _p(taps), L, N, alpha, S, _p(out))
    if rc != 0:
        raise ValueError(f"orc_cdc failed ({rc})")
    return out


def cdc_shift(taps: np.ndarray) -> int:
    taps = np.ascontiguousarray(taps, dtype=np.int8)
    return int(lib().orc_cdc_shift(_p(taps), taps.shape[0]))


def decim_phase(L: int) -> int:
    return int(lib().orc_decim_phase(L))


def requant_decimate(z: np.ndarray, shift: int, phase: int) -> np.ndarray:
    """CDC output int32 [n, 2, 2] -> 5-bit AEQ input int8 [n_sym, 4] at 1 sps."""
    z = np.ascontiguousarray(z, dtype=np.int32)
    n = z.shape[0]
    n_sym = max(0, (n - phase + 1) // 2)
    xo = np.zeros((n_sym, 4), dtype=np.int8)
    m = lib().orc_requant_decimate(_p(z), n, shift, phase, _p(xo))
    assert m == n_sym
    return xo


# --------------------------------------------------------------------- AEQ -----

def aeq_init_taps(K: int = 16, w0: int = 2048) -> np.ndarray:
    T = np.zeros((4, 4, K), dtype=np.int32)
    lib().orc_aeq_init_taps(K, w0, _p(T))
    return T


def aeq(x: np.ndarray, T: np.ndarray, N: int = 32, alpha: int = 2, mu_shift: int = 20,
        rde_a: int = 64, use_fnt: bool = True, period: int = 1, freq_sum: int = 0, hist: int = 0):
    """FNT-AEQ with the RDE update of eq. (6), applied every `period` blocks;
    freq_sum as orc_aeq.  The first `hist` rows of x are input history only
    (read by the windows, no output).  Returns (out int16 [n_sym - hist, 4], T')."""
    x = np.ascontiguousarray(x, dtype=np.int8)
    T = np.ascontiguousarray(T, dtype=np.int32).copy()
    K = T.shape[2]
    n = x.shape[0] - hist
    out = np.zeros((n, 4), dtype=np.int16)
    xp = x.ctypes.data + hist * 4
    rc = lib().orc_aeq(xp, n, N, alpha, K, mu_shift, rde_a, _p(T), _p(out), int(use_fnt), period,
                       freq_sum, hist)
    if rc != 0:
        raise ValueError(f"orc_aeq failed ({rc})")
    return out, T


def aeq_segmented(x: np.ndarray, T0: np.ndarray, N: int = 32, alpha: int = 2, mu_shift: int = 20,
                  rde_a: int = 64, seg_len: int = 0, warmup: int = 0, use_fnt: bool = True, period: int = 1,
                  freq_sum: int = 0):
    """Segmented AEQ (each output segment re-runs from T0 with a warm-up lead,
    reading the K preceding symbols of the stream as input history)."""
    x = np.ascontiguousarray(x, dtype=np.int8)
    T0 = np.ascontiguousarray(T0, dtype=np.int32)
    K = T0.shape[2]
    Tout = np.zeros_like(T0)
    out = np.zeros((x.shape[0], 4), dtype=np.int16)
    rc = lib().orc_aeq_segmented(_p(x), x.shape[0], N, alpha, K, mu_shift, rde_a, _p(T0),
                                 seg_len, warmup, _p(Tout), _p(out), int(use_fnt), period, freq_sum)
    if rc != 0:
        raise ValueError(f"orc_aeq_segmented failed ({rc})")
    return out, Tout


# ------------------------------------------------------------------- chain -----

@dataclass
class ChainParams:
    """Numbers that define one CDC -> requant/resample -> AEQ pass."""
    n_cdc: int = 64
    alpha_cdc: int = 4080
    n_aeq: int = 32
    alpha_aeq: int = 2
    aeq_taps: int = 16
    mu_shift: int = 20
    rde_a: int = 64
    w0: int = 2048
    seg_len: int = 0
    warmup: int = 0
    period: int = 1
    freq_sum: int = 0


def chain(x: np.ndarray, taps: np.ndarray, prm: ChainParams, T0: np.ndarray | None = None,
          use_fnt: bool = True):
    """PDM chain: FNT-CDC (both pols, S = N - L + 1), requantise to 5 bits, keep
    every second sample, FNT-AEQ.  Returns (out int16 [n_sym, 4], T_final)."""
    z = cdc(x, taps, prm.n_cdc, prm.alpha_cdc)
    xa = requant_decimate(z, cdc_shift(taps), decim_phase(taps.shape[0]))
    if T0 is None:
        T0 = aeq_init_taps(prm.aeq_taps, prm.w0)
    if prm.seg_len > 0:
        return aeq_segmented(xa, T0, prm.n_aeq, prm.alpha_aeq, prm.mu_shift, prm.rde_a,
                             prm.seg_len, prm.warmup, use_fnt, prm.period, prm.freq_sum)
    return aeq(xa, T0, prm.n_aeq, prm.alpha_aeq, prm.mu_shift, prm.rde_a, use_fnt, prm.period, prm.freq_sum)


def chain_segment(x: np.ndarray, taps: np.ndarray, prm: ChainParams, seg: int, T0: np.ndarray | None = None):
    """Outputs of AEQ segment `seg` of the segmented chain, computed from the
    input slice it depends on alone (so a long stream can be checked at sampled
    segments).  Returns (first symbol, out int16 [m, 4], final taps)."""
    n = x.shape[0]
    L = taps.shape[0]
    phase = decim_phase(L)
    n_sym = max(0, (n - phase + 1) // 2)
    seg_len = prm.seg_len if prm.seg_len > 0 else max(1, n_sym)
    keep = seg * seg_len
    end = min(n_sym, keep + seg_len)
    begin = max(0, keep - prm.warmup) if prm.seg_len > 0 else 0
    hist = min(begin, prm.aeq_taps)               # input history before the run
    begin -= hist
    t_lo = 2 * begin + phase                      # first 2-sps time the segment reads
    t_hi = 2 * (end - 1) + phase + 1
    s0 = max(0, t_lo - (L - 1))                   # CDC history of the first output
    z = cdc(x[s0:t_hi], taps, prm.n_cdc, prm.alpha_cdc)
    xa = requant_decimate(z[t_lo - s0:], cdc_shift(taps), 0)
    assert xa.shape[0] == end - begin
    if T0 is None:
        T0 = aeq_init_taps(prm.aeq_taps, prm.w0)
    out, T = aeq(xa, T0, prm.n_aeq, prm.alpha_aeq, prm.mu_shift, prm.rde_a, period=prm.period,
                 freq_sum=prm.freq_sum, hist=hist)
    return keep, out[keep - begin - hist:], T
