"""Pins for the CPU oracle: each test ties it to something other than itself --
closed forms, the Fig. 1 worked case, library convolutions (numpy), a float64
derivative of the RDE cost -- so that a dropped term, a wrong sign or a swapped
index anywhere in it fails here.  No GPU needed."""
import os

import numpy as np
import pytest

F = 65537
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- field -----

def test_field_constants(orc):
    # sqrt(2) radix of the CDC (section "Proposed FNT-CDC&AEQ structure"):
    # 4080 = 2^12 - 2^4 squares to 2 modulo 2^16 + 1.
    assert (4080 * 4080) % F == 2
    assert orc.powmod(4080, 2) == 2
    assert orc.powmod(4080, 32) == F - 1            # alpha^(N/2) = -1
    assert orc.powmod(4080, 64) == 1                # eq. (4)
    assert orc.order(4080) == 64
    assert orc.order(2) == 32                       # AEQ radix 2, N = 32
    assert orc.order(256) == 4 and (256 * 256) % F == F - 1   # 2^(q/2) = sqrt(-1)
    for a in (2, 64, 32, 512, 4080, 12345):
        assert (orc.invmod(a) * a) % F == 1
    assert orc.invmod(64) == 64513 and orc.invmod(32) == 63489
    assert orc.invmod(2) == 32769 and orc.invmod(512) == 65409
    # -2^(q-1) and -2^(q/2-1) of eqs. (7)/(8) are 2^-1 and (2 * 2^8)^-1
    assert (F - 2 ** 15) == orc.invmod(2)
    assert (F - 2 ** 7) == orc.invmod(512)


def test_check_transform(orc):
    assert orc.check_transform(64, 4080) == 0
    assert orc.check_transform(32, 2) == 0
    assert orc.check_transform(8, 2, 17) == 0
    assert orc.check_transform(64, 2) != 0          # 2 has order 32, not 64
    assert orc.check_transform(16, 4080) != 0       # alpha^16 != 1
    assert orc.check_transform(32, 4) != 0          # order 16: eq. (4) holds, order does not


def test_decode_edges(orc):
    assert orc.decode(0) == 0
    assert orc.decode(32768) == 32768
    assert orc.decode(32769) == -32768
    assert orc.decode(65536) == -1
    assert orc.decode(5, 17) == 5 and orc.decode(9, 17) == -8


# ------------------------------------------------------------ transforms -----

def test_fnt8_mod17_golden(orc):
    with open(os.path.join(GOLDEN, "fnt8_mod17.txt")) as fh:
        rows = [ln for ln in fh if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 4
    for ln in rows:
        a, b = ln.split("|")
        x = [int(v) for v in a.split()]
        X = [int(v) for v in b.split()]
        assert list(orc.fnt(x, 8, 2, 17)) == X
        assert list(orc.ifnt(X, 8, 2, 17)) == x


@pytest.mark.parametrize("N,alpha", [(64, 4080), (32, 2), (64, 61457)])
def test_fnt_impulse_is_geometric(orc, N, alpha):
    # FNT of a unit impulse at m is the geometric sequence alpha^(m k).
    for m in (0, 1, 5, N - 1):
        x = np.zeros(N, dtype=np.int64)
        x[m] = 1
        X = orc.fnt(x, N, alpha)
        assert list(X) == [pow(alpha, m * k, F) for k in range(N)]


@pytest.mark.parametrize("N,alpha", [(64, 4080), (32, 2)])
def test_fnt_ramp_closed_form(orc, N, alpha):
    # sum_{n<N} (n+1) w^n = N / (w - 1) for w^N = 1, w != 1; N(N+1)/2 at w = 1.
    X = orc.fnt(np.arange(1, N + 1), N, alpha)
    assert X[0] == N * (N + 1) // 2 % F
    for k in range(1, N):
        w = pow(alpha, k, F)
        assert X[k] == N * pow(w - 1, -1, F) % F
    if N == 64:
        assert list(X[:8]) == [2080, 64573, 64, 55890, 21867, 12554, 18734, 55668]


def test_fnt_constant_and_round_trip(orc):
    rng = np.random.default_rng(7)
    for N, alpha, mod in [(64, 4080, F), (32, 2, F), (8, 2, 17)]:
        X = orc.fnt(np.ones(N, dtype=np.int64), N, alpha, mod)
        assert X[0] == N % mod and not X[1:].any()
        for _ in range(3):
            x = rng.integers(0, mod, N)
            assert np.array_equal(orc.ifnt(orc.fnt(x, N, alpha, mod), N, alpha, mod), x)


def test_cyclic_convolution_theorem(orc):
    rng = np.random.default_rng(11)
    for N, alpha in [(64, 4080), (32, 2)]:
        a = rng.integers(0, F, N)
        b = rng.integers(0, F, N)
        ref = np.zeros(N, dtype=object)
        for i in range(N):
            for j in range(N):
                ref[(i + j) % N] += int(a[i]) * int(b[j])
        ref = np.array([int(v) % F for v in ref], dtype=np.int64)
        got = orc.ifnt((orc.fnt(a, N, alpha).astype(object) * orc.fnt(b, N, alpha).astype(object)) % F,
                       N, alpha)
        assert np.array_equal(got, ref)


# ------------------------------------------------------------------- CDC -----

def _cdc_numpy(x, taps):
    """Exact complex integer linear convolution, zero history, via numpy."""
    n, n_pol = x.shape[0], x.shape[1]
    hr = taps[:, 0].astype(np.int64)
    hi = taps[:, 1].astype(np.int64)
    out = np.zeros((n, n_pol, 2), dtype=np.int64)
    for p in range(n_pol):
        xr = x[:, p, 0].astype(np.int64)
        xi = x[:, p, 1].astype(np.int64)
        out[:, p, 0] = (np.convolve(xr, hr) - np.convolve(xi, hi))[:n]
        out[:, p, 1] = (np.convolve(xr, hi) + np.convolve(xi, hr))[:n]
    return out


@pytest.mark.parametrize("n,n_pol,L,S", [(1000, 1, 17, 48), (777, 2, 19, 46), (300, 2, 5, 60),
                                         (64, 1, 17, 48), (47, 2, 17, 48), (1, 2, 17, 48),
                                         (500, 2, 17, 32), (333, 1, 1, 64)])
def test_cdc_equals_linear_convolution(orc, n, n_pol, L, S):
    rng = np.random.default_rng(n * 31 + L)
    x = rng.integers(-16, 16, (n, n_pol, 2)).astype(np.int8)
    taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
    assert np.array_equal(orc.cdc(x, taps, 64, 4080, S), _cdc_numpy(x, taps))


def test_cdc_worst_case_at_the_bound(orc):
    # Constraint (5): 32 taps of (-32, -32) on samples (-16, -16) reach exactly
    # |Im z| = 32 * 1024 = 32768 = (F-1)/2: still exact.  33 taps exceed it.
    x = np.full((200, 2, 2), -16, dtype=np.int8)
    for L, exact in [(32, True), (33, False)]:
        taps = np.full((L, 2), -32, dtype=np.int8)
        got = orc.cdc(x, taps, 64, 4080, 64 - L + 1)
        ref = _cdc_numpy(x, taps)
        assert np.abs(ref).max() >= 32768
        assert np.array_equal(got, ref) == exact


def test_cdc_synthetic_config1_sample(orc):
    import synth
    f = synth.config1(4096)
    assert np.array_equal(orc.cdc(f.x, f.taps), _cdc_numpy(f.x, f.taps))


def test_cdc_alternative_root_same_result(orc):
    # The other square root of 2 (61457) gives other spectra but the same convolution.
    rng = np.random.default_rng(3)
    x = rng.integers(-16, 16, (400, 2, 2)).astype(np.int8)
    taps = rng.integers(-32, 32, (17, 2)).astype(np.int8)
    assert np.array_equal(orc.cdc(x, taps, 64, 61457), orc.cdc(x, taps, 64, 4080))


# -------------------------------------------------------- requant / resample -----

def test_cdc_shift_and_phase(orc):
    # s = the smallest shift with 4^s >= 2 E
    assert orc.cdc_shift(np.array([[0, 0]], dtype=np.int8)) == 0       # E = 0
    assert orc.cdc_shift(np.array([[1, 0]], dtype=np.int8)) == 1       # 2E = 2: 4^0 < 2 <= 4^1
    assert orc.cdc_shift(np.array([[2, 2]], dtype=np.int8)) == 2       # 2E = 16 = 4^2 (equality)
    assert orc.cdc_shift(np.array([[3, 4]], dtype=np.int8)) == 3       # 2E = 50: 16 < 50 <= 64
    assert orc.cdc_shift(np.array([[31, 31]] * 17, dtype=np.int8)) == 8  # 2E = 65348 <= 4^8 = 65536
    assert [orc.decim_phase(L) for L in (5, 7, 17, 19)] == [0, 1, 0, 1]


@pytest.mark.parametrize("L", [17, 31])
def test_cdc_shift_keeps_the_aeq_input_within_the_adc_loading(orc, L):
    """The reading behind the shift (the paper fixes only the 5-bit width): on
    the synthetic 75 km link, whose 5-bit samples have 5 LSB RMS, the
    requantised AEQ input has at most that RMS and almost never saturates.
    One shift less would load it at 6.5-8.4 LSB RMS with 2-8 % of the samples
    at the rails, the BER floor the synthetic comparison found."""
    import synth
    x = synth.received(synth.rng_for(6, 3), 1 << 15, 2, 75.0, 30.0)
    taps = synth.cd_taps(75.0, L)
    s = orc.cdc_shift(taps)
    xa = orc.requant_decimate(orc.cdc(x, taps), s, orc.decim_phase(L)).astype(np.float64)
    rms_in = np.sqrt(np.mean(x.astype(np.float64) ** 2))
    assert np.sqrt(np.mean(xa ** 2)) <= rms_in
    assert np.mean((xa >= 15) | (xa <= -16)) < 1e-3
    xb = orc.requant_decimate(orc.cdc(x, taps), s - 1, orc.decim_phase(L)).astype(np.float64)
    assert np.mean((xb >= 15) | (xb <= -16)) > 1e-2


def test_requant_decimate_hand_cases(orc):
    z = np.zeros((5, 2, 2), dtype=np.int32)
    z[:, 0, 0] = [7, 100, 8, -9, -8]        # XI
    z[:, 0, 1] = [1000, 0, -1000, 0, 255]   # XQ
    z[:, 1, 0] = [-7, 0, 23, 0, 24]         # YI
    z[:, 1, 1] = [0, 0, 0, 0, -24]          # YQ
    x = orc.requant_decimate(z, 4, 0)       # keep t = 0, 2, 4; round half up, /16
    assert x.shape == (3, 4)
    # XI: (7+8)>>4 = 0, (8+8)>>4 = 1, (-8+8)>>4 = 0
    # XQ: (1000+8)>>4 = 63 -> 15, (-1000+8)>>4 = -62 -> -16, (255+8)>>4 = 16 -> 15
    # YI: (-7+8)>>4 = 0, (23+8)>>4 = 1, (24+8)>>4 = 2
    # YQ: 0, 0, (-24+8)>>4 = -1
    assert x.tolist() == [[0, 15, 0, 0], [1, -16, 1, 0], [0, 15, 2, -1]]
    x1 = orc.requant_decimate(z, 0, 1)      # keep t = 1, 3; shift 0 is a plain clip
    assert x1.tolist() == [[15, 0, 0, 0], [-9, 0, 0, 0]]


# ------------------------------------------------------------------- AEQ -----

def _mimo_numpy(x, W):
    """Exact 4x4 integer MIMO convolution, then the output scaling of the AEQ."""
    n = x.shape[0]
    y = np.zeros((n, 4), dtype=np.int64)
    for s2 in range(4):
        for s1 in range(4):
            y[:, s2] += np.convolve(x[:, s1].astype(np.int64), W[s2, s1].astype(np.int64))[:n]
    return np.clip(y >> 7, -32768, 32767)


@pytest.mark.parametrize("N,alpha,n", [(32, 2, 333), (64, 4080, 500), (32, 2, 16), (64, 4080, 5)])
def test_aeq_fixed_taps_equals_mimo_convolution(orc, N, alpha, n):
    rng = np.random.default_rng(N + n)
    x = rng.integers(-16, 16, (n, 4)).astype(np.int8)
    W = rng.integers(-8192, 8192, (4, 4, 16))
    W[0, 0, :] = -8192                      # extremes of the 14-bit tap
    W[1, 1, :] = 8191
    x[: n // 3, 0] = -16
    T = (W << 16).astype(np.int32) + rng.integers(0, 1 << 16, W.shape).astype(np.int32)
    out, T2 = orc.aeq(x, T, N, alpha, mu_shift=63)
    assert np.array_equal(T2, T)
    assert np.array_equal(out, _mimo_numpy(x, W))


def _rde_cost(x, Wf, A):
    """Float64 RDE cost J = sum_n sum_p (R_p - r_p^2)^2 with z = (W * x) / 2^7 and
    the ring R picked from the integer output (held constant, as in the update)."""
    n = x.shape[0]
    y = np.zeros((n, 4))
    for s2 in range(4):
        for s1 in range(4):
            y[:, s2] += np.convolve(x[:, s1].astype(np.float64), Wf[s2, s1])[:n]
    z = y / 128.0
    J = 0.0
    for p in range(2):
        r2 = z[:, 2 * p] ** 2 + z[:, 2 * p + 1] ** 2
        R = np.where(r2 < 6 * A * A, 2 * A * A, np.where(r2 < 14 * A * A, 10 * A * A, 18 * A * A))
        J += np.sum((R - r2) ** 2)
    return J


@pytest.mark.parametrize("N,alpha", [(32, 2), (64, 4080)])
def test_aeq_gradient_matches_rde_cost_derivative(orc, N, alpha):
    """Eq. (6): one block's update, with mu = 1 (m = 0), is -(2^7 / 4) dJ/dW of the
    RDE cost.  Taps are multiples of 2^7 so the integer output carries no floor
    rounding, and the inputs keep every r^2 away from the ring thresholds."""
    K, A = 16, 64
    S = N - K
    rng = np.random.default_rng(N)
    x = rng.integers(-3, 4, (S, 4)).astype(np.int8)
    W = rng.integers(-6, 7, (4, 4, K)) * 128
    T = (W << 16).astype(np.int32)
    out, T2 = orc.aeq(x, T, N, alpha, mu_shift=0, rde_a=A)
    G = (T2.astype(np.int64) - T.astype(np.int64))
    assert np.abs(G).max() > 0
    # the integer output is the exact continuous one here
    assert np.array_equal(out, _mimo_numpy(x, W))
    z = out.astype(np.float64)
    for p in range(2):                       # no output sits on a ring threshold
        r2 = z[:, 2 * p] ** 2 + z[:, 2 * p + 1] ** 2
        assert np.min(np.abs(r2 - 6 * A * A)) > 0 and np.min(np.abs(r2 - 14 * A * A)) > 0
    Wf = W.astype(np.float64)
    h = 1e-3
    num = np.zeros_like(Wf)
    for idx in np.ndindex(Wf.shape):
        Wp = Wf.copy(); Wp[idx] += h
        Wm = Wf.copy(); Wm[idx] -= h
        num[idx] = (_rde_cost(x, Wp, A) - _rde_cost(x, Wm, A)) / (2 * h)
    expect = -(128.0 / 4.0) * num
    assert np.allclose(G, expect, rtol=1e-6, atol=1e-3 * np.abs(expect).max())


def test_aeq_zero_error_keeps_taps(orc):
    # Every output on the inner ring (z = (A, A) -> r^2 = 2A^2 = R): e = 0, G = 0.
    A = 64
    x = np.full((200, 4), 8, dtype=np.int8)
    W = np.zeros((4, 4, 16), dtype=np.int64)
    for s in range(4):
        W[s, s, 0] = 1024                    # y = 1024 * 8 = 8192, z = 64
    T = (W << 16).astype(np.int32)
    out, T2 = orc.aeq(x, T, 32, 2, mu_shift=0, rde_a=A)
    assert (out == 64).all()
    assert np.array_equal(T2, T)


def test_aeq_fnt_path_equals_direct_path_adaptive(orc):
    import synth
    rng = np.random.default_rng(5)
    x = rng.integers(-16, 16, (700, 4)).astype(np.int8)
    T0 = orc.aeq_init_taps(16, 2048)
    for N, alpha in [(32, 2), (64, 4080)]:
        a, Ta = orc.aeq(x, T0, N, alpha, mu_shift=8)
        b, Tb = orc.aeq(x, T0, N, alpha, mu_shift=8, use_fnt=False)
        assert np.array_equal(a, b) and np.array_equal(Ta, Tb)
        assert not np.array_equal(Ta, T0)


def test_aeq_tap_clamp(orc):
    # Huge gradients drive T into the clamp at -2^29 .. 2^29 - 1 (14-bit W).
    x = np.full((64, 4), 15, dtype=np.int8)
    T0 = orc.aeq_init_taps(16, 8000)
    _, T = orc.aeq(x, T0, 32, 2, mu_shift=0, rde_a=1)
    assert T.min() >= -(1 << 29) and T.max() <= (1 << 29) - 1
    assert (T == -(1 << 29)).any() or (T == (1 << 29) - 1).any()


def test_aeq_segmented_rules(orc):
    rng = np.random.default_rng(9)
    x = rng.integers(-16, 16, (400, 4)).astype(np.int8)
    T0 = orc.aeq_init_taps(16, 2048)
    plain, Tp = orc.aeq(x, T0, 32, 2, mu_shift=8)
    one, T1 = orc.aeq_segmented(x, T0, 32, 2, mu_shift=8, seg_len=1000, warmup=50)
    assert np.array_equal(plain, one) and np.array_equal(Tp, T1)
    seg, Ts = orc.aeq_segmented(x, T0, 32, 2, mu_shift=8, seg_len=128, warmup=40)
    for s0 in range(0, 400, 128):
        b = max(0, s0 - 40)
        e = min(400, s0 + 128)
        h = min(b, 16)                       # the K stream symbols before the run are its history
        ref, Tr = orc.aeq(x[b - h:e], T0, 32, 2, mu_shift=8, hist=h)
        assert np.array_equal(seg[s0:e], ref[s0 - b:])
    assert np.array_equal(Ts, Tr)


def test_aeq_segments_continue_the_stream_with_fixed_taps(orc):
    """With fixed taps (mu = 0) every output depends on the 16 inputs up to it
    alone, so segments that read the stream's preceding symbols as history
    reproduce the unsegmented run exactly, with or without warm-up, ragged
    last segment included -- and equal the plain 4x4 MIMO convolution."""
    rng = np.random.default_rng(19)
    x = rng.integers(-16, 16, (1000, 4)).astype(np.int8)
    W = rng.integers(-8192, 8192, (4, 4, 16)).astype(np.int64)
    T0 = (W << 16).astype(np.int32)
    for N, alpha in ((32, 2), (64, 4080)):
        plain, _ = orc.aeq(x, T0, N, alpha, mu_shift=63)
        for seg_len, warm in ((100, 0), (48, 0), (333, 20), (7, 0)):
            got, _ = orc.aeq_segmented(x, T0, N, alpha, mu_shift=63, seg_len=seg_len, warmup=warm)
            assert np.array_equal(got, plain), (N, seg_len, warm)
    y = np.zeros((1000, 4), np.int64)
    for s2 in range(4):
        for s1 in range(4):
            y[:, s2] += np.convolve(x[:, s1].astype(np.int64), W[s2, s1])[:1000]
    assert np.array_equal(plain, np.clip(y >> 7, -32768, 32767))


def test_aeq_converges_on_synthetic_16qam(orc):
    """Context, not parity: the RDE error falls on the synthetic 75 km link
    (31 CD taps, the AEQ step and centre spike of the BER comparison)."""
    import synth
    n_sym = 1 << 15
    x = synth.received(synth.rng_for(6, 2), 2 * n_sym, 2, 75.0, 22.0)
    prm = orc.ChainParams(mu_shift=6, w0=4096)
    out, _ = orc.chain(x, synth.cd_taps(75.0, 31), prm)
    A = prm.rde_a
    z = out.astype(np.float64)
    err = []
    for p in range(2):
        r2 = z[:, 2 * p] ** 2 + z[:, 2 * p + 1] ** 2
        R = np.where(r2 < 6 * A * A, 2 * A * A, np.where(r2 < 14 * A * A, 10 * A * A, 18 * A * A))
        err.append(np.abs(R - r2) / (A * A))
    e = np.mean(err, axis=0)
    q = len(e) // 4
    assert e[-q:].mean() < 0.85 * e[:q].mean()



def test_aeq_update_period_rules(orc):
    """Update period P: P = 1 is the per-block update.  For P > 1 the blocks of
    one period see the same taps, and after every P-th block (and the last) the
    taps move by floor(sum of the period's gradients / 2^m).  Rebuilt period by
    period from fixed-tap runs: a run at m = 0 with one final update yields the
    summed gradient of every block it covers under fixed taps, so the difference
    of two such runs over nested prefixes is one period's gradient."""
    rng = np.random.default_rng(13)
    S, P, m = 16, 3, 8
    x = rng.integers(-2, 3, (S * 7 + 5, 4)).astype(np.int8)     # 8 blocks, ragged tail
    T0 = orc.aeq_init_taps(16, 2048)
    a, Ta = orc.aeq(x, T0, 32, 2, mu_shift=m)
    b, Tb = orc.aeq(x, T0, 32, 2, mu_shift=m, period=1)
    assert np.array_equal(a, b) and np.array_equal(Ta, Tb)
    got, Tg = orc.aeq(x, T0, 32, 2, mu_shift=m, period=P)
    assert not np.array_equal(got, a)                            # the period changes the result
    n = x.shape[0]
    never = 1 << 30

    def gsum(T, hi):
        """Gradient summed over the blocks of x[:hi] under fixed taps T."""
        if hi == 0:
            return np.zeros(T.shape, np.int64)
        _, Tn = orc.aeq(x[:hi], T, 32, 2, mu_shift=0, period=never)
        assert np.abs(Tn).max() < (1 << 29) - 1                  # no clamp at m = 0
        return Tn.astype(np.int64) - T.astype(np.int64)

    T = T0.copy()
    for lo in range(0, n, P * S):
        hi = min(n, lo + P * S)
        fixed, _ = orc.aeq(x[:hi], T, 32, 2, mu_shift=63)
        assert np.array_equal(got[lo:hi], fixed[lo:hi]), lo
        G = gsum(T, hi) - gsum(T, lo)
        T = np.clip(T.astype(np.int64) + (G >> m), -(1 << 29), (1 << 29) - 1).astype(np.int32)
    assert np.array_equal(Tg, T)
    # P at least the block count: fixed taps throughout, one update at the end
    out1, T1 = orc.aeq(x, T0, 32, 2, mu_shift=m, period=8)
    fixed, _ = orc.aeq(x, T0, 32, 2, mu_shift=63)
    assert np.array_equal(out1, fixed)
    assert np.array_equal(T1, (T0.astype(np.int64) + (gsum(T0, n) >> m)).astype(np.int32))


def _centred_mod_f(v):
    """The signed decode of a residue: v mod F in [0, F), then r - F above 32768."""
    r = np.mod(v, 65537)
    return np.where(r > 32768, r - 65537, r)


def test_aeq_freq_sum_literal_is_centred_residue_of_summed_convolution(orc):
    """freq_sum = 1 (NEXT-1, literal): per output and tap group the four inputs'
    products are summed in Z_F before one inverse transform, so the decoded
    group output is the centred residue mod F of the exact summed convolution,
    sum over S1 of conv(W_g[S2][S1], x_S1) -- wrapped where it exceeds
    constraint (5).  With fixed taps (m = 63) the whole output follows from
    numpy integer convolutions."""
    rng = np.random.default_rng(41)
    n = 200
    x = rng.integers(-16, 16, (n, 4)).astype(np.int8)
    x[::5] = -16
    W = rng.choice([8191, 8000, -8192, 4000, 127], size=(4, 4, 16)).astype(np.int64)
    T0 = (W << 16).astype(np.int32)
    for N, alpha in ((32, 2), (64, 4080)):
        got, _ = orc.aeq(x, T0, N, alpha, mu_shift=63, freq_sum=1)
        exact, _ = orc.aeq(x, T0, N, alpha, mu_shift=63, freq_sum=0)
        y = np.zeros((n, 4), np.int64)
        for s2 in range(4):
            for g, wgt in ((0, 128), (1, 1)):
                tot = np.zeros(n, np.int64)
                for s1 in range(4):
                    wg = (W[s2, s1] >> 7) if g == 0 else (W[s2, s1] & 127)
                    tot += np.convolve(x[:, s1].astype(np.int64), wg)[:n]
                y[:, s2] += wgt * _centred_mod_f(tot)
        ref = np.clip(y >> 7, -32768, 32767).astype(np.int16)
        assert np.array_equal(got, ref), N
        assert not np.array_equal(got, exact)          # the case wraps


def test_aeq_freq_sum_exact_where_bound_holds_and_guarded_mode_always(orc):
    """Where 16 sum|taps| stays within 32767 the summed form decodes exactly, so
    freq_sum = 1 equals the per-pair path; freq_sum = 2 (guarded) equals it for
    every input, adaptation included, whether the guard holds or not."""
    rng = np.random.default_rng(42)
    x = rng.integers(-16, 16, (16 * 9 + 7, 4)).astype(np.int8)
    small = np.zeros((4, 4, 16), np.int64)
    small[[0, 1, 2, 3], [0, 1, 2, 3], 8] = 20                     # hi 0, lo 20 on the diagonal
    small[:, :, 7] = 3
    T_small = (small << 16).astype(np.int32)
    for N, alpha in ((32, 2), (64, 4080)):
        a, Ta = orc.aeq(x, T_small, N, alpha, mu_shift=63, freq_sum=0)
        b, Tb = orc.aeq(x, T_small, N, alpha, mu_shift=63, freq_sum=1)
        assert np.array_equal(a, b) and np.array_equal(Ta, Tb)
        T0 = orc.aeq_init_taps(16, 2048) + rng.integers(-(1 << 22), 1 << 22, (4, 4, 16)).astype(np.int32)
        for T in (T0, T_small, orc.aeq_init_taps(16, 2048)):
            a, Ta = orc.aeq(x, T, N, alpha, mu_shift=8, freq_sum=0)
            c, Tc = orc.aeq(x, T, N, alpha, mu_shift=8, freq_sum=2)
            assert np.array_equal(a, c) and np.array_equal(Ta, Tc)
    with pytest.raises(ValueError):
        orc.aeq(x, T_small, 32, 2, use_fnt=False, freq_sum=1)   # no wrap to model without transforms


def _gradient_closed_form(xh, W, hist, A, S=None):
    """Eq. (6) summed over a whole run with the taps held fixed, from numpy alone.

    xh: int [hist + n, 4]; its first `hist` rows are input history (no output),
    zeros before them.  z comes from the exact 4x4 MIMO convolution (numpy),
    e from the 16QAM ring rule, and
        G[S2][S1][k] = sum_t e_p(S2)[t] z_S2[t] x_S1[t - k]
    over every output time t of the run, x reaching back across block
    boundaries and into the history.  With S given, the inputs before each
    block's first time are zeroed instead: the planted mistake of a gradient
    that forgets the previous block."""
    xh = xh.astype(np.int64)
    n = xh.shape[0] - hist
    K = W.shape[2]
    y = np.zeros((n, 4), np.int64)
    for s2 in range(4):
        for s1 in range(4):
            y[:, s2] += np.convolve(xh[:, s1], W[s2, s1].astype(np.int64))[hist:hist + n]
    z = np.clip(y >> 7, -32768, 32767)
    e = np.zeros((n, 2), np.int64)
    for p in range(2):
        r2 = z[:, 2 * p] ** 2 + z[:, 2 * p + 1] ** 2
        R = np.where(r2 < 6 * A * A, 2 * A * A, np.where(r2 < 14 * A * A, 10 * A * A, 18 * A * A))
        e[:, p] = R - r2
    G = np.zeros((4, 4, K), np.int64)
    t = np.arange(n)
    for k in range(K):
        src = hist + t - k
        xv = np.where(src[:, None] >= 0, xh[np.maximum(src, 0)], 0)
        if S is not None:
            xv = np.where(((t - k) >= (t // S) * S)[:, None], xv, 0)
        for s2 in range(4):
            G[s2, :, k] = (e[:, s2 // 2] * z[:, s2])[:, None].T @ xv
    return z, G


@pytest.mark.parametrize("N,alpha,n,hist", [(32, 2, 16 * 5 + 7, 0), (32, 2, 16 * 6 + 3, 16),
                                            (64, 4080, 48 * 4 + 13, 0), (64, 4080, 48 * 5 + 1, 11)])
def test_aeq_multiblock_gradient_closed_form(orc, N, alpha, n, hist):
    """Eq. (6) across blocks: at m = 0 and an update period of at least the
    block count, the taps stay fixed for the whole run and one final update
    adds the summed gradient, so T_out - T0 must equal the numpy closed form
    over all the run's times, whose x[t - k] crosses block boundaries and
    reaches into the input history.  Four or more blocks, ragged tails, both
    transform sizes.  The same closed form with each block's earlier inputs
    zeroed (a gradient that forgets the previous block) must differ."""
    K, A = 16, 8
    rng = np.random.default_rng(1000 + N + n + hist)
    xh = rng.integers(-4, 5, (hist + n, 4)).astype(np.int8)
    W = rng.integers(-40, 41, (4, 4, K)).astype(np.int64)
    for s in range(4):
        W[s, s, K // 2] = 1024
    T0 = (W << 16).astype(np.int32) + rng.integers(0, 1 << 16, W.shape).astype(np.int32)
    never = 1 << 30
    out, T1 = orc.aeq(xh, T0, N, alpha, mu_shift=0, rde_a=A, period=never, hist=hist)
    z, G = _gradient_closed_form(xh, W, hist, A)
    assert np.array_equal(out, z)
    assert np.abs(T0.astype(np.int64) + G).max() < (1 << 29) - 1      # no clamp
    assert (G != 0).all() or np.count_nonzero(G) > 200
    assert np.array_equal(T1.astype(np.int64) - T0, G)
    _, G_forget = _gradient_closed_form(xh, W, hist, A, S=N - K)
    assert not np.array_equal(G_forget, G)
    if hist:
        xz = xh.copy()
        xz[:hist] = 0
        _, G_nohist = _gradient_closed_form(xz, W, hist, A)
        assert not np.array_equal(G_nohist, G)


@pytest.mark.parametrize("N,alpha,seg_len,warmup", [(32, 2, 100, 40), (64, 4080, 150, 60)])
def test_aeq_segment_gradient_closed_form(orc, N, alpha, seg_len, warmup):
    """The same closed form for the last segment of a segmented run: it starts
    `warmup` symbols before its output segment, from T0, and reads the K
    stream symbols before its start as history; its final taps are T0 plus the
    summed gradient over its run."""
    K, A = 16, 8
    n = 3 * seg_len + 17
    rng = np.random.default_rng(77 + N)
    x = rng.integers(-4, 5, (n, 4)).astype(np.int8)
    W = rng.integers(-40, 41, (4, 4, K)).astype(np.int64)
    for s in range(4):
        W[s, s, K // 2] = 1024
    T0 = (W << 16).astype(np.int32)
    never = 1 << 30
    _, Tout = orc.aeq_segmented(x, T0, N, alpha, mu_shift=0, rde_a=A, seg_len=seg_len, warmup=warmup,
                                period=never)
    keep = (n - 1) // seg_len * seg_len
    begin = keep - warmup
    hist = min(begin, K)
    z, G = _gradient_closed_form(x[begin - hist:n], W, hist, A)
    assert np.abs(T0.astype(np.int64) + G).max() < (1 << 29) - 1
    assert np.array_equal(Tout.astype(np.int64) - T0, G)
    _, G_forget = _gradient_closed_form(x[begin - hist:n], W, hist, A, S=N - K)
    assert not np.array_equal(G_forget, G)
