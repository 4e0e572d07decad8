"""The synthetic BER comparison (ber/): the decisions, Gray mapping, alignment
and counting that every scheme shares, pinned to closed forms; the
floating-point comparison receiver pinned on noiseless and mixed signals; and
the integer FNT chain (through the CPU oracle) converging on the synthetic
75 km channel at the CD filter length the comparison uses."""
import math

import numpy as np

import ber
import synth


def test_gray_bits_and_decisions():
    lv = ber.LEVELS
    b = ber.gray_bits(lv)
    assert {tuple(r) for r in b} == {(0, 0), (0, 1), (1, 1), (1, 0)}
    for i in range(3):                                    # neighbours differ in one bit
        assert int(np.abs(b[i] - b[i + 1]).sum()) == 1
    v = np.array([-9.0, -2.01, -1.99, -0.01, 0.01, 1.99, 2.01, 9.0])
    assert np.array_equal(ber.decide(v), [-3, -3, -1, -1, 1, 1, 3, 3])


def test_count_recovers_delay_order_and_gain():
    rng = np.random.default_rng(1)
    s = synth.qam16(rng, 2, 20000)
    d = 7
    z = np.zeros((2, 20000 - d), complex)
    g = [1.7 * np.exp(0.4j), 0.6 * np.exp(-2.1j)]
    z[0] = g[0] * s[1, d:]                                 # output 0 carries polarisation 1, delayed
    z[1] = g[1] * s[0, d:]
    c = ber.count_errors(z, s, skip=1000)
    assert c.errors == 0 and c.bits == 2 * 4 * (20000 - d - 1000)
    assert [p[0] for p in c.per_pol] == [1, 0] and all(p[1] == d for p in c.per_pol)
    assert abs(c.per_pol[0][2] - 1.7) < 1e-9 and abs(c.per_pol[1][2] - 0.6) < 1e-9
    # one level moved by one step: exactly one bit error
    z[0, 5000] += 2.0 * g[0] * (1 if s[1, 5000 + d].real < 0 else -1)
    assert ber.count_errors(z, s, skip=1000).errors == 1


def test_awgn_ber_matches_gray_16qam_closed_form():
    """Symbols plus white Gaussian noise, no channel: the counted BER equals
    the Gray 16QAM bit error probability per real dimension,
    (3/4) Q(1/sigma) + (1/2) Q(3/sigma) - (1/4) Q(5/sigma), within 5 standard
    deviations of the count."""
    rng = np.random.default_rng(2)
    n = 1 << 18
    s = synth.qam16(rng, 2, n)
    sigma = 0.42
    z = s + sigma * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    c = ber.count_errors(z, s, skip=0, max_delay=2)
    Q = lambda x: 0.5 * math.erfc(x / math.sqrt(2))
    p = 0.75 * Q(1 / sigma) + 0.5 * Q(3 / sigma) - 0.25 * Q(5 / sigma)
    # the gain fitted on the known symbols is within 1e-3 of 1 at this n
    assert abs(c.ber - p) < 5 * math.sqrt(p / c.bits) + 2e-3 * p, (c.ber, p)


def test_fd_cdc_undoes_the_fibre_on_a_noiseless_signal():
    """Without noise, the ideal FD-CDC and 2:1 decimation at the symbol
    instants leave the Jones-mixed symbols of the raised-cosine channel: a
    2 x 2 least-squares fit recovers them to within 1 % EVM, away from the
    frame edges (the whole-frame transform is circular)."""
    n_sym = 1 << 14
    tr = synth.transmission(synth.rng_for(6, 99), 2 * n_sym, 2, 75.0, 200.0)
    c = ber.fd_cdc(tr.analog, 75.0)[:, 0::2]
    t = np.arange(2000, n_sym - 2000)
    M = tr.symbols[:, t] @ np.linalg.pinv(c[:, t])
    e = M @ c[:, t] - tr.symbols[:, t]
    evm = math.sqrt(np.mean(np.abs(e) ** 2) / 10.0)
    assert evm < 0.01, evm


def test_float_receiver_converges_on_a_clean_signal():
    """The comparison receiver's blind RDE converges within 2^16 symbols at
    22 dB (its step of 3e-5 needs more than 2^15): BER below 1e-4 after it."""
    n_sym = 1 << 17
    tr = synth.transmission(synth.rng_for(6, 1), 2 * n_sym, 2, 75.0, 22.0)
    c = ber.count_errors(ber.float_receiver(tr.analog, 75.0), tr.symbols, skip=n_sym // 2)
    assert c.ber < 1e-4, c


def test_snr_at_ber_interpolates_log_linearly():
    snrs = [10.0, 12.0, 14.0, 16.0]
    bers = [10 ** (-0.25 * s) for s in snrs]             # log10 BER linear in SNR
    t = 10 ** (-0.25 * 13.3)
    assert abs(ber.snr_at_ber(snrs, bers, t) - 13.3) < 1e-9
    assert ber.snr_at_ber(snrs, bers, 1e-9) is None
    assert ber.snr_at_ber([10.0, 12.0], [0.1, 0.0], 1e-3) is None   # a zero count is not a crossing


def test_integer_chain_converges_on_the_75km_channel(orc):
    """The integer FNT-CDC + FNT-AEQ chain (oracle) with 31 CD taps at 22 dB:
    blind RDE convergence from the centre spike within 2^16 symbols and a BER
    after it below 5e-3 on both polarisations."""
    n_sym = 1 << 17
    tr = synth.transmission(synth.rng_for(6, 0), 2 * n_sym, 2, 75.0, 22.0)
    taps = synth.cd_taps(75.0, 31)
    out, _ = orc.chain(tr.x, taps, orc.ChainParams(n_aeq=32, alpha_aeq=2, mu_shift=6, w0=4096))
    c = ber.count_errors(ber.chain_to_complex(out), tr.symbols, skip=n_sym // 2)
    assert c.ber < 5e-3, c
    assert all(e / nb < 5e-3 for _, _, _, e, nb in c.per_pol), c.per_pol


def test_bench_ber_host_job():
    """bench.py's host job of the BER workload (one SNR and draw): the 5-bit
    samples and symbols it hands to the GPU chain, and the two float
    receivers' BERs, here on a short transmission (no GPU)."""
    import bench
    r = bench._ber_float_job((24.0, 5, 1 << 13, 1 << 12, 32))
    assert r["x"].shape == (1 << 14, 2, 2) and r["x"].dtype == np.int8
    assert r["symbols"].shape == (2, 1 << 13)
    assert 0.0 <= r["float_fd_cdc"] <= 1.0 and 0.0 <= r["float_same_taps"] <= 1.0
    tr = synth.transmission(synth.rng_for(6, 5), 1 << 14, 2, 75.0, 24.0)
    assert np.array_equal(r["x"], tr.x) and np.array_equal(r["symbols"], tr.symbols)
