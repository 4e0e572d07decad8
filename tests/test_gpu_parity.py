"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element
by element on seeded inputs.  Every comparison is bit-exact (integer work)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_04253_gb300 as F  # noqa: E402
import synth  # noqa: E402


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def i16(shape):
    return torch.full(shape, 0x5A5A, dtype=torch.int16, device="cuda")   # poison


def run_cdc(plan, x, taps):
    xd = dev(x)
    out = i16((x.shape[0], x.shape[1], 2))
    F.cdc_run(plan, [F.Frame(xd, out, taps, n_pol=x.shape[1])])
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int32)


# --------------------------------------------------------------------- CDC -----

CDC_CASES = [(1000, 1, 17), (777, 2, 19), (3000, 2, 5), (64, 1, 17), (47, 2, 17), (1, 2, 17),
             (0, 2, 17), (333, 1, 1), (5000, 2, 31), (48 * 32 * 3 + 7, 2, 17), (20000, 2, 12)]


def cdc_plan(cdck, **kw):
    """CDC kernel 1: a block per lane; 2: a block per 8 threads (four-step)."""
    plan = F.Plan(**kw)
    plan.set_cdc_kernel(cdck)
    return plan


@pytest.mark.parametrize("cdck", [1, 2])
@pytest.mark.parametrize("n,n_pol,L", CDC_CASES)
def test_cdc_random_matches_oracle(orc, n, n_pol, L, cdck):
    rng = np.random.default_rng(100 + n + L)
    x = rng.integers(-16, 16, (n, n_pol, 2)).astype(np.int8)
    taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
    plan = cdc_plan(cdck)
    got = run_cdc(plan, x, taps)
    assert np.array_equal(got, orc.cdc(x, taps) if n else np.zeros((0, n_pol, 2), np.int32))


@pytest.mark.parametrize("cdck", [1, 2])
@pytest.mark.parametrize("step,L", [(32, 17), (40, 17), (48, 17), (32, 31), (34, 31)])
def test_cdc_custom_step(orc, step, L, cdck):
    """Includes the Tab. 1 operating point: 50 % overlap (S = 32) with up to
    31 taps, worst-case magnitudes included."""
    rng = np.random.default_rng(step + L)
    x = rng.integers(-16, 16, (4000, 2, 2)).astype(np.int8)
    x[:700] = -16
    taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
    taps[: L // 2] = -32
    got = run_cdc(cdc_plan(cdck, cdc_step=step), x, taps)
    assert np.array_equal(got, orc.cdc(x, taps, 64, 4080, step))


@pytest.mark.parametrize("cdck", [1, 2])
def test_cdc_extremes(orc, cdck):
    n = 4096
    for xv, hv in [(-16, -32), (15, 31), (-16, 31), (-1, -1)]:
        x = np.full((n, 2, 2), xv, dtype=np.int8)
        x[::7, 1, 0] = -xv - 1 if xv < 15 else -16
        taps = np.full((31, 2), hv, dtype=np.int8)
        got = run_cdc(cdc_plan(cdck), x, taps)
        assert np.array_equal(got, orc.cdc(x, taps))


@pytest.mark.parametrize("cdck", [0, 1, 2])
def test_cdc_synthetic_config1(orc, cdck):
    f = synth.config1()
    got = run_cdc(cdc_plan(cdck), f.x, f.taps)
    assert np.array_equal(got, orc.cdc(f.x, f.taps))


@pytest.mark.parametrize("cdck", [1, 2])
@pytest.mark.parametrize("pols", [0, 1, 2])
def test_cdc_batch_of_mixed_frames(orc, pols, cdck):
    """Items of one or of both polarisations (single-pol frames always take one)."""
    rng = np.random.default_rng(77)
    plan = cdc_plan(cdck)
    plan.set_cdc_items(pols)
    frames, refs = [], []
    for i in range(9):
        n = int(rng.integers(0, 9000))
        npol = int(rng.integers(1, 3))
        L = int(rng.integers(1, 32))
        x = rng.integers(-16, 16, (n, npol, 2)).astype(np.int8)
        taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
        out = i16((n, npol, 2))
        frames.append(F.Frame(dev(x), out, taps, n_pol=npol))
        refs.append(orc.cdc(x, taps) if n else np.zeros((0, npol, 2), np.int32))
    F.cdc_run(plan, frames)
    torch.cuda.synchronize()
    for fr, ref in zip(frames, refs):
        assert np.array_equal(fr.out.cpu().numpy().astype(np.int32), ref)


def test_cdc_window_bulk_copy_and_its_bounded_wait(orc):
    """The one-block-per-lane CDC fetches a PDM item's windows with one TMA
    bulk copy: bit-exact, no fault recorded.  With the test hook the copy is
    armed but never issued: the bounded wait runs out, the device fault word
    records it, and the next normal call is exact again."""
    rng = np.random.default_rng(91)
    n = 48 * 32 * 20 + 77
    x = rng.integers(-16, 16, (n, 2, 2)).astype(np.int8)
    taps = rng.integers(-32, 32, (17, 2)).astype(np.int8)
    ref = orc.cdc(x, taps)
    F.device_faults(clear=True)
    assert np.array_equal(run_cdc(cdc_plan(1), x, taps), ref)
    assert F.device_faults() == 0
    bad = cdc_plan(1)
    bad.set_test_inject(1)
    run_cdc(bad, x, taps)
    assert F.device_faults(clear=True) & F.FAULT_CDC_WINDOW_WAIT
    assert F.device_faults() == 0
    assert np.array_equal(run_cdc(cdc_plan(1), x, taps), ref)
    assert F.device_faults() == 0


def test_cdc_rejects_bad_frames():
    plan = F.Plan()
    x = torch.zeros((100, 2, 2), dtype=torch.int8, device="cuda")
    out = i16((100, 2, 2))
    with pytest.raises(F.FntError) as e:
        F.cdc_run(plan, [F.Frame(x, out, np.zeros((32, 2), np.int8))])
    assert e.value.status == F.FNT_ERR_BOUND
    with pytest.raises(F.FntError) as e:
        F.cdc_run(plan, [F.Frame(x, out, np.full((5, 2), 40, np.int8))])
    assert e.value.status == F.FNT_ERR_INVALID
    with pytest.raises(F.FntError):
        F.Plan(alpha_cdc=2)          # order 32, not 64: eq. (4) fails


# --------------------------------------------------------------------- AEQ -----

# AEQ paths: (kernel, tensor-core gradient).  "warp" is one warp per (chain,
# polarisation), "cta" one CTA per (chain, polarisation); all give the same bits.
AEQ_PATHS = {"warp": (1, False), "warp-mma": (1, True), "cta": (2, False)}


def aeq_plan(path, **kw):
    plan = F.Plan(**kw)
    kernel, tensor = AEQ_PATHS[path]
    plan.set_aeq_kernel(kernel)
    plan.set_tensor_gradient(tensor)
    return plan


def run_aeq(plan, x, T=None):
    xd = dev(x)
    out = i16((x.shape[0], 4))
    st = None if T is None else dev(T)
    F.aeq_run(plan, [F.Frame(xd, out, state=st)])
    torch.cuda.synchronize()
    return out.cpu().numpy(), (None if st is None else st.cpu().numpy())


@pytest.mark.parametrize("path", list(AEQ_PATHS))
@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
@pytest.mark.parametrize("n,mu", [(1000, 8), (333, 12), (16, 8), (5, 8), (2000, 63), (4096 + 3, 6)])
def test_aeq_matches_oracle(orc, na, alpha, n, mu, path):
    rng = np.random.default_rng(na * 1000 + n + mu)
    x = rng.integers(-16, 16, (n, 4)).astype(np.int8)
    T0 = orc.aeq_init_taps(16, 2048)
    T0 = T0 + rng.integers(-(1 << 20), 1 << 20, T0.shape).astype(np.int32)
    plan = aeq_plan(path, n_aeq=na, alpha_aeq=alpha, mu_shift=mu, rde_a=64)
    got, Tg = run_aeq(plan, x, T0)
    ref, Tr = orc.aeq(x, T0, na, alpha, mu_shift=mu, rde_a=64)
    assert np.array_equal(got, ref)
    assert np.array_equal(Tg, Tr)


@pytest.mark.parametrize("path", list(AEQ_PATHS))
@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
def test_aeq_extreme_taps(orc, na, alpha, path):
    """Saturated outputs (|z| = 32767 / 32768), |e| near 2^31 and inputs at both
    ends of the 5-bit range: the largest e z the gradient can see."""
    rng = np.random.default_rng(3)
    x = np.full((700, 4), -16, dtype=np.int8)
    x[::3] = 15
    W = rng.choice([-8192, 8191, -1, 0, 127, -128], size=(4, 4, 16)).astype(np.int64)
    cases = [(W << 16).astype(np.int32)]
    xs = [x]
    x2 = np.full((700, 4), -16, dtype=np.int8)
    x2[::7] = 15
    for wv in (8191, -8192):                       # every tap at an end of the range
        cases.append(np.full((4, 4, 16), wv << 16, dtype=np.int64).astype(np.int32))
        xs.append(x2)
    for xi, T0 in zip(xs, cases):
        for mu, a in ((30, 4096), (40, 1)):
            plan = aeq_plan(path, n_aeq=na, alpha_aeq=alpha, mu_shift=mu, rde_a=a)
            got, Tg = run_aeq(plan, xi, T0)
            ref, Tr = orc.aeq(xi, T0, na, alpha, mu_shift=mu, rde_a=a)
            assert np.array_equal(got, ref) and np.array_equal(Tg, Tr)
    assert np.abs(got.astype(np.int64)).max() >= 32767          # saturated outputs were covered


@pytest.mark.parametrize("path", list(AEQ_PATHS))
@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
@pytest.mark.parametrize("xv", [-1, 15, -16])
def test_aeq_constant_worst_case_inputs(orc, na, alpha, path, xv):
    """Constant inputs at the special residue (-1 maps to 65536 in every
    transform input) and at both ends of the 5-bit range, adapting from the
    plan's taps and from random 14-bit taps."""
    rng = np.random.default_rng(45)
    x = np.full((900, 4), xv, dtype=np.int8)
    Trand = (rng.integers(-8192, 8192, (4, 4, 16)).astype(np.int64) << 16).astype(np.int32)
    for T0 in (orc.aeq_init_taps(16, 2048), Trand):
        plan = aeq_plan(path, n_aeq=na, alpha_aeq=alpha, mu_shift=20)
        got, Tg = run_aeq(plan, x, T0)
        ref, Tr = orc.aeq(x, T0, na, alpha, mu_shift=20, rde_a=64)
        assert np.array_equal(got, ref) and np.array_equal(Tg, Tr)


def test_aeq_no_state_uses_plan_init(orc):
    rng = np.random.default_rng(4)
    x = rng.integers(-16, 16, (900, 4)).astype(np.int8)
    plan = F.Plan(mu_shift=9, tap_init=3000)
    got, _ = run_aeq(plan, x, None)
    ref, _ = orc.aeq(x, orc.aeq_init_taps(16, 3000), 32, 2, mu_shift=9, rde_a=64)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
def test_aeq_segmented_matches_oracle(orc, na, alpha):
    rng = np.random.default_rng(5)
    x = rng.integers(-16, 16, (5000, 4)).astype(np.int8)
    plan = F.Plan(n_aeq=na, alpha_aeq=alpha, mu_shift=9, aeq_segment=700, aeq_warmup=150)
    T0 = orc.aeq_init_taps(16, 2048) + rng.integers(-(1 << 22), 1 << 22, (4, 4, 16)).astype(np.int32)
    # segments start from the state as it was at the call; the state ends with the last segment's taps
    got, Tg = run_aeq(plan, x, T0)
    ref, Tr = orc.aeq_segmented(x, T0, na, alpha, mu_shift=9, rde_a=64, seg_len=700, warmup=150)
    assert np.array_equal(got, ref)
    assert np.array_equal(Tg, Tr)
    # without a state every segment starts from the plan's taps
    got2, _ = run_aeq(plan, x, None)
    ref2, _ = orc.aeq_segmented(x, orc.aeq_init_taps(16, 2048), na, alpha, mu_shift=9, rde_a=64,
                                seg_len=700, warmup=150)
    assert np.array_equal(got2, ref2)


@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("taps", ["init", "random", "wrapping", "small"])
def test_aeq_freq_sum_matches_oracle(orc, na, alpha, mode, taps):
    """Frequency-domain summation over the inputs (literal: wraps like the
    oracle's; guarded: equal to the per-pair path), adaptive, with an update
    period and with the tensor-core gradient too."""
    rng = np.random.default_rng(na + 10 * mode + len(taps))
    x = rng.integers(-16, 16, (1500, 4)).astype(np.int8)
    if taps == "init":
        T0 = orc.aeq_init_taps(16, 2048)
    elif taps == "random":
        T0 = orc.aeq_init_taps(16, 2048) + rng.integers(-(1 << 22), 1 << 22, (4, 4, 16)).astype(np.int32)
    elif taps == "wrapping":
        x[::4] = -16
        T0 = (rng.choice([8191, 8000, -8192, 4000, 127], size=(4, 4, 16)).astype(np.int64) << 16).astype(np.int32)
    else:
        W = np.zeros((4, 4, 16), np.int64)
        W[[0, 1, 2, 3], [0, 1, 2, 3], 8] = 20
        W[:, :, 7] = 3
        T0 = (W << 16).astype(np.int32)
    for mu, period, tensor in ((10, 1, False), (12, 3, True), (63, 1, False)):
        plan = F.Plan(n_aeq=na, alpha_aeq=alpha, mu_shift=mu, aeq_update_period=period, aeq_freq_sum=mode)
        plan.set_tensor_gradient(tensor)
        got, Tg = run_aeq(plan, x, T0)
        ref, Tr = orc.aeq(x, T0, na, alpha, mu_shift=mu, rde_a=64, period=period, freq_sum=mode)
        assert np.array_equal(got, ref), (mu, period, tensor)
        assert np.array_equal(Tg, Tr), (mu, period, tensor)
        if mode == 2:
            base, _ = orc.aeq(x, T0, na, alpha, mu_shift=mu, rde_a=64, period=period)
            assert np.array_equal(got, base)


def test_chain_freq_sum_guarded_segmented(orc):
    f = synth.config2(1 << 14)
    kw = dict(n_aeq=64, alpha_aeq=4080, mu_shift=9)
    plan = F.Plan(aeq_segment=864, aeq_warmup=48, aeq_freq_sum=2, **kw)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out = i16((nsym, 4))
    T0 = orc.aeq_init_taps(16, 2048)
    st = dev(T0)
    F.cdc_aeq_run(plan, [F.Frame(dev(f.x), out, f.taps, st)])
    torch.cuda.synchronize()
    ref, Tr = orc.chain(f.x, f.taps, orc.ChainParams(seg_len=864, warmup=48, **kw), T0=T0)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(st.cpu().numpy(), Tr)


@pytest.mark.parametrize("path", list(AEQ_PATHS))
@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
@pytest.mark.parametrize("period,n", [(2, 1000), (3, 333), (5, 4099), (64, 5000), (64, 700), (4, 16)])
def test_aeq_update_period_matches_oracle(orc, na, alpha, period, n, path):
    """Update period P: the summed gradient of P blocks is applied after every
    P-th block and the last; the taps (and their cached spectra) are fixed in
    between."""
    rng = np.random.default_rng(na + 7 * period + n)
    x = rng.integers(-16, 16, (n, 4)).astype(np.int8)
    T0 = orc.aeq_init_taps(16, 2048) + rng.integers(-(1 << 20), 1 << 20, (4, 4, 16)).astype(np.int32)
    plan = aeq_plan(path, n_aeq=na, alpha_aeq=alpha, mu_shift=12, aeq_update_period=period)
    got, Tg = run_aeq(plan, x, T0)
    ref, Tr = orc.aeq(x, T0, na, alpha, mu_shift=12, rde_a=64, period=period)
    assert np.array_equal(got, ref)
    assert np.array_equal(Tg, Tr)
    if n > 2 * (na - 16) and period < 64:
        every, _ = orc.aeq(x, T0, na, alpha, mu_shift=12, rde_a=64)
        assert not np.array_equal(ref, every)           # the case exercises the period


@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
def test_chain_segmented_update_period_matches_oracle(orc, na, alpha):
    """Periods count from each segment's warm-up start."""
    f = synth.config2(1 << 13)
    kw = dict(n_aeq=na, alpha_aeq=alpha, mu_shift=9)
    plan = F.Plan(aeq_segment=1000, aeq_warmup=120, aeq_update_period=4, **kw)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out = i16((nsym, 4))
    T0 = orc.aeq_init_taps(16, 2048)
    st = dev(T0)
    F.cdc_aeq_run(plan, [F.Frame(dev(f.x), out, f.taps, st)])
    torch.cuda.synchronize()
    prm = orc.ChainParams(seg_len=1000, warmup=120, period=4, **kw)
    ref, Tr = orc.chain(f.x, f.taps, prm, T0=T0)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(st.cpu().numpy(), Tr)


def test_chain_segmented_state_carried_over_calls(orc):
    """A long stream processed call after call: each call's segments start from
    the taps the previous call ended with."""
    f = synth.config2(1 << 13)
    kw = dict(n_aeq=64, alpha_aeq=4080, mu_shift=9, aeq_segment=1024, aeq_warmup=128)
    plan = F.Plan(**kw)
    prm = orc.ChainParams(n_aeq=64, alpha_aeq=4080, mu_shift=9, seg_len=1024, warmup=128)
    xd = dev(f.x)
    T = orc.aeq_init_taps(16, 2048)
    st = dev(T)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    b = F.Batch(plan, [F.Frame(xd, i16((nsym, 4)), f.taps, st)], F.OP_CHAIN, use_graph=True)
    for call in range(3):
        b.launch()
        torch.cuda.synchronize()
        ref, T = orc.chain(f.x, f.taps, prm, T0=T)
        assert np.array_equal(b.frames[0].out.cpu().numpy(), ref), call
        assert np.array_equal(st.cpu().numpy(), T), call


# ------------------------------------------------------------------- chain -----

def oracle_chain(orc, x, taps, **kw):
    prm = orc.ChainParams(**kw)
    return orc.chain(x, taps, prm)


@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
@pytest.mark.parametrize("cdck", [1, 2])
def test_chain_synthetic_matches_oracle(orc, na, alpha, cdck):
    f = synth.config2(1 << 12)
    plan = cdc_plan(cdck, n_aeq=na, alpha_aeq=alpha, mu_shift=9)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out = i16((nsym, 4))
    st = dev(np.zeros((4, 4, 16), np.int32))
    st.copy_(dev(orc.aeq_init_taps(16, 2048)))
    F.cdc_aeq_run(plan, [F.Frame(dev(f.x), out, f.taps, st)])
    torch.cuda.synchronize()
    ref, Tr = oracle_chain(orc, f.x, f.taps, n_aeq=na, alpha_aeq=alpha, mu_shift=9)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(st.cpu().numpy(), Tr)


def test_chain_batch_mixed_lengths_and_taps(orc):
    rng = np.random.default_rng(8)
    plan = F.Plan(mu_shift=9)
    frames, refs = [], []
    for i in range(7):
        n = int(rng.integers(0, 6000))
        L = int(rng.choice([5, 7, 9, 17, 19, 31]))
        x = rng.integers(-16, 16, (n, 2, 2)).astype(np.int8)
        taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
        out = i16((F.chain_nsym(n, L), 4))
        frames.append(F.Frame(dev(x), out, taps))
        refs.append(oracle_chain(orc, x, taps, mu_shift=9)[0])
    F.cdc_aeq_run(plan, frames)
    torch.cuda.synchronize()
    for fr, ref in zip(frames, refs):
        assert np.array_equal(fr.out.cpu().numpy(), ref)


def test_chain_segmented_and_prepared_batch(orc):
    f = synth.config2(1 << 13)
    kw = dict(n_aeq=64, alpha_aeq=4080, mu_shift=9, aeq_segment=1024, aeq_warmup=256)
    plan = F.Plan(**kw)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out1 = i16((nsym, 4))
    out2 = i16((nsym, 4))
    xd = dev(f.x)
    F.cdc_aeq_run(plan, [F.Frame(xd, out1, f.taps)])
    b = F.Batch(plan, [F.Frame(xd, out2, f.taps)], F.OP_CHAIN, use_graph=True)
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    ref, _ = oracle_chain(orc, f.x, f.taps, seg_len=1024, warmup=256, **{k: v for k, v in kw.items()
                                                                         if k in ("n_aeq", "alpha_aeq", "mu_shift")})
    assert np.array_equal(out1.cpu().numpy(), ref)
    assert np.array_equal(out2.cpu().numpy(), ref)
    assert b.kernel_count() == 2


def test_chain_host_buffers_equal_device(orc):
    f = synth.config2(1 << 12)
    plan = F.Plan(mu_shift=9)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    host_out = np.zeros((nsym, 4), np.int16)
    F.cdc_aeq_run(plan, [F.Frame(np.ascontiguousarray(f.x), host_out, f.taps)], host=True)
    ref, _ = oracle_chain(orc, f.x, f.taps, mu_shift=9)
    assert np.array_equal(host_out, ref)


@pytest.mark.parametrize("pin_in,pin_out", [(True, True), (True, False), (False, True)])
def test_host_buffers_pinned_in_place_and_pageable_staged(orc, pin_in, pin_out):
    """host_buffers = 1: page-locked buffers are read and written in place by
    the kernels, pageable ones are staged; every mix gives the oracle's bits,
    for the chain, the CDC alone and the AEQ alone."""
    rng = np.random.default_rng(40)

    def host(a, pinned):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.pin_memory() if pinned else t

    f = synth.config2(1 << 12)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    xin = host(f.x, pin_in)
    out = host(np.full((nsym, 4), 0x3333, np.int16), pin_out)
    F.cdc_aeq_run(F.Plan(mu_shift=9), [F.Frame(xin, out, f.taps)], host=True)
    ref, _ = oracle_chain(orc, f.x, f.taps, mu_shift=9)
    assert np.array_equal(out.numpy(), ref)

    x1 = rng.integers(-16, 16, (3000, 2, 2)).astype(np.int8)
    taps = rng.integers(-32, 32, (19, 2)).astype(np.int8)
    o1 = host(np.zeros((3000, 2, 2), np.int16), pin_out)
    F.cdc_run(F.Plan(), [F.Frame(host(x1, pin_in), o1, taps)], host=True)
    assert np.array_equal(o1.numpy().astype(np.int32), orc.cdc(x1, taps))

    xa = rng.integers(-16, 16, (1500, 4)).astype(np.int8)
    oa = host(np.zeros((1500, 4), np.int16), pin_out)
    F.aeq_run(F.Plan(mu_shift=9), [F.Frame(host(xa, pin_in), oa)], host=True)
    refa, _ = orc.aeq(xa, orc.aeq_init_taps(16, 2048), 32, 2, mu_shift=9, rde_a=64)
    assert np.array_equal(oa.numpy(), refa)


def test_prepared_batch_on_page_locked_host_buffers(orc):
    """A prepared (graph) batch over page-locked host buffers, replayed on a
    carried state, equals the oracle step by step; pageable buffers are refused."""
    f = synth.config2(1 << 13)
    plan = F.Plan(n_aeq=64, alpha_aeq=4080, mu_shift=9, aeq_segment=864, aeq_warmup=48)
    prm = orc.ChainParams(n_aeq=64, alpha_aeq=4080, mu_shift=9, seg_len=864, warmup=48)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    xh = torch.from_numpy(f.x).pin_memory()
    oh = torch.full((nsym, 4), 0x2222, dtype=torch.int16).pin_memory()
    T = orc.aeq_init_taps(16, 2048)
    st = dev(T)
    b = F.Batch(plan, [F.Frame(xh, oh, f.taps, st)], F.OP_CHAIN, use_graph=True, host=True)
    for step in range(2):
        b.launch()
        torch.cuda.synchronize()
        ref, T = orc.chain(f.x, f.taps, prm, T0=T)
        assert np.array_equal(oh.numpy(), ref), step
        assert np.array_equal(st.cpu().numpy(), T), step
    b.close()
    with pytest.raises(F.FntError) as e:
        F.Batch(plan, [F.Frame(torch.from_numpy(f.x), torch.zeros((nsym, 4), dtype=torch.int16), f.taps)],
                F.OP_CHAIN, host=True)
    assert e.value.status == F.FNT_ERR_INVALID


@pytest.mark.parametrize("graph", [True, False])
def test_prepared_host_batch_input_copy(orc, graph):
    """Host-buffer batches with the input copied by DMA ahead of the kernels:
    new data written into the page-locked inputs between launches, two batches
    queued back to back on one stream (the second's copy not waiting for the
    first's kernels), per-stage launches, and switching the copy off again all
    equal the oracle, step by step on a carried state."""
    f = synth.config2(1 << 13)
    rng = np.random.default_rng(41)
    plan = F.Plan(n_aeq=64, alpha_aeq=4080, mu_shift=9, aeq_segment=864, aeq_warmup=0)
    prm = orc.ChainParams(n_aeq=64, alpha_aeq=4080, mu_shift=9, seg_len=864, warmup=0)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    xs = [f.x, rng.integers(-16, 16, f.x.shape).astype(np.int8)]
    xh = [torch.from_numpy(x.copy()).pin_memory() for x in xs]
    oh = [torch.full((nsym, 4), 0x2222, dtype=torch.int16).pin_memory() for _ in xs]
    T = orc.aeq_init_taps(16, 2048)
    st = dev(T)
    bs = [F.Batch(plan, [F.Frame(xh[r], oh[r], f.taps, st)], F.OP_CHAIN, use_graph=graph, host=True) for r in (0, 1)]
    for b in bs:
        b.set_input_copy(True)
    s = torch.cuda.Stream()
    for step in range(3):
        new = [rng.integers(-16, 16, f.x.shape).astype(np.int8) for _ in xs] if step else xs
        for r in (0, 1):
            xh[r].copy_(torch.from_numpy(new[r]))
        bs[0].launch(s)
        bs[1].launch(s)                       # its copy may run during the first batch's kernels
        s.synchronize()
        for r in (0, 1):
            ref, T = orc.chain(new[r], f.taps, prm, T0=T)
            assert np.array_equal(oh[r].numpy(), ref), (step, r)
        assert np.array_equal(st.cpu().numpy(), T), step
    # per-stage launches copy before the CDC stage
    x3 = rng.integers(-16, 16, f.x.shape).astype(np.int8)
    xh[0].copy_(torch.from_numpy(x3))
    bs[0].launch_stage(0, s)
    bs[0].launch_stage(1, s)
    s.synchronize()
    ref, T = orc.chain(x3, f.taps, prm, T0=T)
    assert np.array_equal(oh[0].numpy(), ref)
    # and off again: in-place reads of the host input
    bs[1].set_input_copy(False)
    x4 = rng.integers(-16, 16, f.x.shape).astype(np.int8)
    xh[1].copy_(torch.from_numpy(x4))
    bs[1].launch(s)
    s.synchronize()
    ref, T = orc.chain(x4, f.taps, prm, T0=T)
    assert np.array_equal(oh[1].numpy(), ref)
    for b in bs:
        b.close()
    bd = F.Batch(plan, [F.Frame(dev(f.x), i16((nsym, 4)), f.taps, dev(T))], F.OP_CHAIN)
    with pytest.raises(F.FntError) as e:
        bd.set_input_copy(True)                # device buffers: nothing to copy
    assert e.value.status == F.FNT_ERR_INVALID
    bd.close()


def test_prepared_aeq_batch_input_copy(orc):
    """An AEQ-only host-buffer batch with the input copy: the AEQ stage is the
    one that reads the input, by graph launch and by per-stage launch, on a
    carried state."""
    rng = np.random.default_rng(42)
    plan = F.Plan(mu_shift=9)
    n = 3000
    xh = torch.from_numpy(rng.integers(-16, 16, (n, 4)).astype(np.int8)).pin_memory()
    oh = torch.zeros((n, 4), dtype=torch.int16).pin_memory()
    T = orc.aeq_init_taps(16, 2048)
    st = dev(T)
    b = F.Batch(plan, [F.Frame(xh, oh, None, st)], F.OP_AEQ, use_graph=True, host=True)
    b.set_input_copy(True)
    s = torch.cuda.Stream()
    for step in range(3):
        x = rng.integers(-16, 16, (n, 4)).astype(np.int8)
        xh.copy_(torch.from_numpy(x))
        if step < 2:
            b.launch(s)
        else:
            b.launch_stage(0, s)              # nothing: the op has no CDC stage
            b.launch_stage(1, s)
        s.synchronize()
        ref, T = orc.aeq(x, T, 32, 2, mu_shift=9, rde_a=64)
        assert np.array_equal(oh.numpy(), ref), step
        assert np.array_equal(st.cpu().numpy(), T), step
    b.close()


@pytest.mark.parametrize("tap_init", [2048, 1000])
def test_plan_initial_taps_equal_the_oracle_init(orc, tap_init):
    """The plan's initial AEQ taps (fnt_plan_initial_taps) are the oracle's
    init, and a frame state started from them gives the same bits as a frame
    without a state."""
    plan = F.Plan(mu_shift=9, tap_init=tap_init)
    init = plan.initial_state()
    assert np.array_equal(init, orc.aeq_init_taps(16, tap_init))
    rng = np.random.default_rng(43)
    x = rng.integers(-16, 16, (2000, 4)).astype(np.int8)
    o1, o2 = i16((2000, 4)), i16((2000, 4))
    F.aeq_run(plan, [F.Frame(dev(x), o1)])
    F.aeq_run(plan, [F.Frame(dev(x), o2, None, dev(init))])
    torch.cuda.synchronize()
    assert np.array_equal(o1.cpu().numpy(), o2.cpu().numpy())


@pytest.mark.parametrize("occ,warps", [(4, 4), (12, 4), (20, 2)])
def test_aeq_occupancy_cap_gives_the_same_bits(orc, occ, warps):
    """Capping the AEQ warps per SM (shared memory reserved per CTA) changes
    only residency: a batch of uneven frames with fresh taps gives the same
    bits as without the cap, and a frame equals the oracle."""
    rng = np.random.default_rng(44)
    plan = F.Plan(mu_shift=9)
    lens = [4096, 9000, 20000, 333, 60000]
    fr = [synth.random_frame(rng, n, 2, int(rng.choice([5, 17, 19]))) for n in lens]
    def run(cap):
        plan.set_launch(aeq_warps=warps)
        plan.set_aeq_occupancy(cap)
        outs = [i16((F.chain_nsym(f.x.shape[0], f.taps.shape[0]), 4)) for f in fr]
        F.cdc_aeq_run(plan, [F.Frame(dev(f.x), o, f.taps) for f, o in zip(fr, outs)])
        torch.cuda.synchronize()
        return [o.cpu().numpy() for o in outs]
    base = run(0)
    capped = run(occ)
    for a, b in zip(base, capped):
        assert np.array_equal(a, b)
    ref, _ = orc.chain(fr[3].x, fr[3].taps, orc.ChainParams(mu_shift=9))
    assert np.array_equal(capped[3], ref)
    with pytest.raises(F.FntError):
        plan.set_aeq_occupancy(65)


def test_chain_full_size_cfg2_sampled_segments(orc):
    """The benchmark's workload at full size (2^21 samples per polarisation,
    segments of 864 with stream history, carried state), launched as bench.py
    launches it; sampled segments recomputed one by one by the oracle."""
    f = synth.config2()
    assert f.x.shape == (1 << 21, 2, 2)
    plan = F.Plan(n_aeq=64, alpha_aeq=4080, mu_shift=9, aeq_segment=864, aeq_warmup=0)
    prm = orc.ChainParams(n_aeq=64, alpha_aeq=4080, mu_shift=9, seg_len=864, warmup=0)
    T0 = orc.aeq_init_taps(16, 2048)
    st = dev(T0)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out = i16((nsym, 4))
    xd = dev(f.x)
    b = F.Batch(plan, [F.Frame(xd, out, f.taps, st)], F.OP_CHAIN, use_graph=False)
    b.launch_stage(0)
    b.launch_stage(1)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    # the pipelined graph launch of the same work gives the same bits
    st2 = dev(T0)
    out2 = i16((nsym, 4))
    plan.set_pipeline(4)
    bp = F.Batch(plan, [F.Frame(xd, out2, f.taps, st2)], F.OP_CHAIN, use_graph=True)
    bp.launch()
    torch.cuda.synchronize()
    assert bp.kernel_count() > 2
    assert np.array_equal(out2.cpu().numpy(), got)
    assert torch.equal(st2, st)
    # and so do two-polarisation CDC items with the tensor-core gradient
    st3 = dev(T0)
    out3 = i16((nsym, 4))
    plan.set_pipeline(1)
    plan.set_cdc_items(2)
    plan.set_tensor_gradient(True)
    bt = F.Batch(plan, [F.Frame(xd, out3, f.taps, st3)], F.OP_CHAIN, use_graph=True)
    bt.launch()
    torch.cuda.synchronize()
    assert np.array_equal(out3.cpu().numpy(), got)
    assert torch.equal(st3, st)
    n_seg = (nsym + 863) // 864
    rng = np.random.default_rng(2)
    segs = sorted({0, 1, n_seg // 2, n_seg - 2, n_seg - 1, *rng.integers(0, n_seg, 15).tolist()})
    for s in segs:
        keep, ref, Tend = orc.chain_segment(f.x, f.taps, prm, s, T0=T0)
        assert np.array_equal(got[keep:keep + ref.shape[0]], ref), s
        if s == n_seg - 1:
            assert np.array_equal(st.cpu().numpy(), Tend)


def test_pipelined_batch_equals_oracle_and_unpipelined(orc):
    """Prepared chain batches cut into chunks (CDC of chunk k on the caller's
    stream, AEQ of chunk k on a side stream) give the same bits as one CDC
    launch followed by one AEQ launch, and as the oracle."""
    rng = np.random.default_rng(12)
    frames_np = []
    for _ in range(40):
        n = int(2 ** rng.uniform(10, 14.5))
        L = int(rng.choice([5, 9, 13, 17, 19]))
        frames_np.append((rng.integers(-16, 16, (n, 2, 2)).astype(np.int8),
                          rng.integers(-32, 32, (L, 2)).astype(np.int8)))
    outs = {}
    for chunks, graph, pols in [(4, True, 1), (3, False, 2), (1, False, 0), (5, True, 2)]:
        plan = F.Plan(mu_shift=9)
        plan.set_pipeline(chunks)
        plan.set_cdc_items(pols)
        frames = [F.Frame(dev(x), i16((F.chain_nsym(x.shape[0], t.shape[0]), 4)), t) for x, t in frames_np]
        b = F.Batch(plan, frames, F.OP_CHAIN, use_graph=graph)
        b.launch()
        b.launch()
        torch.cuda.synchronize()
        outs[chunks] = [fr.out.cpu().numpy() for fr in frames]
        if chunks > 1 and graph:
            assert b.kernel_count() > 2
    for a, b_, c, d in zip(outs[4], outs[3], outs[1], outs[5]):
        assert np.array_equal(a, c) and np.array_equal(b_, c) and np.array_equal(d, c)
    for i in (0, 7, 39):
        ref, _ = orc.chain(frames_np[i][0], frames_np[i][1], orc.ChainParams(mu_shift=9))
        assert np.array_equal(outs[4][i], ref)


def test_one_plan_from_two_threads_on_two_streams(orc):
    """A plan is shared by threads: each thread's one-shot calls (pinned host
    buffers, its own stream, its own staging ring, the plan's memory pool)
    return the oracle's bits, call after call, while the other thread runs."""
    import threading
    rng = np.random.default_rng(50)
    plan = F.Plan(mu_shift=9, aeq_segment=512, aeq_warmup=0)
    prm = orc.ChainParams(mu_shift=9, seg_len=512, warmup=0)
    cases = []
    for t in range(2):
        n = int(rng.integers(3000, 9000))
        L = int(rng.choice([5, 17, 19]))
        x = rng.integers(-16, 16, (n, 2, 2)).astype(np.int8)
        taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
        cases.append((x, taps, orc.chain(x, taps, prm)[0]))
    errors = []

    def worker(t):
        try:
            x, taps, ref = cases[t]
            stream = torch.cuda.Stream()
            xh = torch.from_numpy(x).pin_memory()
            oh = torch.zeros(ref.shape, dtype=torch.int16).pin_memory()
            for k in range(25):
                oh.fill_(0x1111)
                F.cdc_aeq_run(plan, [F.Frame(xh, oh, taps)], stream=stream, host=True)
                if not np.array_equal(oh.numpy(), ref):
                    errors.append((t, k))
                    return
        except Exception as e:          # reported below
            errors.append((t, repr(e)))

    th = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join()
    assert errors == []
