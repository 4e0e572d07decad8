"""GPU parity of the CTA-per-chain AEQ kernel (aeq_serial.cu) against the CPU
oracle and against the warp-per-chain kernel: long serial chains under the
paper's update rule (eq. (6)), batches of uneven frames with carried states,
segments, more chains than SMs, prepared graph batches.  Bit-exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_04253_gb300 as F  # noqa: E402
import synth  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def poison(shape):
    return torch.full(shape, 0x3C3C, dtype=torch.int16, device="cuda")


def plan_for(kernel, **kw):
    p = F.Plan(**kw)
    p.set_aeq_kernel(kernel)
    return p


@pytest.mark.parametrize("na,alpha,n", [(32, 2, (1 << 17) + 3), (64, 4080, (1 << 15) + 29)])
def test_long_chain_matches_oracle(orc, na, alpha, n):
    """One chain of thousands of blocks (8193 at N = 32, as the longest cfg-3
    frame; 683 at N = 64), adaptive from random taps, state in and out."""
    rng = np.random.default_rng(na + n)
    x = rng.integers(-16, 16, (n, 4)).astype(np.int8)
    T0 = orc.aeq_init_taps(16, 2048) + rng.integers(-(1 << 21), 1 << 21, (4, 4, 16)).astype(np.int32)
    ref, Tr = orc.aeq(x, T0, na, alpha, mu_shift=9, rde_a=64)
    for kernel in (2, 1):
        st = dev(T0)
        out = poison((n, 4))
        F.aeq_run(plan_for(kernel, n_aeq=na, alpha_aeq=alpha, mu_shift=9), [F.Frame(dev(x), out, state=st)])
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), kernel
        assert np.array_equal(st.cpu().numpy(), Tr), kernel


@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
def test_chain_batch_uneven_frames_both_kernels(orc, na, alpha):
    """Chain batch of frames of uneven length (one empty, one shorter than a
    block), different CD taps, half of them with a carried state."""
    rng = np.random.default_rng(11 + na)
    lens = [0, 7, 900, 5000, 12345, 333, 2048, 64]
    frames_np = []
    for i, n in enumerate(lens):
        L = [5, 7, 17, 19, 11, 17, 13, 3][i]
        taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
        x = rng.integers(-16, 16, (n, 2, 2)).astype(np.int8)
        T0 = orc.aeq_init_taps(16, 2048) + rng.integers(-(1 << 20), 1 << 20, (4, 4, 16)).astype(np.int32)
        frames_np.append((x, taps, T0 if i % 2 else None))
    kw = dict(n_aeq=na, alpha_aeq=alpha, mu_shift=10)
    prm = orc.ChainParams(**kw)
    results = {}
    for kernel in (2, 1):
        frames, outs, states = [], [], []
        for x, taps, T0 in frames_np:
            o = poison((F.chain_nsym(x.shape[0], taps.shape[0]), 4))
            st = None if T0 is None else dev(T0)
            frames.append(F.Frame(dev(x), o, taps, st))
            outs.append(o)
            states.append(st)
        F.cdc_aeq_run(plan_for(kernel, **kw), frames)
        torch.cuda.synchronize()
        results[kernel] = ([o.cpu().numpy() for o in outs], [None if s is None else s.cpu().numpy() for s in states])
    for i, (x, taps, T0) in enumerate(frames_np):
        ref, Tr = orc.chain(x, taps, prm, T0=T0)
        for kernel in (2, 1):
            got, sts = results[kernel]
            assert np.array_equal(got[i], ref), (kernel, i)
            if T0 is not None:
                assert np.array_equal(sts[i], Tr), (kernel, i)


@pytest.mark.parametrize("na,alpha", [(32, 2), (64, 4080)])
def test_segmented_chain_on_cta_kernel(orc, na, alpha):
    """Segments with warm-up and stream history, update period 3, on the CTA
    kernel (40 items)."""
    f = synth.config2(40000)
    kw = dict(n_aeq=na, alpha_aeq=alpha, mu_shift=9)
    plan = plan_for(2, aeq_segment=1000, aeq_warmup=96, aeq_update_period=3, **kw)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out = poison((nsym, 4))
    T0 = orc.aeq_init_taps(16, 2048)
    st = dev(T0)
    F.cdc_aeq_run(plan, [F.Frame(dev(f.x), out, f.taps, st)])
    torch.cuda.synchronize()
    ref, Tr = orc.chain(f.x, f.taps, orc.ChainParams(seg_len=1000, warmup=96, period=3, **kw), T0=T0)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(st.cpu().numpy(), Tr)


def test_more_chains_than_sms_both_kernels_equal(orc):
    """600 frames (1200 items, several CTA waves): the two kernels give the
    same bits; a few frames checked against the oracle."""
    rng = np.random.default_rng(21)
    n = 600
    xs = [rng.integers(-16, 16, (int(m), 4)).astype(np.int8) for m in rng.integers(1, 900, n)]
    T0s = [orc.aeq_init_taps(16, 2048) + rng.integers(-(1 << 20), 1 << 20, (4, 4, 16)).astype(np.int32)
           for _ in range(n)]
    got = {}
    for kernel in (2, 1):
        outs, sts, frames = [], [], []
        for x, T0 in zip(xs, T0s):
            o = poison((x.shape[0], 4))
            s = dev(T0)
            frames.append(F.Frame(dev(x), o, state=s))
            outs.append(o)
            sts.append(s)
        F.aeq_run(plan_for(kernel, mu_shift=8), frames)
        torch.cuda.synchronize()
        got[kernel] = ([o.cpu().numpy() for o in outs], [s.cpu().numpy() for s in sts])
    for i in range(n):
        assert np.array_equal(got[1][0][i], got[2][0][i]), i
        assert np.array_equal(got[1][1][i], got[2][1][i]), i
    for i in (0, 17, n - 1):
        ref, Tr = orc.aeq(xs[i], T0s[i], 32, 2, mu_shift=8, rde_a=64)
        assert np.array_equal(got[2][0][i], ref) and np.array_equal(got[2][1][i], Tr)


def test_prepared_graph_batch_serial_stream_carries_taps(orc):
    """The cfg-2 shape on a short stream: a prepared graph batch of the chain
    with the AEQ unsegmented (the paper's update rule over the whole stream),
    launched twice on a carried state; each launch continues the adaptation."""
    f = synth.config2(1 << 14)
    kw = dict(n_aeq=64, alpha_aeq=4080, mu_shift=9)
    plan = F.Plan(**kw)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out = poison((nsym, 4))
    T0 = orc.aeq_init_taps(16, 2048)
    st = dev(T0)
    b = F.Batch(plan, [F.Frame(dev(f.x), out, f.taps, st)], F.OP_CHAIN, use_graph=True)
    T = T0
    for _ in range(2):
        b.launch()
        torch.cuda.synchronize()
        ref, T = orc.chain(f.x, f.taps, orc.ChainParams(**kw), T0=T)
        assert np.array_equal(out.cpu().numpy(), ref)
        assert np.array_equal(st.cpu().numpy(), T)


def test_automatic_kernel_choices():
    """The automatic choices the launches make (results never depend on them):
    the CTA-per-chain AEQ for few long chains only, never with summation in
    Z_F; the split-block CDC below two 32-block items per SM."""
    p = F.Plan(n_aeq=64, alpha_aeq=4080)
    assert p.aeq_kernel_for(1, 1 << 20) == 2                 # one long stream
    assert p.aeq_kernel_for(76, 256 * 48) == 2               # 152 items, 256 blocks
    assert p.aeq_kernel_for(76, 256 * 48 - 48) == 1          # 255 blocks: short chains
    assert p.aeq_kernel_for(77, 1 << 20) == 1                # more items than SMs
    p.set_aeq_kernel(1)
    assert p.aeq_kernel_for(1, 1 << 20) == 1
    p.set_aeq_kernel(2)
    assert p.aeq_kernel_for(1000, 16) == 2
    fs = F.Plan(aeq_freq_sum=2)
    fs.set_aeq_kernel(2)
    assert fs.aeq_kernel_for(1, 1 << 20) == 1                # summation lives in the warp kernel
    c = F.Plan()
    assert c.cdc_kernel_for(43) == 2 and c.cdc_kernel_for(303) == 2 and c.cdc_kernel_for(304) == 1
    c.set_cdc_kernel(1)
    assert c.cdc_kernel_for(1) == 1
