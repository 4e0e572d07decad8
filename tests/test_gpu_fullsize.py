"""Full-size workloads in the launch configuration bench.py times, checked on
samples the oracle recomputes one by one: the 2^27-sample stream (AEQ N = 32,
2^16-symbol segments with 2^12 warm-up, two-polarisation CDC items) and the
batch of 4096 uneven frames (5-19 taps, fresh AEQ per frame)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_04253_gb300 as F  # noqa: E402
import synth  # noqa: E402

MU = 9


def test_stream_2pow27_sampled_segments(orc):
    f = synth.config5()
    assert f.x.shape == (1 << 27, 2, 2) and f.taps.shape[0] == 19
    seg, warm = 1 << 16, 1 << 12
    plan = F.Plan(n_aeq=32, alpha_aeq=2, mu_shift=MU, aeq_segment=seg, aeq_warmup=warm)
    prm = orc.ChainParams(n_aeq=32, alpha_aeq=2, mu_shift=MU, seg_len=seg, warmup=warm)
    T0 = orc.aeq_init_taps(16, 2048)
    st = torch.from_numpy(T0).cuda()
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    out = torch.full((nsym, 4), 0x4444, dtype=torch.int16, device="cuda")
    b = F.Batch(plan, [F.Frame(torch.from_numpy(f.x).cuda(), out, f.taps, st)], F.OP_CHAIN, use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    n_seg = (nsym + seg - 1) // seg
    rng = np.random.default_rng(5)
    for s in sorted({0, 1, n_seg - 1, int(rng.integers(2, n_seg - 1))}):
        keep, ref, Tend = orc.chain_segment(f.x, f.taps, prm, s, T0=T0)
        assert np.array_equal(got[keep:keep + ref.shape[0]], ref), s
        if s == n_seg - 1:
            assert np.array_equal(st.cpu().numpy(), Tend)


def test_batch_of_4096_frames_sampled(orc):
    frames_np = synth.config3()
    assert len(frames_np) == 4096
    plan = F.Plan(n_aeq=32, alpha_aeq=2, mu_shift=MU)
    frames = []
    for fn in frames_np:
        o = torch.full((F.chain_nsym(fn.x.shape[0], fn.taps.shape[0]), 4), 0x4444, dtype=torch.int16,
                       device="cuda")
        frames.append(F.Frame(torch.from_numpy(fn.x).cuda(), o, fn.taps))
    b = F.Batch(plan, frames, F.OP_CHAIN, use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    lens = np.array([fn.x.shape[0] for fn in frames_np])
    rng = np.random.default_rng(6)
    pick = {int(np.argmax(lens)), int(np.argmin(lens)), *rng.integers(0, len(frames_np), 3).tolist()}
    for i in sorted(pick):
        ref, _ = orc.chain(frames_np[i].x, frames_np[i].taps, orc.ChainParams(mu_shift=MU))
        assert np.array_equal(frames[i].out.cpu().numpy(), ref), i


def test_cfg2_stream_serial_recurrence_whole_output(orc):
    """The bench's headline workload in its launch configuration: the 2^21-
    sample stream (2^20 symbols per polarisation, 17 taps, AEQ N = 64) as one
    prepared graph batch with the AEQ unsegmented, so that eq. (6) updates the
    taps after every one of the 21846 blocks of each polarisation's serial
    recurrence (the CTA-per-chain kernel).  Every output symbol and the final
    taps are compared with the oracle; a second launch continues from the
    carried taps and is compared on its first and last blocks."""
    f = synth.config2()
    assert f.x.shape == (1 << 21, 2, 2) and f.taps.shape[0] == 17
    kw = dict(n_aeq=64, alpha_aeq=4080, mu_shift=MU)
    plan = F.Plan(**kw)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    assert plan.aeq_kernel_for(1, nsym) == 2
    out = torch.full((nsym, 4), 0x4444, dtype=torch.int16, device="cuda")
    T0 = orc.aeq_init_taps(16, 2048)
    st = torch.from_numpy(T0).cuda()
    b = F.Batch(plan, [F.Frame(torch.from_numpy(f.x).cuda(), out, f.taps, st)], F.OP_CHAIN, use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    T1 = st.cpu().numpy()
    ref, Tr = orc.chain(f.x, f.taps, orc.ChainParams(**kw), T0=T0)
    assert np.array_equal(got, ref)
    assert np.array_equal(T1, Tr)
    b.launch()
    torch.cuda.synchronize()
    got2 = out.cpu().numpy()
    head, _ = orc.chain(f.x[: 48 * 2 * 40], f.taps, orc.ChainParams(**kw), T0=Tr)
    assert np.array_equal(got2[: head.shape[0] - 24], head[: head.shape[0] - 24])
    assert not np.array_equal(got2, got)


def test_ber_link_chain_matches_oracle(orc):
    """The configuration of the synthetic BER comparison: 75 km at 22 dB with
    the library's longest CD filter (31 taps, S = 34), AEQ N = 32 adapting from
    a centre spike of 4096 with mu_shift 6, 2^17 symbols per polarisation.
    Every output symbol of the GPU chain equals the oracle's."""
    n_sym = 1 << 17
    tr = synth.transmission(synth.rng_for(6, 0), 2 * n_sym, 2, 75.0, 22.0)
    taps = synth.cd_taps(75.0, 31)
    plan = F.Plan(n_aeq=32, alpha_aeq=2, mu_shift=6, tap_init=4096)
    nsym = F.chain_nsym(tr.x.shape[0], 31)
    out = torch.full((nsym, 4), 0x5555, dtype=torch.int16, device="cuda")
    F.cdc_aeq_run(plan, [F.Frame(torch.from_numpy(tr.x).cuda(), out, taps)])
    torch.cuda.synchronize()
    ref, _ = orc.chain(tr.x, taps, orc.ChainParams(n_aeq=32, alpha_aeq=2, mu_shift=6, w0=4096))
    assert np.array_equal(out.cpu().numpy(), ref)
