"""fnt_cdc_aeq_run_noalloc: the one-frame chain for callers that cannot allocate
device memory where they process a frame (a latency-critical receive loop, or an
application whose own allocator owns all device memory).  Its scratch is a fixed
array inside libfnt; the results must equal those of fnt_cdc_aeq_run bit for
bit, call after call.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_04253_gb300 as F  # noqa: E402
import synth  # noqa: E402


def _poison(nsym):
    return torch.full((nsym, 4), 0x5A5A, dtype=torch.int16, device="cuda")


def test_noalloc_equals_allocating_entry_point_twice_segmented():
    f = synth.config2(1 << 15)
    plan = F.Plan(n_aeq=64, alpha_aeq=4080, mu_shift=9, aeq_segment=2048, aeq_warmup=512)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    x = torch.from_numpy(f.x).cuda()
    ref = _poison(nsym)
    F.cdc_aeq_run(plan, [F.Frame(x, ref, f.taps)])
    torch.cuda.synchronize()
    for _ in range(2):
        out = _poison(nsym)
        F.cdc_aeq_run_noalloc(plan, F.Frame(x, out, f.taps))
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    # segments starting from a carried tap state, two calls in a row
    init = torch.zeros((4, 4, 16), dtype=torch.int32, device="cuda")
    init[[0, 1, 2, 3], [0, 1, 2, 3], 8] = 2048 << 16
    st_ref, st_new = init.clone(), init.clone()
    for call in range(2):
        ref, out = _poison(nsym), _poison(nsym)
        F.cdc_aeq_run(plan, [F.Frame(x, ref, f.taps, st_ref)])
        F.cdc_aeq_run_noalloc(plan, F.Frame(x, out, f.taps, st_new))
        torch.cuda.synchronize()
        assert torch.equal(out, ref), call
        assert torch.equal(st_new, st_ref), call


@pytest.mark.parametrize("period", [1, 3])
def test_noalloc_equals_allocating_entry_point_twice_with_state(period):
    rng = np.random.default_rng(31)
    plan = F.Plan(mu_shift=9, aeq_update_period=period)
    init = torch.zeros((4, 4, 16), dtype=torch.int32, device="cuda")
    init[[0, 1, 2, 3], [0, 1, 2, 3], 8] = 2048 << 16
    st_ref, st_new = init.clone(), init.clone()
    for call in range(2):
        n = int(rng.integers(3000, 9000))
        L = int(rng.choice([5, 17, 19]))
        xh = rng.integers(-16, 16, (n, 2, 2)).astype(np.int8)
        taps = rng.integers(-32, 32, (L, 2)).astype(np.int8)
        x = torch.from_numpy(xh).cuda()
        nsym = F.chain_nsym(n, L)
        ref, out = _poison(nsym), _poison(nsym)
        F.cdc_aeq_run(plan, [F.Frame(x, ref, taps, st_ref)])
        F.cdc_aeq_run_noalloc(plan, F.Frame(x, out, taps, st_new))
        torch.cuda.synchronize()
        assert torch.equal(out, ref), call
        assert torch.equal(st_new, st_ref), call


def test_noalloc_equals_the_oracle(orc):
    """Directly against the CPU oracle: the serial AEQ (one recurrence over the
    frame) and a segmented plan, from the plan's initial taps."""
    f = synth.config2(1 << 12)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    x = torch.from_numpy(f.x).cuda()
    for kw in (dict(n_aeq=64, alpha_aeq=4080, mu_shift=9), dict(mu_shift=9, seg_len=1000, warmup=100)):
        pkw = {k: v for k, v in kw.items() if k not in ("seg_len", "warmup")}
        if "seg_len" in kw:
            pkw.update(aeq_segment=kw["seg_len"], aeq_warmup=kw["warmup"])
        out = _poison(nsym)
        F.cdc_aeq_run_noalloc(F.Plan(**pkw), F.Frame(x, out, f.taps))
        torch.cuda.synchronize()
        ref, _ = orc.chain(f.x, f.taps, orc.ChainParams(**kw))
        assert np.array_equal(out.cpu().numpy(), ref), kw


@pytest.mark.parametrize("limits", ["tables", "serial"])
def test_noalloc_at_its_limits_equals_allocating_entry_point(limits):
    """A frame of exactly FNT_NOALLOC_MAX_SAMPLES samples.  "tables": CDC step
    32 and 256-symbol AEQ segments, so both work tables are at their maximum
    (4096 CDC items, FNT_NOALLOC_MAX_SEGMENTS chains) and the intermediate
    symbols fill their region to the last byte; "serial": the unsegmented AEQ.
    Two calls in a row, bit-exact against fnt_cdc_aeq_run."""
    n = F.NOALLOC_MAX_SAMPLES
    f = synth.config2(n // 2)
    assert f.x.shape[0] == n
    if limits == "tables":
        plan = F.Plan(mu_shift=9, cdc_step=32, aeq_segment=256)
        assert F.chain_nsym(n, f.taps.shape[0]) // 256 == 4096
    else:
        plan = F.Plan(n_aeq=64, alpha_aeq=4080, mu_shift=9)
    nsym = F.chain_nsym(n, f.taps.shape[0])
    x = torch.from_numpy(f.x).cuda()
    init = torch.from_numpy(plan.initial_state()).cuda()
    st_ref, st_new = init.clone(), init.clone()
    for call in range(2):
        ref, out = _poison(nsym), _poison(nsym)
        F.cdc_aeq_run(plan, [F.Frame(x, ref, f.taps, st_ref)])
        F.cdc_aeq_run_noalloc(plan, F.Frame(x, out, f.taps, st_new))
        torch.cuda.synchronize()
        assert torch.equal(out, ref), call
        assert torch.equal(st_new, st_ref), call


def test_noalloc_refuses_a_capturing_stream():
    """The call cannot be captured in a CUDA graph: on a capturing stream it
    returns FNT_ERR_INVALID and enqueues nothing; it works again afterwards."""
    plan = F.Plan(mu_shift=9)
    f = synth.config2(1 << 10)
    nsym = F.chain_nsym(f.x.shape[0], f.taps.shape[0])
    x = torch.from_numpy(f.x).cuda()
    out = _poison(nsym)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        out.add_(0)
        with pytest.raises(F.FntError) as e:
            F.cdc_aeq_run_noalloc(plan, F.Frame(x, out, f.taps), stream=side)
    assert e.value.status == F.FNT_ERR_INVALID
    ref = _poison(nsym)
    F.cdc_aeq_run(plan, [F.Frame(x, ref, f.taps)])
    F.cdc_aeq_run_noalloc(plan, F.Frame(x, out, f.taps))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_noalloc_rejects_frames_beyond_its_scratch():
    """Frames one sample pair beyond the limit, and plans that cut a frame into
    more segments than the table holds.  The buffers have the lengths the
    frames claim, so no access could leave them even past the checks."""
    plan = F.Plan()
    n = F.NOALLOC_MAX_SAMPLES + 2
    taps = np.ones((17, 2), np.int8)
    x = torch.zeros((n, 2, 2), dtype=torch.int8, device="cuda")
    out = torch.zeros((F.chain_nsym(n, 17), 4), dtype=torch.int16, device="cuda")
    with pytest.raises(F.FntError) as e:
        F.cdc_aeq_run_noalloc(plan, F.Frame(x, out, taps))
    assert e.value.status == F.FNT_ERR_BOUND
    tiny = F.Plan(aeq_segment=16, aeq_warmup=0)
    n = F.NOALLOC_MAX_SAMPLES
    with pytest.raises(F.FntError) as e:
        F.cdc_aeq_run_noalloc(tiny, F.Frame(x[:n], out, taps, n=n))
    assert e.value.status == F.FNT_ERR_BOUND
