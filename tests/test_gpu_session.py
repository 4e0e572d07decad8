"""Serving session on the GPU: continuous batching over links with device-
resident AEQ state, checked bit-exactly against the oracle's sequential
per-link processing, alone and in the mix; admission cap, checkpoint/resume,
host-side fault injection."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_04253_gb300 as F  # noqa: E402

MU = 9


def make_links(rng, n_links):
    return [rng.integers(-32, 32, (int(rng.choice([5, 9, 17, 19])), 2)).astype(np.int8) for _ in range(n_links)]


def make_frames(rng, n_links, per_link, lo=200, hi=5000):
    frames = []
    for i in range(n_links * per_link):
        link = int(rng.integers(0, n_links))
        n = int(rng.integers(lo, hi))
        frames.append((link, rng.integers(-16, 16, (n, 2, 2)).astype(np.int8)))
    return frames


def oracle_sequential(orc, links, frames):
    prm = orc.ChainParams(mu_shift=MU)
    T = {l: orc.aeq_init_taps(16, prm.w0) for l in range(len(links))}
    outs = []
    for link, x in frames:
        out, T[link] = orc.chain(x, links[link], prm, T0=T[link])
        outs.append(out)
    return outs, T


def run_session(plan, links, frames, cap=1 << 30, streams=4, one_at_a_time=False, host=False):
    s = F.Session(plan, len(links), cap, streams)
    for l, taps in enumerate(links):
        s.set_link(l, taps)
    outs = [None] * len(frames)
    tickets = {}
    done = 0
    for i, (link, x) in enumerate(frames):
        nsym = F.chain_nsym(x.shape[0], links[link].shape[0])
        if host:
            xd = torch.from_numpy(x).pin_memory()
            od = torch.zeros((nsym, 4), dtype=torch.int16).pin_memory()
        else:
            xd = torch.from_numpy(x).cuda()
            od = torch.zeros((nsym, 4), dtype=torch.int16, device="cuda")
        torch.cuda.synchronize()
        while True:
            tk = s.try_submit(link, xd, od)
            if tk is not None:
                break
            for c in s.poll(timeout_us=100000):
                assert c["status"] == F.FNT_OK
                done += 1
        tickets[tk] = (i, od)
        if one_at_a_time:
            while s.pending():
                for c in s.poll(timeout_us=100000):
                    assert c["status"] == F.FNT_OK
                    done += 1
    while s.pending():
        for c in s.poll(timeout_us=100000):
            assert c["status"] == F.FNT_OK
            done += 1
    assert done == len(frames)
    for tk, (i, od) in tickets.items():
        outs[i] = od.cpu().numpy()
    states = [s.get_link_state(l) for l in range(len(links))]
    s.close()
    return outs, states


def test_session_mix_matches_sequential_oracle_and_alone(orc):
    rng = np.random.default_rng(21)
    links = make_links(rng, 6)
    frames = make_frames(rng, 6, 4)
    plan = F.Plan(mu_shift=MU)
    ref, Tref = oracle_sequential(orc, links, frames)
    mix, Tmix = run_session(plan, links, frames)
    alone, Talone = run_session(plan, links, frames, one_at_a_time=True, streams=1)
    for i in range(len(frames)):
        assert np.array_equal(mix[i], ref[i]), i
        assert np.array_equal(alone[i], mix[i]), i
    for l in range(len(links)):
        assert np.array_equal(Tmix[l], Tref[l])
        assert np.array_equal(Talone[l], Tref[l])


def test_session_host_pinned_buffers(orc):
    rng = np.random.default_rng(22)
    links = make_links(rng, 3)
    frames = make_frames(rng, 3, 3)
    ref, _ = oracle_sequential(orc, links, frames)
    got, _ = run_session(F.Plan(mu_shift=MU), links, frames, host=True)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_session_admission_cap_refuses_then_admits():
    rng = np.random.default_rng(23)
    links = make_links(rng, 2)
    plan = F.Plan(mu_shift=MU)
    s = F.Session(plan, 2, 64 * 1024, 1)
    for l, t in enumerate(links):
        s.set_link(l, t)
    x = torch.from_numpy(rng.integers(-16, 16, (20000, 2, 2)).astype(np.int8)).cuda()
    o1 = torch.zeros((F.chain_nsym(20000, links[0].shape[0]), 4), dtype=torch.int16, device="cuda")
    o2 = torch.zeros((F.chain_nsym(20000, links[1].shape[0]), 4), dtype=torch.int16, device="cuda")
    t1 = s.submit(0, x, o1)             # 10000 symbols x 4 B = 40 KB of the 64 KB cap
    assert s.try_submit(1, x, o2) is None
    got = []
    while not got:
        got = s.poll(timeout_us=1000000)
    assert got[0]["ticket"] == t1 and got[0]["status"] == F.FNT_OK
    assert s.try_submit(1, x, o2) is not None
    s.close()
    with pytest.raises(F.FntError) as e:
        s2 = F.Session(plan, 1, 64 * 1024, 1)
        s2.set_link(0, links[0])
        big = torch.zeros((200000, 2, 2), dtype=torch.int8, device="cuda")
        ob = torch.zeros((100000, 4), dtype=torch.int16, device="cuda")
        s2.submit(0, big, ob)
    assert e.value.status == F.FNT_ERR_BOUND


def test_session_checkpoint_resume_bit_exact(orc):
    rng = np.random.default_rng(24)
    links = make_links(rng, 2)
    frames = make_frames(rng, 2, 4)
    plan = F.Plan(mu_shift=MU)
    full, Tfull = run_session(plan, links, frames)
    k = len(frames) // 2
    first, Tmid = run_session(plan, links, frames[:k])
    s = F.Session(plan, len(links), 1 << 30, 2)
    for l, taps in enumerate(links):
        s.set_link(l, taps)
        s.set_link_state(l, Tmid[l])
    outs = []
    for link, x in frames[k:]:
        od = torch.zeros((F.chain_nsym(x.shape[0], links[link].shape[0]), 4), dtype=torch.int16, device="cuda")
        s.submit(link, torch.from_numpy(x).cuda(), od)
        outs.append(od)
    while s.pending():
        for c in s.poll(timeout_us=100000):
            assert c["status"] == F.FNT_OK
    for i, od in enumerate(outs):
        assert np.array_equal(od.cpu().numpy(), full[k + i])
    for l in range(len(links)):
        assert np.array_equal(s.get_link_state(l), Tfull[l])
    s.close()


def test_session_injected_failure_recovers(orc):
    rng = np.random.default_rng(25)
    links = make_links(rng, 1)
    plan = F.Plan(mu_shift=MU)
    s = F.Session(plan, 1, 1 << 28, 1)
    s.set_link(0, links[0])
    x = rng.integers(-16, 16, (3000, 2, 2)).astype(np.int8)
    xd = torch.from_numpy(x).cuda()
    od = torch.zeros((F.chain_nsym(3000, links[0].shape[0]), 4), dtype=torch.int16, device="cuda")
    T0 = s.get_link_state(0)
    s.inject_failures(1)
    s.submit(0, xd, od)
    res = []
    while not res:
        res = s.poll(timeout_us=1000000)
    assert res[0]["status"] == F.FNT_ERR_CUDA
    assert np.array_equal(s.get_link_state(0), T0)          # state untouched
    s.submit(0, xd, od)
    res = []
    while not res:
        res = s.poll(timeout_us=1000000)
    assert res[0]["status"] == F.FNT_OK
    ref, _ = orc.chain(x, links[0], orc.ChainParams(mu_shift=MU))
    assert np.array_equal(od.cpu().numpy(), ref)
    assert s.poll(timeout_us=1000) == []                     # nothing pending: times out
    s.close()


def test_session_rejects_pageable_host_buffers():
    plan = F.Plan()
    s = F.Session(plan, 1, 1 << 20, 1)
    s.set_link(0, np.ones((5, 2), np.int8))
    x = np.zeros((100, 2, 2), np.int8)
    o = np.zeros((50, 4), np.int16)
    with pytest.raises(F.FntError) as e:
        s.submit(0, x, o)
    assert e.value.status == F.FNT_ERR_INVALID
    s.close()


@pytest.mark.parametrize("period", [1, 2])
def test_session_segmented_plan_matches_sequential_oracle(orc, period):
    """With AEQ segments in the plan, each served frame's segments start from
    the link's taps as the frame began; per link this equals sequential oracle
    processing with the same segment rule (and update period)."""
    rng = np.random.default_rng(26)
    links = make_links(rng, 4)
    frames = make_frames(rng, 4, 3, lo=4000, hi=12000)
    plan = F.Plan(mu_shift=MU, aeq_segment=512, aeq_warmup=16, aeq_update_period=period)
    got, Tgot = run_session(plan, links, frames)
    prm = orc.ChainParams(mu_shift=MU, seg_len=512, warmup=16, period=period)
    T = {l: orc.aeq_init_taps(16, prm.w0) for l in range(len(links))}
    for i, (link, x) in enumerate(frames):
        ref, T[link] = orc.chain(x, links[link], prm, T0=T[link])
        assert np.array_equal(got[i], ref), i
    for l in range(len(links)):
        assert np.array_equal(Tgot[l], T[l])


def _device_frames(frames, links, host=False):
    xs, outs = [], []
    for link, x in frames:
        nsym = F.chain_nsym(x.shape[0], links[link].shape[0])
        if host:
            xs.append(torch.from_numpy(x).pin_memory())
            outs.append(torch.zeros((nsym, 4), dtype=torch.int16).pin_memory())
        else:
            xs.append(torch.from_numpy(x).cuda())
            outs.append(torch.zeros((nsym, 4), dtype=torch.int16, device="cuda"))
    torch.cuda.synchronize()
    return xs, outs


def _drain(s, n):
    got = []
    while len(got) < n:
        got.extend(s.poll_array(timeout_us=1000000).tolist())
    return got


@pytest.mark.parametrize("streams,host", [(4, False), (2, True), (8, False)])
def test_session_submit_many_chains_links_on_device(orc, streams, host):
    """A burst admitted with one call: every link's frames are queued behind one
    another on the device (several per link in flight at once) and still give
    the sequential oracle's bits and final taps."""
    rng = np.random.default_rng(27)
    links = make_links(rng, 5)
    frames = make_frames(rng, 5, 6)
    ref, Tref = oracle_sequential(orc, links, frames)
    s = F.Session(F.Plan(mu_shift=MU), len(links), 1 << 30, streams)
    for l, taps in enumerate(links):
        s.set_link(l, taps)
    xs, outs = _device_frames(frames, links, host)
    reqs = F.Requests([l for l, _ in frames], xs, outs)
    tk = s.submit_many(reqs)
    assert len(tk) == len(frames) and len(set(tk)) == len(frames)
    done = _drain(s, len(frames))
    assert all(c[2] == F.FNT_OK for c in done)
    for i in range(len(frames)):
        assert np.array_equal(outs[i].cpu().numpy(), ref[i]), i
    for l in range(len(links)):
        assert np.array_equal(s.get_link_state(l), Tref[l])
    s.close()


def test_session_next_frame_launches_before_previous_completes(orc):
    """With n_streams waves, n_streams frames of ONE link are all launched by the
    admitting call, before any completion is observed: the order between them
    is kept on the device."""
    rng = np.random.default_rng(28)
    links = make_links(rng, 1)
    frames = [(0, rng.integers(-16, 16, (20000, 2, 2)).astype(np.int8)) for _ in range(4)]
    ref, Tref = oracle_sequential(orc, links, frames)
    s = F.Session(F.Plan(mu_shift=MU), 1, 1 << 30, 4)
    s.set_link(0, links[0])
    xs, outs = _device_frames(frames, links)
    tk = s.submit_many(F.Requests([0] * 4, xs, outs))
    done = sorted(_drain(s, 4))                      # by ticket
    assert [c[0] for c in done] == tk
    starts = [c[5] for c in done]
    assert max(starts) < min(c[6] for c in done)
    for i in range(4):
        assert np.array_equal(outs[i].cpu().numpy(), ref[i]), i
    assert np.array_equal(s.get_link_state(0), Tref[0])
    s.close()


def test_session_failed_wave_between_chained_frames(orc):
    """Frame 1 in flight, frame 2's wave fails at launch, frame 3 queued behind
    frame 1 on the device: frames 1 and 3 equal the oracle run over frames 1, 3."""
    rng = np.random.default_rng(29)
    links = make_links(rng, 1)
    frames = [(0, rng.integers(-16, 16, (30000, 2, 2)).astype(np.int8)) for _ in range(3)]
    s = F.Session(F.Plan(mu_shift=MU), 1, 1 << 30, 2)
    s.set_link(0, links[0])
    xs, outs = _device_frames(frames, links)
    t1 = s.submit(0, xs[0], outs[0])
    s.inject_failures(1)
    t2 = s.submit(0, xs[1], outs[1])
    t3 = s.submit(0, xs[2], outs[2])
    res = {c[0]: c[2] for c in _drain(s, 3)}
    assert res == {t1: F.FNT_OK, t2: F.FNT_ERR_CUDA, t3: F.FNT_OK}
    ref, Tref = oracle_sequential(orc, links, [frames[0], frames[2]])
    assert np.array_equal(outs[0].cpu().numpy(), ref[0])
    assert np.array_equal(outs[2].cpu().numpy(), ref[1])
    assert np.array_equal(s.get_link_state(0), Tref[0])
    s.close()


def test_session_submit_many_stops_at_cap_and_bad_request():
    rng = np.random.default_rng(30)
    links = make_links(rng, 2)
    s = F.Session(F.Plan(mu_shift=MU), 2, 64 * 1024, 1)
    for l, t in enumerate(links):
        s.set_link(l, t)
    x = torch.from_numpy(rng.integers(-16, 16, (20000, 2, 2)).astype(np.int8)).cuda()
    o = [torch.zeros((F.chain_nsym(20000, links[l].shape[0]), 4), dtype=torch.int16, device="cuda")
         for l in (0, 1, 0)]
    reqs = F.Requests([0, 1, 0], [x, x, x], o)
    tk = s.submit_many(reqs)                          # 40 KB each under a 64 KB cap: one fits
    assert len(tk) == 1
    _drain(s, 1)
    tk2 = s.submit_many(reqs, start=1)
    assert len(tk2) == 1 and tk2[0] > tk[0]
    _drain(s, 1)
    bad = F.Requests([0, 5], [x, x], [o[0], o[1]])
    with pytest.raises(F.FntError) as e:
        s.submit_many(bad)
    assert e.value.status == F.FNT_ERR_NOT_FOUND
    assert s.pending() == 1                           # the valid prefix was admitted
    _drain(s, 1)
    bad.rec["reserved"][0] = 1
    with pytest.raises(F.FntError) as e:
        s.submit_many(bad)
    assert e.value.status == F.FNT_ERR_INVALID and s.pending() == 0
    assert s.submit_many(reqs, start=3) == []
    s.close()


@pytest.mark.parametrize("variant", ["tensor_gradient", "period3", "segmented_tensor_n64", "cdc_both_items"])
def test_session_plan_variants_match_sequential_oracle(orc, variant):
    """The session runs whatever the plan selects (gradient on the tensor cores,
    an update period, N = 64 segments, two-polarisation CDC items): each link's
    frames, chained on the device, equal sequential oracle processing."""
    rng = np.random.default_rng(31)
    links = make_links(rng, 3)
    frames = make_frames(rng, 3, 4, lo=2000, hi=9000)
    kw, okw = {}, {}
    if variant == "period3":
        kw, okw = dict(aeq_update_period=3), dict(period=3)
    elif variant == "segmented_tensor_n64":
        kw = dict(n_aeq=64, alpha_aeq=4080, aeq_segment=432, aeq_warmup=0)
        okw = dict(n_aeq=64, alpha_aeq=4080, seg_len=432, warmup=0)
    plan = F.Plan(mu_shift=MU, **kw)
    if "tensor" in variant:
        plan.set_tensor_gradient(True)
    if variant == "cdc_both_items":
        plan.set_cdc_items(2)
    s = F.Session(plan, len(links), 1 << 30, 2)
    for l, taps in enumerate(links):
        s.set_link(l, taps)
    xs, outs = _device_frames(frames, links)
    assert len(s.submit_many(F.Requests([l for l, _ in frames], xs, outs))) == len(frames)
    assert all(c[2] == F.FNT_OK for c in _drain(s, len(frames)))
    prm = orc.ChainParams(mu_shift=MU, **okw)
    T = {l: orc.aeq_init_taps(16, prm.w0) for l in range(len(links))}
    for i, (link, x) in enumerate(frames):
        ref, T[link] = orc.chain(x, links[link], prm, T0=T[link])
        assert np.array_equal(outs[i].cpu().numpy(), ref), (variant, i)
    for l in range(len(links)):
        assert np.array_equal(s.get_link_state(l), T[l])
    s.close()


def test_session_tiny_and_empty_frames_in_a_burst(orc):
    """Zero-length, one-sample and short frames mixed with normal ones in one
    admitted burst, several per link: every completion is OK, every output and
    every link's final taps equal sequential oracle processing."""
    rng = np.random.default_rng(32)
    links = make_links(rng, 3)
    sizes = [0, 1, 2, 3, 17, 33, 4000, 0, 1, 5000, 2, 64, 0]
    frames = [(i % 3, rng.integers(-16, 16, (n, 2, 2)).astype(np.int8)) for i, n in enumerate(sizes)]
    ref, Tref = oracle_sequential(orc, links, frames)
    s = F.Session(F.Plan(mu_shift=MU), len(links), 1 << 28, 2)
    for l, taps in enumerate(links):
        s.set_link(l, taps)
    xs, outs = [], []
    for link, x in frames:
        nsym = F.chain_nsym(x.shape[0], links[link].shape[0])
        xs.append(torch.from_numpy(x).cuda() if x.shape[0] else torch.zeros((0, 2, 2), dtype=torch.int8, device="cuda"))
        outs.append(torch.full((max(nsym, 1), 4), 0x1111, dtype=torch.int16, device="cuda"))
    torch.cuda.synchronize()
    tk = s.submit_many(F.Requests([l for l, _ in frames], xs, outs))
    assert len(tk) == len(frames)
    done = _drain(s, len(frames))
    assert all(c[2] == F.FNT_OK for c in done)
    nsyms = {c[0]: c[3] for c in done}
    for i, (link, x) in enumerate(frames):
        nsym = ref[i].shape[0]
        assert nsyms[tk[i]] == nsym, i
        assert np.array_equal(outs[i].cpu().numpy()[:nsym], ref[i]), i
    for l in range(len(links)):
        assert np.array_equal(s.get_link_state(l), Tref[l])
    s.close()


def test_session_cancel_a_queued_request_and_stats(orc):
    """One main lane and four chain lanes: eight frames of one link admitted
    together launch five waves at once and queue three.  A queued one can be
    cancelled (it completes as FNT_ERR_CANCELLED and the link's other frames
    equal the oracle run without it); a launched one cannot.  The session's
    counters account for all of it."""
    rng = np.random.default_rng(33)
    links = make_links(rng, 1)
    frames = [(0, rng.integers(-16, 16, (6000, 2, 2)).astype(np.int8)) for _ in range(8)]
    s = F.Session(F.Plan(mu_shift=MU), 1, 1 << 28, 1)
    s.set_link(0, links[0])
    xs, outs = _device_frames(frames, links)
    tk = s.submit_many(F.Requests([0] * 8, xs, outs))
    st = s.stats()
    assert (st["admitted"], st["waves"], st["chained_waves"], st["queued"], st["in_flight"]) == (8, 5, 4, 3, 5)
    assert not s.cancel(tk[0])                 # launched: runs to completion
    assert s.cancel(tk[6])                     # queued
    assert not s.cancel(tk[6])                 # already cancelled
    done = {c[0]: c[2] for c in _drain(s, 8)}
    assert done[tk[6]] == F.FNT_ERR_CANCELLED
    assert all(done[t] == F.FNT_OK for i, t in enumerate(tk) if i != 6)
    kept = [i for i in range(8) if i != 6]
    ref, Tref = oracle_sequential(orc, links, [frames[i] for i in kept])
    for j, i in enumerate(kept):
        assert np.array_equal(outs[i].cpu().numpy(), ref[j]), i
    assert np.array_equal(s.get_link_state(0), Tref[0])
    st = s.stats()
    assert (st["completed"], st["cancelled"], st["failed"], st["queued"], st["in_flight"]) == (7, 1, 0, 0, 0)
    assert st["arena_used"] == 0 and st["arena_peak"] > 0
    assert (st["wave_frames"], st["max_wave"]) == (7, 1)
    s.close()
