// session.cu -- serving: a continuous-batching request loop over many links.
//
// Each link has fixed CD taps and an AEQ tap state that lives in device memory
// and carries across the link's frames.  Requests are admitted while the
// session's device arena (capped at mem_cap bytes) can hold their buffers:
// intermediate CDC->AEQ symbols (and, for segmented frames, a copy of the link's
// taps).  Inputs and outputs stay where the caller put them: device memory, or
// page-locked host memory that the kernels read and write directly.
//
// A scheduler packs admitted frames into waves, at most one frame per link, and
// runs the CDC and AEQ kernels of a whole wave on a lane (a stream running one
// wave at a time), recording an event after it.  The oldest frame of every link
// with nothing on the device goes into a wave on one of n_streams main lanes.
// The next frame of a link whose latest frame is still on the device goes into a
// chained wave with the next frames of every other link whose latest frame is in
// that same wave; a chained wave runs on one of kChainLanes * n_streams chain
// lanes, whose stream first waits on the event of that one wave.  A link's frames
// thus run in submission order and its tap state is read and written by one chain
// at a time; the host keeps the device fed without waiting for completions; and
// no frame waits behind an unrelated link's dependency or holds a main lane while
// it waits.  With AEQ segments in the plan, a long frame's segments start from
// the link's taps as the frame began and run in parallel; the last one writes the
// link's taps.  Completion is observed on the host by querying each wave's event.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fnt.h"
#include "host.h"
#include "internal.h"

namespace fnt {
namespace {

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// First-fit allocator over [0, cap) with coalescing of free ranges.
class Arena {
   public:
    explicit Arena(size_t cap) : cap_(cap) {
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t bytes, size_t &off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                const size_t next = it->first + bytes;
                free_.erase(it);
                if (rest) free_[next] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    size_t used() const { return used_; }
    void release(size_t off, size_t bytes) {
        if (!bytes) return;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
   private:
    size_t cap_;
    size_t used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    uint64_t ticket = 0;
    int link = 0;
    const int8_t *in = nullptr;   // device-accessible input (device memory, or the device
    void *out = nullptr;          // mapping of page-locked host memory) and output
    int64_t n = 0;
    int64_t n_sym = 0;
    size_t off = 0, bytes = 0;    // arena reservation
    size_t off_scratch = 0, off_init = 0;
    uint64_t prev_wave = 0;       // the link's latest in-flight frame before this one:
    int prev_wi = -1;             // id and pool index of its wave
    double submit_us = 0, start_us = 0;
};

struct LinkState {
    bool configured = false;
    int L = 0;
    int8_t taps[64] = {0};
    int shift = 0, phase = 0, S = 0;
    int inflight = 0;            // frames of this link launched and not yet completed
    uint64_t last_wave = 0;      // id and pool index of the wave holding its latest
    int last_wi = -1;            // in-flight frame (-1: nothing on the device)
    std::deque<Request> fifo;    // admitted, not yet launched
};

// One wave: its requests, device work tables (and their page-locked staging)
// and the event recorded after its kernels.
struct Wave {
    uint64_t id = 0;
    cudaEvent_t done = nullptr;
    char *d_tables = nullptr;
    size_t d_cap = 0;
    char *h_tables = nullptr;
    size_t h_cap = 0;
    std::vector<Request> reqs;
};

// A stream running at most one wave (index into the wave pool) at a time.
struct Lane {
    cudaStream_t stream = nullptr;
    int wave = -1;
};

constexpr int kChainLanes = 4;   // chain lanes per main lane
constexpr size_t kInitialTables = 64 << 10;   // a wave's first table allocation

}  // namespace
}  // namespace fnt

using namespace fnt;

struct fnt_session {
    const fnt_plan *plan = nullptr;
    int n_links = 0;
    size_t cap = 0;
    char *arena_mem = nullptr;
    Arena arena{0};
    int32_t *d_state = nullptr;           // [n_links][16][K]
    std::vector<LinkState> links;
    int n_main = 0;
    std::vector<Lane> lanes;              // n_main main lanes, then the chain lanes
    std::vector<Wave> waves;              // one per lane
    std::vector<int> free_waves;
    uint64_t next_wave = 1;
    std::vector<char *> retired;          // outgrown table staging, freed at destroy
    fnt_session_stats stats{};            // counters (queued / in_flight filled on read)
    std::deque<fnt_completion> done;
    uint64_t next_ticket = 1;
    int admitted = 0;                     // admitted and not yet returned by poll
    int inject_failures = 0;              // host-side fault injection (tests)
    std::mutex mu;
};

namespace fnt {
namespace {

constexpr int kMaxWave = 1024;

// One launch copies the taps of every segmented frame of a wave (link state ->
// the frame's copy), instead of one API copy per frame.
struct StateCopy {
    const int32_t *src;
    int32_t *dst;
};

__global__ void copy_states(const StateCopy *__restrict__ cp, int n) {
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        for (int t = threadIdx.x; t < 16 * kAeqK; t += blockDim.x) cp[i].dst[t] = cp[i].src[t];
}

bool segmented(const fnt_plan *p, int64_t n_sym) { return p->d.aeq_segment > 0 && n_sym > p->d.aeq_segment; }

size_t request_bytes(const fnt_plan *p, const Request &r) {
    size_t b = up256((size_t)r.n_sym * 4);                 // AEQ input symbols
    if (segmented(p, r.n_sym)) b += up256(kStateBytes);   // the link's taps as the frame began
    return b;
}

// Makes room for `bytes` of tables in a wave object, without a device-wide
// synchronisation (which cudaFree would imply, stalling every wave in flight):
// device tables come from the plan's stream-ordered pool on the stream about to
// use them, and an outgrown page-locked staging buffer is kept until the session
// is destroyed.  The wave object is free, so nothing in flight uses either.
fnt_status grow(fnt_session *ss, Wave &s, size_t bytes, cudaStream_t stream) {
    if (bytes <= s.d_cap) return FNT_OK;
    const size_t cap = std::max({bytes, s.d_cap * 2, kInitialTables});
    if (s.d_tables) cudaFreeAsync(s.d_tables, stream);
    if (s.h_tables) ss->retired.push_back(s.h_tables);
    s.d_tables = nullptr;
    s.h_tables = nullptr;
    s.d_cap = s.h_cap = 0;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&s.d_tables, cap, ss->plan->pool, stream);
    if (e != cudaSuccess) return cuda_fail(e, "session: table memory");
    e = cudaMallocHost(&s.h_tables, cap);
    if (e != cudaSuccess) return cuda_fail(e, "session: table staging");
    s.d_cap = s.h_cap = cap;
    return FNT_OK;
}

// Builds the wave's tables in its staging memory and enqueues on `stream`: a wait
// for `dep` (if not null), the table upload, the state copies, the kernels and
// the wave's event.
fnt_status launch_wave(fnt_session *ss, cudaStream_t stream, Wave &wave, cudaEvent_t dep) {
    if (ss->inject_failures > 0) {
        --ss->inject_failures;
        return fail(FNT_ERR_CUDA, "session: injected wave failure");
    }
    Work w;
    w.op = FNT_OP_CHAIN;
    const int nf = (int)wave.reqs.size();
    w.frames.resize(nf);
    for (int i = 0; i < nf; ++i) {
        const Request &r = wave.reqs[i];
        const LinkState &lk = ss->links[r.link];
        DevFrame &df = w.frames[i];
        memset(&df, 0, sizeof df);
        df.in = r.in;
        df.out = r.out;
        df.aeq_in = (int8_t *)(ss->arena_mem + r.off_scratch);
        df.state = ss->d_state + (size_t)r.link * 16 * kAeqK;
        df.n = r.n;
        df.n_sym = r.n_sym;
        df.n_pol = 2;
        df.L = lk.L;
        df.S = lk.S;
        df.shift = lk.shift;
        df.phase = lk.phase;
        memcpy(df.taps, lk.taps, sizeof df.taps);
        const int64_t nblk = (r.n + lk.S - 1) / lk.S;
        for (int64_t b = 0; b < nblk; b += kBlocksPerItem)
            for (int pol = 0; pol < 2; ++pol)
                w.items.push_back(make_int4(i, (int)b, (int)std::min<int64_t>(kBlocksPerItem, nblk - b), pol));
        if (r.n_sym > 0 && !segmented(ss->plan, r.n_sym)) {
            AeqChain c{};
            c.frame = i;
            c.write_state = 1;
            c.begin = 0;
            c.keep = 0;
            c.end = r.n_sym;
            c.init = df.state;
            c.init_copy = -1;
            w.chains.push_back(c);
        } else if (r.n_sym > 0) {
            // segments start from the link's taps as the frame began (copied below);
            // the last one writes the link's taps
            const int64_t seg = ss->plan->d.aeq_segment;
            for (int64_t k = 0; k < r.n_sym; k += seg) {
                AeqChain c{};
                c.frame = i;
                c.keep = k;
                c.end = std::min(r.n_sym, k + seg);
                c.begin = std::max<int64_t>(0, k - ss->plan->d.aeq_warmup);
                c.lo = std::max<int64_t>(0, c.begin - kAeqK);   // the stream's preceding symbols
                c.write_state = c.end == r.n_sym;
                c.init = (const int32_t *)(ss->arena_mem + r.off_init);
                c.init_copy = -1;
                w.chains.push_back(c);
            }
        }
    }
    std::stable_sort(w.chains.begin(), w.chains.end(),
                     [](const AeqChain &a, const AeqChain &b) { return a.end > b.end; });
    w.item_cut = {0, (int)w.items.size()};
    w.chain_cut = {0, (int)w.chains.size()};
    layout(w);
    std::vector<StateCopy> copies;
    for (const Request &r : wave.reqs)
        if (segmented(ss->plan, r.n_sym))
            copies.push_back({ss->d_state + (size_t)r.link * 16 * kAeqK, (int32_t *)(ss->arena_mem + r.off_init)});
    const size_t off_copies = w.total;
    const size_t bytes = off_copies + copies.size() * sizeof(StateCopy);
    fnt_status st = grow(ss, wave, bytes, stream);
    if (st != FNT_OK) return st;
    point_spectra(w, wave.d_tables);              // after grow: the tables may have moved
    memcpy(wave.h_tables + w.off_frames, w.frames.data(), w.frames.size() * sizeof(DevFrame));
    if (!w.items.empty()) memcpy(wave.h_tables + w.off_items, w.items.data(), w.items.size() * sizeof(int4));
    if (!w.chains.empty())
        memcpy(wave.h_tables + w.off_chains, w.chains.data(), w.chains.size() * sizeof(AeqChain));
    if (!copies.empty()) memcpy(wave.h_tables + off_copies, copies.data(), copies.size() * sizeof(StateCopy));
    cudaError_t e = dep ? cudaStreamWaitEvent(stream, dep, 0) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(e, "session: wave dependency");
    e = cudaMemcpyAsync(wave.d_tables, wave.h_tables, bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "session: table upload");
    if (!copies.empty()) {
        copy_states<<<std::min<int>((int)copies.size(), 1024), 256, 0, stream>>>(
            (const StateCopy *)(wave.d_tables + off_copies), (int)copies.size());
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "session: state copy launch");
    }
    st = launch_work(ss->plan, w, wave.d_tables, stream);
    if (st != FNT_OK) return st;
    e = cudaEventRecord(wave.done, stream);
    if (e != cudaSuccess) return cuda_fail(e, "session: event record");
    return FNT_OK;
}

// Returns a finished (or never launched) wave's requests as completions and the
// wave to the pool.  A link whose latest in-flight frame was in this wave has
// none left on the device; when the launch failed, its previous in-flight frame
// (if any) is its latest again.
void complete(fnt_session *ss, int wi, int status, double t, bool launch_failed) {
    Wave &wave = ss->waves[wi];
    for (const Request &r : wave.reqs) {
        ss->arena.release(r.off, r.bytes);
        LinkState &lk = ss->links[r.link];
        --lk.inflight;
        if (lk.last_wave == wave.id) {
            lk.last_wave = launch_failed ? r.prev_wave : 0;
            lk.last_wi = launch_failed ? r.prev_wi : -1;
        }
        fnt_completion c{};
        c.ticket = r.ticket;
        c.link = r.link;
        c.status = status;
        c.n_sym = status == FNT_OK ? r.n_sym : 0;
        c.submit_us = r.submit_us;
        c.start_us = r.start_us;
        c.done_us = t;
        ss->done.push_back(c);
        ++(status == FNT_OK ? ss->stats.completed : ss->stats.failed);
    }
    wave.reqs.clear();
    ss->free_waves.push_back(wi);
}

// Launches one wave on lane `li` holding the oldest frame of each link in
// `ready`; its stream first waits for `dep` when that is not null.
void form_wave(fnt_session *ss, int li, cudaEvent_t dep, std::vector<std::pair<double, int>> &ready) {
    std::sort(ready.begin(), ready.end());
    if ((int)ready.size() > kMaxWave) ready.resize(kMaxWave);
    Lane &lane = ss->lanes[li];
    const int wi = ss->free_waves.back();
    ss->free_waves.pop_back();
    Wave &wave = ss->waves[wi];
    wave.id = ss->next_wave++;
    const double t = now_us();
    for (auto &pr : ready) {
        LinkState &lk = ss->links[pr.second];
        Request r = lk.fifo.front();
        lk.fifo.pop_front();
        r.prev_wave = lk.last_wave;
        r.prev_wi = lk.last_wi;
        lk.last_wave = wave.id;
        lk.last_wi = wi;
        ++lk.inflight;
        r.start_us = t;
        wave.reqs.push_back(r);
    }
    lane.wave = wi;
    fnt_status st;
    {
        Range trace("fnt session wave");
        st = launch_wave(ss, lane.stream, wave, dep);
    }
    if (st == FNT_OK) {
        ++ss->stats.waves;
        ss->stats.chained_waves += dep != nullptr;
        ss->stats.wave_frames += wave.reqs.size();
        ss->stats.max_wave = std::max<uint64_t>(ss->stats.max_wave, wave.reqs.size());
    } else {
        // nothing of a failed wave is trusted: its requests complete with the error
        cudaStreamSynchronize(lane.stream);
        lane.wave = -1;
        complete(ss, wi, st, now_us(), true);
    }
}

// Forms and launches waves while frames are admitted and lanes are free: frames
// of links with nothing on the device on free main lanes; then chained waves,
// the group waiting on the wave that holds the oldest waiting frame first.
void schedule(fnt_session *ss) {
    std::vector<std::pair<double, int>> ready;
    const int n_lanes = (int)ss->lanes.size();
    for (int li = 0; li < ss->n_main; ++li) {
        if (ss->lanes[li].wave >= 0) continue;
        ready.clear();
        for (int l = 0; l < ss->n_links; ++l) {
            const LinkState &lk = ss->links[l];
            if (lk.last_wi < 0 && !lk.fifo.empty()) ready.push_back({lk.fifo.front().submit_us, l});
        }
        if (ready.empty()) break;
        form_wave(ss, li, nullptr, ready);
    }
    for (int li = ss->n_main; li < n_lanes; ++li) {
        if (ss->lanes[li].wave >= 0) continue;
        int dep = -1;
        double oldest = 0;
        for (int l = 0; l < ss->n_links; ++l) {
            const LinkState &lk = ss->links[l];
            if (lk.last_wi >= 0 && !lk.fifo.empty() && (dep < 0 || lk.fifo.front().submit_us < oldest)) {
                dep = lk.last_wi;
                oldest = lk.fifo.front().submit_us;
            }
        }
        if (dep < 0) break;
        ready.clear();
        for (int l = 0; l < ss->n_links; ++l) {
            const LinkState &lk = ss->links[l];
            if (lk.last_wi == dep && !lk.fifo.empty()) ready.push_back({lk.fifo.front().submit_us, l});
        }
        form_wave(ss, li, ss->waves[dep].done, ready);
    }
}

void reap(fnt_session *ss) {
    for (Lane &lane : ss->lanes) {
        if (lane.wave < 0) continue;
        cudaError_t e = cudaEventQuery(ss->waves[lane.wave].done);
        if (e == cudaErrorNotReady) continue;
        const int wi = lane.wave;
        lane.wave = -1;
        complete(ss, wi, e == cudaSuccess ? FNT_OK : FNT_ERR_CUDA, now_us(), false);
    }
}

// Validates and admits one request into its link's queue (caller holds the lock).
fnt_status admit(fnt_session *ss, int32_t link, const void *in, int64_t n, void *out, uint64_t *ticket) {
    if (link < 0 || link >= ss->n_links) return fail(FNT_ERR_NOT_FOUND, "no link %d", link);
    LinkState &lk = ss->links[link];
    if (!lk.configured) return fail(FNT_ERR_INVALID, "link %d has no taps", link);
    if (n < 0 || (n > 0 && (!in || !out))) return fail(FNT_ERR_INVALID, "bad frame");
    Request r;
    r.link = link;
    r.in = (const int8_t *)in;
    r.out = out;
    r.n = n;
    r.n_sym = chain_nsym(n, lk.phase);
    if (n > 0) {
        void *din = device_view(in), *dout = device_view(out);
        if (!din || !dout)
            return fail(FNT_ERR_INVALID, "submit: in/out must be device memory or page-locked host memory");
        if (((uintptr_t)din % 4) || ((uintptr_t)dout % 4)) return fail(FNT_ERR_INVALID, "submit: 4-byte alignment");
        r.in = (const int8_t *)din;
        r.out = dout;
    }
    r.bytes = std::max<size_t>(256, request_bytes(ss->plan, r));
    if (r.bytes > ss->cap) return fail(FNT_ERR_BOUND, "submit: frame needs %zu bytes > cap %zu", r.bytes, ss->cap);
    if (!ss->arena.alloc(r.bytes, r.off)) return fail(FNT_ERR_BUSY, "submit: memory cap reached");
    r.off_scratch = r.off;
    r.off_init = r.off + up256((size_t)r.n_sym * 4);
    r.ticket = ss->next_ticket++;
    r.submit_us = now_us();
    lk.fifo.push_back(r);
    ++ss->admitted;
    ++ss->stats.admitted;
    ss->stats.arena_peak = std::max<uint64_t>(ss->stats.arena_peak, ss->arena.used());
    *ticket = r.ticket;
    return FNT_OK;
}

}  // namespace
}  // namespace fnt

extern "C" fnt_status fnt_session_create(const fnt_plan *plan, int32_t n_links, size_t mem_cap_bytes,
                                         int32_t n_streams, fnt_session **out) {
    if (!plan || !out) return fail(FNT_ERR_INVALID, "null argument");
    *out = nullptr;
    if (n_links < 1 || n_streams < 1 || n_streams > 64 || mem_cap_bytes < 4096)
        return fail(FNT_ERR_INVALID, "session: need n_links >= 1, 1 <= n_streams <= 64, mem_cap >= 4 KiB");
    fnt_status dst = check_device(plan);
    if (dst != FNT_OK) return dst;
    fnt_session *ss = new (std::nothrow) fnt_session();
    if (!ss) return fail(FNT_ERR_NOMEM, "host memory");
    ss->plan = plan;
    ss->n_links = n_links;
    ss->cap = mem_cap_bytes;
    ss->arena = Arena(mem_cap_bytes);
    ss->links.resize(n_links);
    cudaError_t e = cudaMalloc(&ss->arena_mem, mem_cap_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ss->d_state, (size_t)n_links * 16 * kAeqK * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaFree(ss->arena_mem);
        delete ss;
        return e == cudaErrorMemoryAllocation ? fail(FNT_ERR_NOMEM, "session: device memory")
                                              : cuda_fail(e, "session: cudaMalloc");
    }
    std::vector<int32_t> init((size_t)n_links * 16 * kAeqK);
    for (int l = 0; l < n_links; ++l) memcpy(&init[(size_t)l * 16 * kAeqK], plan->h_init, sizeof plan->h_init);
    cudaMemcpy(ss->d_state, init.data(), init.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    ss->n_main = n_streams;
    ss->lanes.resize((size_t)n_streams * (1 + kChainLanes));
    for (Lane &l : ss->lanes) cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking);
    ss->waves.resize(ss->lanes.size());
    for (int i = (int)ss->waves.size() - 1; i >= 0; --i) {
        cudaEventCreateWithFlags(&ss->waves[i].done, cudaEventDisableTiming);
        ss->free_waves.push_back(i);
    }
    *out = ss;
    return FNT_OK;
}

extern "C" fnt_status fnt_session_set_link(fnt_session *ss, int32_t link, const int8_t *taps, int32_t L) {
    if (!ss) return fail(FNT_ERR_INVALID, "null session");
    std::lock_guard<std::mutex> g(ss->mu);
    if (link < 0 || link >= ss->n_links) return fail(FNT_ERR_NOT_FOUND, "no link %d", link);
    LinkState &lk = ss->links[link];
    if (lk.inflight || !lk.fifo.empty()) return fail(FNT_ERR_BUSY, "link %d has requests in the session", link);
    if (!taps || L < 1) return fail(FNT_ERR_INVALID, "link %d: no taps", link);
    if (L > kMaxCdTaps) return fail(FNT_ERR_BOUND, "link %d: %d taps > %d (constraint (5))", link, L, kMaxCdTaps);
    for (int k = 0; k < 2 * L; ++k)
        if (taps[k] < -32 || taps[k] > 31) return fail(FNT_ERR_INVALID, "link %d: tap outside 6 bits", link);
    const int S = ss->plan->d.cdc_step ? ss->plan->d.cdc_step : kCdcN - L + 1;
    if (S < 32 || S > kCdcN - L + 1) return fail(FNT_ERR_BOUND, "link %d: step %d with %d taps", link, S, L);
    memset(lk.taps, 0, sizeof lk.taps);
    memcpy(lk.taps, taps, 2 * L);
    lk.L = L;
    lk.S = S;
    lk.shift = cdc_shift_of(taps, L);
    lk.phase = decim_phase_of(L);
    lk.configured = true;
    cudaError_t e = cudaMemcpy(ss->d_state + (size_t)link * 16 * kAeqK, ss->plan->h_init, sizeof ss->plan->h_init,
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "session: state reset");
    return FNT_OK;
}

extern "C" fnt_status fnt_session_submit(fnt_session *ss, int32_t link, const void *in, int64_t n, void *out,
                                         uint64_t *ticket) {
    if (!ss || !ticket) return fail(FNT_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> g(ss->mu);
    fnt_status st = admit(ss, link, in, n, out, ticket);
    if (st == FNT_OK) schedule(ss);
    return st;
}

extern "C" fnt_status fnt_session_submit_many(fnt_session *ss, const fnt_request *reqs, int32_t n_reqs,
                                              uint64_t *tickets, int32_t *n_admitted) {
    if (!ss || !n_admitted || n_reqs < 0 || (n_reqs > 0 && (!reqs || !tickets)))
        return fail(FNT_ERR_INVALID, "bad argument");
    *n_admitted = 0;
    std::lock_guard<std::mutex> g(ss->mu);
    fnt_status st = FNT_OK;
    for (int32_t i = 0; i < n_reqs && st == FNT_OK; ++i) {
        const fnt_request &q = reqs[i];
        st = q.reserved ? fail(FNT_ERR_INVALID, "request %d: reserved field not 0", i)
                        : admit(ss, q.link, q.in, q.n, q.out, &tickets[i]);
        if (st == FNT_OK) ++*n_admitted;
    }
    if (*n_admitted > 0) schedule(ss);
    return st;
}

extern "C" fnt_status fnt_session_cancel(fnt_session *ss, uint64_t ticket) {
    if (!ss) return fail(FNT_ERR_INVALID, "null session");
    std::lock_guard<std::mutex> g(ss->mu);
    for (LinkState &lk : ss->links) {
        for (auto it = lk.fifo.begin(); it != lk.fifo.end(); ++it) {
            if (it->ticket != ticket) continue;
            ss->arena.release(it->off, it->bytes);
            fnt_completion c{};
            c.ticket = it->ticket;
            c.link = it->link;
            c.status = FNT_ERR_CANCELLED;
            c.submit_us = it->submit_us;
            c.done_us = now_us();
            ss->done.push_back(c);
            ++ss->stats.cancelled;
            lk.fifo.erase(it);
            return FNT_OK;
        }
    }
    return fail(FNT_ERR_NOT_FOUND, "cancel: ticket %llu is not waiting for launch", (unsigned long long)ticket);
}

extern "C" fnt_status fnt_session_get_stats(fnt_session *ss, fnt_session_stats *out) {
    if (!ss || !out) return fail(FNT_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> g(ss->mu);
    *out = ss->stats;
    out->arena_used = ss->arena.used();
    out->queued = 0;
    out->in_flight = 0;
    for (const LinkState &lk : ss->links) {
        out->queued += (int32_t)lk.fifo.size();
        out->in_flight += lk.inflight;
    }
    return FNT_OK;
}

extern "C" fnt_status fnt_session_poll(fnt_session *ss, int32_t timeout_us, fnt_completion *done, int32_t max_done,
                                       int32_t *n_done) {
    if (!ss || !n_done || max_done < 0 || (max_done > 0 && !done)) return fail(FNT_ERR_INVALID, "bad argument");
    *n_done = 0;
    const double t_end = now_us() + std::max(0, timeout_us);
    for (;;) {
        {
            std::lock_guard<std::mutex> g(ss->mu);
            reap(ss);
            schedule(ss);
            while (*n_done < max_done && !ss->done.empty()) {
                done[(*n_done)++] = ss->done.front();
                ss->done.pop_front();
                --ss->admitted;
            }
            if (*n_done > 0) return FNT_OK;
            if (max_done == 0) return FNT_OK;
        }
        if (now_us() >= t_end) return fail(FNT_ERR_TIMEOUT, "poll: nothing completed within %d us", timeout_us);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" int32_t fnt_session_pending(const fnt_session *ss) { return ss ? ss->admitted : 0; }

static fnt_status link_idle(fnt_session *ss, int32_t link) {
    if (link < 0 || link >= ss->n_links) return fail(FNT_ERR_NOT_FOUND, "no link %d", link);
    const LinkState &lk = ss->links[link];
    if (lk.inflight || !lk.fifo.empty()) return fail(FNT_ERR_BUSY, "link %d has requests in the session", link);
    return FNT_OK;
}

extern "C" fnt_status fnt_session_get_link_state(fnt_session *ss, int32_t link, int32_t *state) {
    if (!ss || !state) return fail(FNT_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> g(ss->mu);
    fnt_status st = link_idle(ss, link);
    if (st != FNT_OK) return st;
    cudaError_t e = cudaMemcpy(state, ss->d_state + (size_t)link * 16 * kAeqK, 16 * kAeqK * sizeof(int32_t),
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? FNT_OK : cuda_fail(e, "session: get state");
}

extern "C" fnt_status fnt_session_set_link_state(fnt_session *ss, int32_t link, const int32_t *state) {
    if (!ss || !state) return fail(FNT_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> g(ss->mu);
    fnt_status st = link_idle(ss, link);
    if (st != FNT_OK) return st;
    cudaError_t e = cudaMemcpy(ss->d_state + (size_t)link * 16 * kAeqK, state, 16 * kAeqK * sizeof(int32_t),
                               cudaMemcpyHostToDevice);
    return e == cudaSuccess ? FNT_OK : cuda_fail(e, "session: set state");
}

extern "C" fnt_status fnt_session_inject_failures(fnt_session *ss, int32_t n_waves) {
    if (!ss || n_waves < 0) return fail(FNT_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> g(ss->mu);
    ss->inject_failures = n_waves;
    return FNT_OK;
}

extern "C" fnt_status fnt_session_destroy(fnt_session *ss) {
    if (!ss) return FNT_OK;
    // drain: launch what is admitted, wait for every wave
    for (;;) {
        bool idle = true;
        {
            std::lock_guard<std::mutex> g(ss->mu);
            reap(ss);
            schedule(ss);
            for (const Lane &l : ss->lanes) idle = idle && l.wave < 0;
            for (const LinkState &lk : ss->links) idle = idle && lk.fifo.empty();
        }
        if (idle) break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (Lane &l : ss->lanes) {
        if (!l.stream) continue;
        cudaStreamSynchronize(l.stream);
        cudaStreamDestroy(l.stream);
    }
    for (Wave &w : ss->waves) {
        if (w.done) cudaEventDestroy(w.done);
        if (w.d_tables) cudaFree(w.d_tables);
        if (w.h_tables) cudaFreeHost(w.h_tables);
    }
    for (char *h : ss->retired) cudaFreeHost(h);
    cudaFree(ss->arena_mem);
    cudaFree(ss->d_state);
    delete ss;
    return FNT_OK;
}
