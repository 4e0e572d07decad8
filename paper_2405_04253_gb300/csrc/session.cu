// session.cu -- serving: a continuous-batching request loop over many links.
//
// Each link has fixed CD taps and an AEQ tap state that lives in device memory
// and carries across the link's frames.  Requests are admitted while the
// session's device arena (capped at mem_cap bytes) can hold their buffers:
// intermediate CDC->AEQ symbols (and, for segmented frames, a copy of the link's
// taps).  Inputs and outputs stay where the caller put them: device memory, or
// page-locked host memory that the kernels read and write directly.  A scheduler packs the oldest ready frame of each
// idle link into a wave, runs the CDC and AEQ kernels for the whole wave on one
// of n_streams streams, and records an event; up to n_streams waves run at
// once, so requests admitted while others are on the GPU overlap with them.  A
// link is idle while none of its frames is in flight, which keeps every link's
// frames in submission order (its tap state is read and written by one chain at
// a time).  With AEQ segments in the plan, a long frame's segments start from the
// link's taps as the frame began and run in parallel; the last one writes the
// link's taps.  Completion is observed on the host by querying the wave's event.
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
    double submit_us = 0, start_us = 0;
};

struct LinkState {
    bool configured = false;
    int L = 0;
    int8_t taps[64] = {0};
    int shift = 0, phase = 0, S = 0;
    bool busy = false;           // a frame of this link is in flight
    std::deque<Request> fifo;    // admitted, not yet launched
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    char *d_tables = nullptr;    // device work tables of the slot's wave
    size_t d_cap = 0;
    char *h_tables = nullptr;    // page-locked staging of the same
    size_t h_cap = 0;
    std::vector<Request> reqs;
    int status = FNT_OK;
};

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
    std::vector<Slot> slots;
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

fnt_status grow(Slot &s, size_t bytes) {
    if (bytes <= s.d_cap) return FNT_OK;
    size_t cap = std::max(bytes, s.d_cap * 2);
    if (s.d_tables) cudaFree(s.d_tables);
    if (s.h_tables) cudaFreeHost(s.h_tables);
    s.d_tables = nullptr;
    s.h_tables = nullptr;
    s.d_cap = s.h_cap = 0;
    cudaError_t e = cudaMalloc(&s.d_tables, cap);
    if (e != cudaSuccess) return cuda_fail(e, "session: table memory");
    e = cudaMallocHost(&s.h_tables, cap);
    if (e != cudaSuccess) return cuda_fail(e, "session: table staging");
    s.d_cap = s.h_cap = cap;
    return FNT_OK;
}

// Builds the wave's tables in the slot's staging memory and enqueues copies,
// kernels and result copies on the slot's stream.
fnt_status launch_wave(fnt_session *ss, Slot &slot) {
    if (ss->inject_failures > 0) {
        --ss->inject_failures;
        return fail(FNT_ERR_CUDA, "session: injected wave failure");
    }
    Work w;
    w.op = FNT_OP_CHAIN;
    const int nf = (int)slot.reqs.size();
    w.frames.resize(nf);
    for (int i = 0; i < nf; ++i) {
        const Request &r = slot.reqs[i];
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
    for (const Request &r : slot.reqs)
        if (segmented(ss->plan, r.n_sym))
            copies.push_back({ss->d_state + (size_t)r.link * 16 * kAeqK, (int32_t *)(ss->arena_mem + r.off_init)});
    const size_t off_copies = w.total;
    const size_t bytes = off_copies + copies.size() * sizeof(StateCopy);
    fnt_status st = grow(slot, bytes);
    if (st != FNT_OK) return st;
    point_spectra(w, slot.d_tables);              // after grow: the tables may have moved
    memcpy(slot.h_tables + w.off_frames, w.frames.data(), w.frames.size() * sizeof(DevFrame));
    if (!w.items.empty()) memcpy(slot.h_tables + w.off_items, w.items.data(), w.items.size() * sizeof(int4));
    if (!w.chains.empty())
        memcpy(slot.h_tables + w.off_chains, w.chains.data(), w.chains.size() * sizeof(AeqChain));
    if (!copies.empty()) memcpy(slot.h_tables + off_copies, copies.data(), copies.size() * sizeof(StateCopy));
    cudaError_t e = cudaMemcpyAsync(slot.d_tables, slot.h_tables, bytes, cudaMemcpyHostToDevice, slot.stream);
    if (e != cudaSuccess) return cuda_fail(e, "session: table upload");
    if (!copies.empty()) {
        copy_states<<<std::min<int>((int)copies.size(), 1024), 256, 0, slot.stream>>>(
            (const StateCopy *)(slot.d_tables + off_copies), (int)copies.size());
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "session: state copy launch");
    }
    st = launch_work(ss->plan, w, slot.d_tables, slot.stream);
    if (st != FNT_OK) return st;
    e = cudaEventRecord(slot.done, slot.stream);
    if (e != cudaSuccess) return cuda_fail(e, "session: event record");
    return FNT_OK;
}

void complete(fnt_session *ss, Slot &slot, int status, double t) {
    for (const Request &r : slot.reqs) {
        ss->arena.release(r.off, r.bytes);
        ss->links[r.link].busy = false;
        fnt_completion c{};
        c.ticket = r.ticket;
        c.link = r.link;
        c.status = status;
        c.n_sym = status == FNT_OK ? r.n_sym : 0;
        c.submit_us = r.submit_us;
        c.start_us = r.start_us;
        c.done_us = t;
        ss->done.push_back(c);
    }
    slot.reqs.clear();
    slot.busy = false;
}

// Forms and launches waves while a slot is free and a link has a ready frame.
void schedule(fnt_session *ss) {
    for (Slot &slot : ss->slots) {
        if (slot.busy) continue;
        std::vector<std::pair<double, int>> ready;
        for (int l = 0; l < ss->n_links; ++l) {
            LinkState &lk = ss->links[l];
            if (!lk.busy && !lk.fifo.empty()) ready.push_back({lk.fifo.front().submit_us, l});
        }
        if (ready.empty()) return;
        std::sort(ready.begin(), ready.end());
        if ((int)ready.size() > kMaxWave) ready.resize(kMaxWave);
        const double t = now_us();
        for (auto &pr : ready) {
            LinkState &lk = ss->links[pr.second];
            Request r = lk.fifo.front();
            lk.fifo.pop_front();
            lk.busy = true;
            r.start_us = t;
            slot.reqs.push_back(r);
        }
        slot.busy = true;
        fnt_status st = launch_wave(ss, slot);
        if (st != FNT_OK) {
            // nothing of a failed wave is trusted: its requests complete with the error
            cudaStreamSynchronize(slot.stream);
            complete(ss, slot, st, now_us());
        }
    }
}

void reap(fnt_session *ss) {
    for (Slot &slot : ss->slots) {
        if (!slot.busy) continue;
        cudaError_t e = cudaEventQuery(slot.done);
        if (e == cudaErrorNotReady) continue;
        complete(ss, slot, e == cudaSuccess ? FNT_OK : FNT_ERR_CUDA, now_us());
    }
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
    ss->slots.resize(n_streams);
    for (Slot &s : ss->slots) {
        cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    }
    *out = ss;
    return FNT_OK;
}

extern "C" fnt_status fnt_session_set_link(fnt_session *ss, int32_t link, const int8_t *taps, int32_t L) {
    if (!ss) return fail(FNT_ERR_INVALID, "null session");
    std::lock_guard<std::mutex> g(ss->mu);
    if (link < 0 || link >= ss->n_links) return fail(FNT_ERR_NOT_FOUND, "no link %d", link);
    LinkState &lk = ss->links[link];
    if (lk.busy || !lk.fifo.empty()) return fail(FNT_ERR_BUSY, "link %d has requests in the session", link);
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
    *ticket = r.ticket;
    schedule(ss);
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
    if (lk.busy || !lk.fifo.empty()) return fail(FNT_ERR_BUSY, "link %d has requests in the session", link);
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
            for (const Slot &s : ss->slots) idle = idle && !s.busy;
            for (const LinkState &lk : ss->links) idle = idle && lk.fifo.empty();
        }
        if (idle) break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (Slot &s : ss->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.d_tables) cudaFree(s.d_tables);
        if (s.h_tables) cudaFreeHost(s.h_tables);
    }
    cudaFree(ss->arena_mem);
    cudaFree(ss->d_state);
    delete ss;
    return FNT_OK;
}
