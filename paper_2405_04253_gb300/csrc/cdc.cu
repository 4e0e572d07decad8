// cdc.cu -- FNT-CDC kernel: overlap-save complex convolution through length-64
// Fermat number transforms over Z_65537 with radix sqrt(2) = 4080 (section
// "Proposed FNT-CDC&AEQ structure"; eqs. (1), (2), (5), (7), (8)).
//
// Work item = 32 consecutive overlap-save blocks of one polarisation of a frame,
// one warp; lane l owns block b0 + l entirely in registers:
//   u = x_re + 2^8 x_im, v = x_re - 2^8 x_im          (2^8 = sqrt(-1) mod F)
//   P = FNT(u) . H_u,   Q = FNT(v) . H_v                (H = FNT of the taps,
//                                                        times N^-1 2^-1)
//   z_re = IFNT(P + Q),  z_im = IFNT(-2^8 (P - Q))       (eqs. (7) and (8))
// By linearity FNT(u) = X + 2^8 Xh with X, Xh the transforms of the real and
// imaginary parts, so this is eqs. (7)/(8) with two forward transforms instead
// of four and the constants -2^15 = 2^-1 and -2^7 = 2^-9 folded into H.
//
// Memory path: each warp copies its 32 input windows (64 samples each, 16 B
// loads coalesced) into a [position][lane] shared-memory transpose (33-word
// rows: conflict-free for the column reads of the lanes and the row writes of
// the fill), and writes results back through the same buffers with coalesced
// 8-byte (CDC) or 4-byte (chain) stores.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "zf.cuh"

namespace fnt {

namespace {

constexpr int kN = kCdcN;
constexpr int64_t kAlpha = 4080;
constexpr int kRow = 33;                                 // padded smem row (words)
constexpr int kWarpWords = 2 * kN * kRow + 2 * kN + 4;   // win, o0, H_u, H_v, mbarrier
// N^-1 * 2^-1 folded into the tap spectra
constexpr int32_t kHScale = zcent(zinv(kN) * zinv(2) % kF);

__device__ __forceinline__ int32_t sx8(uint32_t w, int sh) { return (int32_t)(w << (24 - sh)) >> 24; }

__device__ __forceinline__ int32_t sat5(int32_t v) { return v < -16 ? -16 : (v > 15 ? 15 : v); }

// 4-byte asynchronous global -> shared copy; src_size 0 writes zeros.
__device__ __forceinline__ void cp_async4(uint32_t *smem, const uint32_t *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------- bulk-copy window fill ----
//
// A PDM work item of one polarisation covers 32 windows, one contiguous span of the input,
// [base, base + 31 S + 64) samples.  Where that span, widened to 16-byte
// boundaries, lies inside the frame (and the input is 16-byte aligned), the
// warp fetches it with one 1-D TMA bulk copy (cp.async.bulk) into its output
// buffer, which is free until the block's results are written, and transposes
// it into the padded window layout in shared memory.  Completion is an
// mbarrier whose wait is bounded: after about 5 ms it records
// kFaultCdcWindowWait in the device fault word, waits once more (bounded) for
// the copy still in flight, and the warp stops.

__device__ unsigned g_fnt_faults = 0;

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arms the barrier for `bytes` and, unless `issue` is false (test hook), starts
// the copy global -> shared.  dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar, bool issue) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst), b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // earlier generic accesses of dst first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
    if (issue)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
                     "l"(src), "r"(bytes), "r"(b)
                     : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with parity ph, for at most about limit_ns (and a bounded
// number of polls); false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned ph, uint64_t limit_ns) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 20); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(b), "r"(ph), "r"(1000u)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) break;
    }
    return false;
}

// Eqs. (7)/(8) on the two product spectra: P <- P + Q (z_re's spectrum, 2^-1
// N^-1 folded into H) and Q <- -2^8 (P - Q) (z_im's: 2^-9 = 2^-1 (-2^8)).
template <class A>
FNT_HD void cdc_combine(const A &ar, int32_t (&P)[kN], int32_t (&Q)[kN]) {
#pragma unroll
    for (int i = 0; i < kN; ++i) {
        const int32_t a = P[i] + Q[i];
        const int32_t b = P[i] - Q[i];
        P[i] = rho(a);
        Q[i] = ar.mulpow2(b, -256);
    }
}

// The spectral stage of a block: the pointwise products with the tap spectra
// (H_u, H_v at hs, hs + N) and eqs. (7)/(8).  make_q forms v and its transform
// in Q between the two products, which keeps P's product ahead of Q's
// transform (fewer live registers).  The kernel runs the stage with ZArith;
// the host runs the same code with a counting policy for the Tab. 1 counts.
template <class A, class MakeQ>
FNT_HD void cdc_spectral_stage(const A &ar, int32_t (&P)[kN], int32_t (&Q)[kN], const int32_t *hs, MakeQ make_q) {
    spectral_products(ar, P, hs);
    make_q(Q);
    spectral_products(ar, Q, hs + kN);
    cdc_combine(ar, P, Q);
}

// One block of one polarisation: window words w[j] = win[j][lane]; results
// (re, im) as int16 into o[j][lane] for all 64 window positions.  `o` may be
// `win` itself: every output depends on every input of the lane's column, so
// all reads precede all writes.  The two inverse transforms run as a two-trip
// loop so that their unrolled code exists once (instruction-cache footprint).
__device__ __forceinline__ void cdc_block(const uint32_t *win, uint32_t *o, const int32_t *hs, int lane, int sh) {
    int32_t P[kN], Q[kN];
#pragma unroll
    for (int j = 0; j < kN; ++j) {
        const uint32_t w = win[j * kRow + lane];
        P[j] = sx8(w, sh) + 256 * sx8(w, sh + 8);
    }
    fnt_fwd<kN, kAlpha, 13>(P);                      // |u| <= 16 + 256 * 16 < 2^13
    cdc_spectral_stage(ZArith{}, P, Q, hs, [&](int32_t (&q)[kN]) {
#pragma unroll
        for (int j = 0; j < kN; ++j) {
            const uint32_t w = win[j * kRow + lane];
            q[j] = sx8(w, sh) - 256 * sx8(w, sh + 8);
        }
        fnt_fwd<kN, kAlpha, 13>(q);
    });
    int16_t *o16 = (int16_t *)o;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        fnt_inv<kN, kAlpha, 17>(P);
        // |z| <= 31 * 1024 < 32767, so the centred residue is the value
#pragma unroll
        for (int j = 0; j < kN; ++j) o16[2 * (j * kRow + lane) + pass] = (int16_t)rhoc(P[j]);
        if (pass == 0) {
#pragma unroll
            for (int i = 0; i < kN; ++i) P[i] = Q[i];
        }
    }
}

// Tap spectra of each frame, once per frame: H_u[k] and H_v[k] (u = h_re +
// 2^8 h_im, v = h_re - 2^8 h_im) times N^-1 2^-1, entry i holding
// k = bitrev(i), as centred residues: thread t < 64 computes H_u at i = t,
// thread 64 + i computes H_v.  One CTA of 128 threads per frame.
__global__ void __launch_bounds__(2 * kN) cdc_spectra_kernel(const DevFrame *__restrict__ frames, int n_frames) {
    __shared__ int32_t s_pow[kN];
    if (threadIdx.x < kN) s_pow[threadIdx.x] = zcent(zpow(kAlpha, threadIdx.x));
    __syncthreads();
    const int i = threadIdx.x & (kN - 1);
    const int32_t sg = threadIdx.x < kN ? 256 : -256;
    const int k = (int)(__brev((unsigned)i) >> 26);
    for (int f = blockIdx.x; f < n_frames; f += gridDim.x) {
        const DevFrame &fr = frames[f];
        int32_t a = 0;
        for (int m = 0; m < fr.L; ++m) {
            const int32_t hr = fr.taps[2 * m], hi = fr.taps[2 * m + 1];
            a += rho((hr + sg * hi) * s_pow[(m * k) & (kN - 1)]);     // |a| < 31 * 98304 < 2^22
        }
        fr.hspec[threadIdx.x] = rhoc(rho(rhoc(a) * kHScale));
    }
}

// BOTH: items may cover both polarisations of a PDM frame (item.w = 2); such a
// warp runs the two blocks of each lane back to back from one window fill and
// one tap-spectrum set, and stores each symbol's 4-byte word at once.  That
// form needs more registers, so it runs 2 CTAs per SM instead of 3.
template <bool CHAIN, bool BOTH>
__global__ void __launch_bounds__(128, BOTH ? 2 : 3) cdc_kernel(const DevFrame *__restrict__ frames,
                                                     const int4 *__restrict__ items, int n_items) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint32_t *win = smem + warp * kWarpWords;     // [64][33] input words (both polarisations)
    uint32_t *o0 = win + kN * kRow;               // [64][33] results of the item's polarisation
    int32_t *hs = (int32_t *)(o0 + kN * kRow);    // H_u [64], H_v [64] in bit-reversed order
    uint64_t *bar = (uint64_t *)(hs + 2 * kN);    // the warp's window barrier (8-byte aligned)
    unsigned phase = 0;
    if (!BOTH && lane == 0) mbar_init(bar);
    __syncwarp();

    for (int it = blockIdx.x * wpb + warp; it < n_items; it += gridDim.x * wpb) {
        const int4 item = items[it];
        const DevFrame &fr = frames[item.x];
        const int64_t b0 = item.y;
        const int nb = item.z;
        const int pol = item.w;                       // polarisation this warp computes, 2 = both
        const int S = fr.S;
        const int npol = fr.n_pol;
        const int64_t n = fr.n;

        // the frame's tap spectra (cdc_spectra_kernel), 4 words per lane
#pragma unroll
        for (int h = 0; h < 4; ++h) hs[lane + 32 * h] = fr.hspec[lane + 32 * h];

        // Input windows: window l covers samples base + l*S + [0, 64).  All 64
        // loads of a lane are in flight at once: asynchronous 4-byte copies
        // straight into shared memory for PDM (zero-filled outside the frame),
        // register-staged 2-byte loads for one polarisation.
        const int64_t base = b0 * S - (kN - S);
        const int64_t a0 = base & ~(int64_t)3;                          // 16-byte boundaries
        const int64_t a1 = (base + (int64_t)(nb - 1) * S + kN + 3) & ~(int64_t)3;
        // (one-polarisation items only: with two-polarisation items, 2 CTAs per SM,
        // the bulk copy and transpose measured 8 % slower than the 4-byte copies)
        if (!BOTH && npol == 2 && nb == kBlocksPerItem && a0 >= 0 && a1 <= n && ((uintptr_t)fr.in & 15) == 0) {
            const uint32_t *src = (const uint32_t *)fr.in;
            if (lane == 0)
                bulk_load(o0, src + a0, (unsigned)((a1 - a0) * 4), bar, !(fr.flags & kFrameInjectTmaTimeout));
            // one decision for the warp: lanes whose own waits disagree at the limit
            // all take the fault path (the re-wait then returns at once)
            const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, phase, 5000000));
            phase ^= 1;
            if (!ok) {
                if (lane == 0) atomicOr(&g_fnt_faults, kFaultCdcWindowWait);
                mbar_wait(bar, phase ^ 1, 5000000);   // the copy that may still be in flight
                return;
            }
            const int off = (int)(base - a0);
#pragma unroll 8
            for (int l = 0; l < kBlocksPerItem; ++l) {
                win[lane * kRow + l] = o0[off + l * S + lane];
                win[(lane + 32) * kRow + l] = o0[off + l * S + lane + 32];
            }
        } else if (npol == 2) {
            const uint32_t *src = (const uint32_t *)fr.in;
#pragma unroll
            for (int l = 0; l < 32; ++l) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = lane + 32 * h;
                    const int64_t t = base + (int64_t)l * S + j;
                    const bool ok = l < nb && t >= 0 && t < n;
                    cp_async4(win + j * kRow + l, ok ? src + t : src, ok);
                }
            }
            cp_async_wait_all();
        } else {
            const uint16_t *src = (const uint16_t *)fr.in;
#pragma unroll 4
            for (int l0 = 0; l0 < 32; l0 += 8) {
                uint32_t v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int l = l0 + (q >> 1), j = lane + 32 * (q & 1);
                    const int64_t t = base + (int64_t)l * S + j;
                    v[q] = (l < nb && t >= 0 && t < n) ? (uint32_t)__ldg(src + t) : 0u;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) win[(lane + 32 * (q & 1)) * kRow + l0 + (q >> 1)] = v[q];
            }
        }
        __syncwarp();

        // item.w = 2: both polarisations from the same windows and tap spectra;
        // polarisation 1's results overwrite the lane's own window column
        const bool two = BOTH && pol == 2;
        if constexpr (BOTH) {
            const int p_first = two ? 0 : pol, p_end = two ? 2 : pol + 1;
#pragma unroll 1
            for (int pp = p_first; pp < p_end; ++pp) cdc_block(win, pp > p_first ? win : o0, hs, lane, 16 * pp);
        } else {
            cdc_block(win, o0, hs, lane, 16 * pol);
        }
        __syncwarp();

        if (!CHAIN) {
            int16_t *out = (int16_t *)fr.out;
            for (int l = 0; l < nb; ++l) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int jj = lane + 32 * h;
                    const int64_t t = (b0 + l) * S + jj;
                    if (jj < S && t < n) {
                        const int pos = (kN - S + jj) * kRow + l;
                        if (two)
                            *(uint2 *)(out + t * 4) = make_uint2(o0[pos], win[pos]);
                        else
                            *(uint32_t *)(out + (t * npol + pol) * 2) = o0[pos];
                    }
                }
            }
        } else {
            // requantise to 5 bits and keep times t = phase (mod 2)
            const int sft = fr.shift;
            const int32_t rnd = sft > 0 ? (1 << (sft - 1)) : 0;
            for (int l = 0; l < nb; ++l) {
                const int64_t t0 = (b0 + l) * S;
                const int jj = (int)((t0 - fr.phase) & 1) + 2 * lane;
                const int64_t t = t0 + jj;
                if (jj < S && t < n) {
                    const int pos = (kN - S + jj) * kRow + l;
                    const int64_t sym = (t - fr.phase) >> 1;
                    const uint32_t w0 = o0[pos];
                    const uint32_t q0 = (uint32_t)(sat5(((int32_t)(int16_t)(w0 & 0xFFFF) + rnd) >> sft) & 0xFF) |
                                        ((uint32_t)(sat5((((int32_t)w0 >> 16) + rnd) >> sft) & 0xFF) << 8);
                    if (two) {
                        // the symbol's whole 4-byte word (XI, XQ, YI, YQ)
                        const uint32_t w1 = win[pos];
                        const uint32_t q1 = (uint32_t)(sat5(((int32_t)(int16_t)(w1 & 0xFFFF) + rnd) >> sft) & 0xFF) |
                                            ((uint32_t)(sat5((((int32_t)w1 >> 16) + rnd) >> sft) & 0xFF) << 8);
                        ((uint32_t *)fr.aeq_in)[sym] = q0 | (q1 << 16);
                    } else {
                        // this polarisation's two bytes (I, Q) of the symbol's word
                        ((uint16_t *)fr.aeq_in)[2 * sym + pol] = (uint16_t)q0;
                    }
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------- small work ----
//
// When the work has too few blocks to give every SM a few warps at one block
// per lane (a single 65,536-sample frame is 1366 blocks: 43 warps), a block is
// split over 8 threads instead.  Each 64-point transform runs as a four-step
// 8 x 8 transform: with j = 8 j1 + j2 and k = k1 + 8 k2,
//   X[k1 + 8 k2] = sum_j2 beta^(j2 k2) alpha^(j2 k1) sum_j1 beta^(j1 k1) x[8 j1 + j2],
// beta = alpha^8, so thread j2 transforms its 8 samples (stride 8), applies the
// twiddles alpha^(j2 k1), and after a transpose through shared memory thread k1
// transforms over j2 and holds X[k1 + 8 k2].  Products with the tap spectra and
// eqs. (7)/(8) are local; each inverse runs the same four steps with
// alpha^-1, leaving z[n2 + 8 n1] in thread n2.  The work items are the same
// 32-block items: eight warps take an item, four blocks each.
constexpr int kSplitBlocksPerWarp = 4;
constexpr int kSplitWarpsPerItem = kBlocksPerItem / kSplitBlocksPerWarp;
constexpr int kSplitTP = 9;                                // transpose row pitch (words)
constexpr int kSplitWarpWords = kSplitBlocksPerWarp * 2 * 8 * kSplitTP;
constexpr int kSplitWarps = 2;                             // warps per CTA
constexpr int64_t kBeta = zpow(kAlpha, 8);                 // order 8

__device__ __forceinline__ int br3(int i) { return ((i & 1) << 2) | (i & 2) | ((i >> 2) & 1); }

__device__ __forceinline__ int32_t centred64(int64_t v) {
    v %= kF;
    if (v < 0) v += kF;
    return v > 32768 ? (int32_t)(v - kF) : (int32_t)v;
}

// Steps B and C of the four-step transform: twiddle the 8 values (register i of
// step A) by tw[i], write them to row br3(i) (ROW_BR) or row i, column t, of the
// block's 8 x 8 buffer, then read row t in bit-reversed (READ_BR) or natural
// column order for step D.
template <bool ROW_BR, bool READ_BR>
__device__ __forceinline__ void split_exchange(int32_t (&x)[8], const int32_t (&tw)[8], int32_t *T, int t) {
#pragma unroll
    for (int i = 0; i < 8; ++i) T[(ROW_BR ? br3(i) : i) * kSplitTP + t] = mulred(x[i], tw[i]);   // < 2^17
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = T[t * kSplitTP + (READ_BR ? br3(i) : i)];
    __syncwarp();
}

template <bool CHAIN>
__global__ void __launch_bounds__(32 * kSplitWarps) cdc_split_kernel(const DevFrame *__restrict__ frames,
                                                                    const int4 *__restrict__ items, int n_items) {
    __shared__ int32_t smem[kSplitWarps * kSplitWarpWords];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 3, t = lane & 7;                 // block of the warp, thread of the block
    int32_t *TU = smem + warp * kSplitWarpWords + q * 2 * 8 * kSplitTP, *TV = TU + 8 * kSplitTP;
    // twiddles alpha^(t br3(i)) (forward, step B) and alpha^(-n t) (inverse, step B)
    int32_t tw1[8], tw2[8];
    {
        int64_t a = 1, ai = 1;
        for (int i = 0; i < t; ++i) {
            a = a * kAlpha % kF;
            ai = ai * zinv(kAlpha) % kF;
        }
        int64_t pw[8], pwi = 1;
        pw[0] = 1;
#pragma unroll
        for (int i = 1; i < 8; ++i) pw[i] = pw[i - 1] * a % kF;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            tw1[i] = centred64(pw[br3(i)]);
            tw2[i] = centred64(pwi);
            pwi = pwi * ai % kF;
        }
    }
    const int wpg = gridDim.x * kSplitWarps;
    for (int w = blockIdx.x * kSplitWarps + warp; w < n_items * kSplitWarpsPerItem; w += wpg) {
        const int4 item = items[w / kSplitWarpsPerItem];
        const int lb = kSplitBlocksPerWarp * (w % kSplitWarpsPerItem) + q;   // block within the item
        const DevFrame &fr = frames[item.x];
        const int S = fr.S, npol = fr.n_pol;
        const int64_t n = fr.n;
        const bool active = lb < item.z;
        const int64_t b = (int64_t)item.y + lb;
        const int64_t base = b * S - (kN - S);
        // tap spectra in this thread's order: register i is frequency t + 8 br3(i),
        // stored by cdc_spectra_kernel at index bitrev_6(k)
        int32_t hu[8], hv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = t + 8 * br3(i);
            const int idx = (int)(__brev((unsigned)k) >> 26);
            hu[i] = fr.hspec[idx];
            hv[i] = fr.hspec[kN + idx];
        }
        const int p_first = item.w == 2 ? 0 : item.w, p_end = item.w == 2 ? 2 : item.w + 1;
        for (int pol = p_first; pol < p_end; ++pol) {
            int32_t U[8], V[8];
#pragma unroll
            for (int j1 = 0; j1 < 8; ++j1) {
                const int64_t sidx = base + 8 * j1 + t;
                int32_t re = 0, im = 0;
                if (active && sidx >= 0 && sidx < n) {
                    const int8_t *px = fr.in + (sidx * npol + pol) * 2;
                    re = px[0];
                    im = px[1];
                }
                U[j1] = re + 256 * im;
                V[j1] = re - 256 * im;
            }
            // forward: step A over j1, B and C, D over j2 -> X[t + 8 br3(i)]
            fnt_fwd<8, kBeta, 13>(U);
            fnt_fwd<8, kBeta, 13>(V);
            split_exchange<true, false>(U, tw1, TU, t);
            split_exchange<true, false>(V, tw1, TV, t);
            fnt_fwd<8, kBeta, 17>(U);
            fnt_fwd<8, kBeta, 17>(V);
            // products with the tap spectra and eqs. (7)/(8)
            const ZArith za;
            spectral_products(za, U, hu);
            spectral_products(za, V, hv);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int32_t a = U[i] + V[i], c = U[i] - V[i];
                U[i] = rho(a);
                V[i] = za.mulpow2(c, -256);
            }
            // inverse: step A over k2 (bit-reversed input), B and C, D over k1 -> z[t + 8 n1]
            fnt_inv<8, kBeta, 17>(U);
            fnt_inv<8, kBeta, 17>(V);
            split_exchange<false, true>(U, tw2, TU, t);
            split_exchange<false, true>(V, tw2, TV, t);
            fnt_inv<8, kBeta, 17>(U);
            fnt_inv<8, kBeta, 17>(V);
            if (!active) continue;
            // |z| <= 31 * 1024 < 32767, so the centred residue is the value
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                const int pos = t + 8 * n1;
                if (pos < kN - S) continue;
                const int64_t so = b * S + pos - (kN - S);
                if (so >= n) continue;
                const int32_t re = rhoc(U[n1]), im = rhoc(V[n1]);
                if (!CHAIN) {
                    ((uint32_t *)fr.out)[so * npol + pol] = ((uint32_t)re & 0xFFFFu) | ((uint32_t)im << 16);
                } else if (((so - fr.phase) & 1) == 0 && so >= fr.phase) {
                    const int sft = fr.shift;
                    const int32_t rnd = sft > 0 ? (1 << (sft - 1)) : 0;
                    const uint32_t qv = (uint32_t)(sat5((re + rnd) >> sft) & 0xFF) |
                                        ((uint32_t)(sat5((im + rnd) >> sft) & 0xFF) << 8);
                    ((uint16_t *)fr.aeq_in)[2 * ((so - fr.phase) >> 1) + pol] = (uint16_t)qv;
                }
            }
        }
    }
}

}  // namespace

size_t cdc_smem_bytes(int warps) { return (size_t)warps * kWarpWords * sizeof(uint32_t); }

// Pointwise products mod F per overlap-save block and polarisation (P = FNT(u)
// H_u and Q = FNT(v) H_v): the spectral stage the kernel runs (cdc_block),
// executed on the host with the counting policy.
int cdc_mults_per_block() {
    int mults = 0, shifts = 0;
    int32_t P[kN] = {}, Q[kN] = {}, hs[2 * kN] = {};
    cdc_spectral_stage(CountArith{&mults, &shifts}, P, Q, hs, [](int32_t (&)[kN]) {});
    return mults;
}
int cdc_butterflies_per_block() { return 4 * (kN / 2) * 6; }

cudaError_t cdc_read_faults(unsigned *faults, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(faults, g_fnt_faults, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_fnt_faults, &zero, sizeof zero);
    }
    return e;
}

cudaError_t cdc_configure() {
    const int max_smem = (int)cdc_smem_bytes(8);
    cudaError_t e = cudaFuncSetAttribute(cdc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cdc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cdc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cdc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

cudaError_t cdc_spectra_launch(const DevFrame *frames, int n_frames, cudaStream_t stream) {
    if (n_frames <= 0) return cudaSuccess;
    cdc_spectra_kernel<<<n_frames < 65535 ? n_frames : 65535, 2 * kN, 0, stream>>>(frames, n_frames);
    return cudaGetLastError();
}

cudaError_t cdc_launch(const DevFrame *frames, const int4 *items, int n_items, bool chain, bool both, int warps,
                       int grid, cudaStream_t stream, bool split) {
    if (n_items <= 0) return cudaSuccess;
    if (split) {
        const int sgrid = (int)std::min<int64_t>(((int64_t)n_items * kSplitWarpsPerItem + kSplitWarps - 1) / kSplitWarps,
                                                 1 << 20);
        if (chain)
            cdc_split_kernel<true><<<sgrid, 32 * kSplitWarps, 0, stream>>>(frames, items, n_items);
        else
            cdc_split_kernel<false><<<sgrid, 32 * kSplitWarps, 0, stream>>>(frames, items, n_items);
        return cudaGetLastError();
    }
    const dim3 block(32 * warps);
    const size_t smem = cdc_smem_bytes(warps);
    if (chain && both)
        cdc_kernel<true, true><<<grid, block, smem, stream>>>(frames, items, n_items);
    else if (chain)
        cdc_kernel<true, false><<<grid, block, smem, stream>>>(frames, items, n_items);
    else if (both)
        cdc_kernel<false, true><<<grid, block, smem, stream>>>(frames, items, n_items);
    else
        cdc_kernel<false, false><<<grid, block, smem, stream>>>(frames, items, n_items);
    return cudaGetLastError();
}

}  // namespace fnt
