// aeq.cu -- FNT-AEQ kernel: 4x4 real-valued MIMO equaliser with two 7-bit tap
// groups and the RDE tap update of eq. (6) (section "Proposed FNT-CDC&AEQ
// structure"), over Z_65537 with N = 32 / radix 2 or N = 64 / radix 4080.
//
// Work item = one AEQ chain (a frame, or one segment of a long frame) and one
// output polarisation p: the outputs S2 = 2p, 2p+1 depend on the shared input
// but not on each other's taps, so the two polarisations of a chain are
// independent recurrences and run in two warps.  Inside a warp,
//   lane = 2 t + h,   t = 8 o + 2 s1 + g   (o: output of the pair, s1: input
//                                           stream, g: tap group hi / lo)
// and the length-N transform pair of task t is split over its two lanes by
// even / odd frequency (h = frequency parity):
//   forward  X[2k'+h] = FNT_{N/2, alpha^2}( a_j + a_{j+N/2}            (h = 0)
//                                           (a_j - a_{j+N/2}) alpha^j ) (h = 1)
//   inverse  x[n']       = E0[n'] + alpha^-n' E1[n']
//            x[n' + N/2] = E0[n'] - alpha^-n' E1[n'],  E_h = IFNT_{N/2, alpha^2}(half h)
// so each lane runs ordinary N/2-point transforms with compile-time twiddles
// and one shuffle per output finishes the inverse.  The zero-padded taps sit in
// the first half, so the forward split needs no shuffle at all.
// At P = 1 the 16 master taps of each filter S1 -> S2 sit in a per-warp table
// in shared memory: each of the filter's four lanes accumulates the gradient of
// 4 of them, updates those 4 and writes them back, and every lane reads all 16
// for its tap transform.  At P > 1 every lane of the filter holds all 16 in
// registers and the four lanes swap their updated quarters once per period.  The gradient itself, a (4 inputs x 16
// taps) x symbols x (2 outputs) contraction, runs exactly on the tensor cores
// (gradient_mma below).  The input spectra (taps-independent) are
// computed 8 blocks ahead, one full N-point transform per lane, with N^-1
// folded in.  With an update period P > 1 the gradient is summed over P blocks
// and applied after every P-th block and the last one; in between the taps do
// not change, so each lane keeps its tap half-spectrum in shared memory and
// transforms the taps once per period.
#include <algorithm>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "zf.cuh"

namespace fnt {

namespace {

template <int NA, int64_t ALPHA>
struct AeqCfg {
    static constexpr int K = kAeqK;
    static constexpr int M = NA / 2;                         // values per lane
    static constexpr int SA = NA - K;                        // symbols per block
    // blocks per input-spectrum batch: 8 at N = 32 (one N-point transform per
    // lane); 4 at N = 64 (one N/2-point half per lane), which halves the staging
    // and spectrum memory so that more warps fit on an SM
    static constexpr int PRE = NA == 64 ? 4 : 8;
    // code-size choices: at N = 32 the fully unrolled forms are small and
    // faster; at N = 64 one N/2-point code copy run twice and a gradient loop
    // over 8-symbol runs keep the kernel inside the instruction cache
    static constexpr bool FULL_INPUT = NA == 32;             // input spectra as one N-point transform
    static constexpr int GRAD_OUTER = NA == 32 ? (NA - kAeqK) / 8 : 1;   // 8-symbol runs unrolled
    static constexpr int XS = PRE * SA + K;                  // staged input symbols (char4 words)
    static constexpr int HALF = M + 1;                       // padded half row
    static constexpr int XF_ROW = 2 * HALF + 1;              // conflict-free: rows 3 banks apart
    static constexpr int XF = PRE * 4 * XF_ROW;              // input spectra [PRE][4][2][M]
    static constexpr int RED_ROW = SA + 1;
    static constexpr int GS = 4 * K * 8;                     // gradient limb sums [S1][k][o, limb]
    static constexpr int RED = 16 * RED_ROW > GS ? 16 * RED_ROW : GS;  // per-task outputs, then GS
    static constexpr int KT = SA / 16;                       // k-steps of the gradient product
    static constexpr int EZ_ROW = SA / 2 + 4;                // f16 pairs per limb row; conflict-free
    static constexpr int EZH = 8 * EZ_ROW;                   // e z limbs [o, limb][SA] as f16
    static constexpr int EZ = EZH > 4 * SA ? EZH : 4 * SA;   // ... or e z limb pairs [2][SA] as int2
    static constexpr int WORDS = 2 * XS + XF + RED + EZ;     // xs double-buffered
    // then, at P = 1, the master taps [filter (o, s1)][k] (rows padded so that
    // 16-byte accesses are conflict-free); at P > 1 the tap half-spectra
    // [M][lane] of the period (the taps then stay in registers)
    static constexpr int TROW = K + 4;
    static constexpr int TAPS = 8 * TROW;
    static constexpr int WCACHE = 32 * M;
    static_assert(SA % 16 == 0 && (2 * XS + XF) % 4 == 0 && RED % 4 == 0 && WORDS % 4 == 0,
                  "16-byte aligned regions");
    static constexpr int32_t NINV = zcent(zinv(NA));
    static constexpr int64_t ALPHA2 = ALPHA * ALPHA % kF;    // radix of the half transforms
    static constexpr int64_t AINV = zinv(ALPHA);
};

__device__ __forceinline__ int32_t sx8(uint32_t w, int sh) { return (int32_t)(w << (24 - sh)) >> 24; }

// 4-byte asynchronous global -> shared copy; src_size 0 writes zeros.
__device__ __forceinline__ void cp_async4(uint32_t *smem, const uint32_t *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// (int64) a * b + c with one wide multiply-add.
__device__ __forceinline__ int64_t mad_wide(int32_t a, int32_t b, int64_t c) {
    int64_t d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// dst[q] = x[t_first + q] for q < WORDS, zero outside [lo, hi), issued asynchronously.
template <int WORDS>
__device__ __forceinline__ void stage_async(uint32_t *dst, const uint32_t *x, int64_t t_first, int64_t lo, int64_t hi,
                                            int lane) {
    for (int q = lane; q < WORDS; q += 32) {
        const int64_t t = t_first + q;
        const bool ok = t >= lo && t < hi;
        cp_async4(dst + q, ok ? x + t : x, ok);
    }
}

// Lane h = 1 of the forward split: (a_j - 0) * alpha^j for the zero-padded taps
// (|result| < 2^17).
template <int NA, int64_t ALPHA, int J>
struct SplitTaps {
    static __device__ __forceinline__ void run(int32_t (&x)[NA / 2], const int32_t (&w)[kAeqK], bool odd) {
        constexpr int32_t W = TwTab<NA, ALPHA>::tab.w[J];
        x[J] = odd ? rho(w[J] * W) : w[J];                          // |w W| < 2^22
        if constexpr (J + 1 < kAeqK) SplitTaps<NA, ALPHA, J + 1>::run(x, w, odd);
    }
};

// Even / odd split of an N-sample 5-bit input window (the first DIF stage):
// y_j = a_j + a_{j+N/2} (even half) or (a_j - a_{j+N/2}) alpha^j (odd half).
template <int NA, int64_t ALPHA, int J>
struct SplitInput {
    static __device__ __forceinline__ void run(int32_t (&y)[NA / 2], const uint32_t *xw, int sh, bool odd) {
        constexpr int32_t W = TwTab<NA, ALPHA>::tab.w[J];
        const int32_t a = sx8(xw[J], sh), b = sx8(xw[J + NA / 2], sh);
        y[J] = odd ? rho((a - b) * W) : a + b;                      // |a - b| <= 31: no overflow
        if constexpr (J + 1 < NA / 2) SplitInput<NA, ALPHA, J + 1>::run(y, xw, sh, odd);
    }
};

// Last inverse stage, fused with the store of the kept outputs.  Lane 0 holds
// E0, lane 1 holds E1 (natural order); output n' is E0[n'] + alpha^-n' E1[n']
// and output n' + M is E0[n'] - alpha^-n' E1[n'] (M = N/2).  Overlap-save keeps
// the outputs n >= K, as block position i = n - K.
//   JoinBoth, n' in [K, M): both outputs are kept; lane 0 forms the sum and
//     lane 1 the difference, after exchanging E0[n'] and alpha^-n' E1[n'].
//   JoinDiff, n' in [0, K): only the difference is kept; lane 0 forms it for
//     n' = j and lane 1 for n' = j + K/2 (j < K/2), one exchange serving both.
// Every lane thus produces (N - K)/2 outputs and no discarded one.  Each
// output v (|true value| <= 32512) is stored as it is; when the inputs were
// summed in Z_F (DEC) it is decoded first and masked by wgt (0 for all but the
// first input lane).  The tap-group weights 128 / 1 are applied where the
// outputs are summed.
template <bool DEC>
__device__ __forceinline__ int32_t join_value(int32_t v) {
    v = rhoc(v);
    return DEC ? decode(v) : v;
}

template <int NA, int64_t AINV, bool DEC, int J>
struct JoinBoth {
    static __device__ __forceinline__ void run(const int32_t (&x)[NA / 2], int32_t *row, int32_t wgt, bool odd) {
        constexpr int32_t W = TwTab<NA, AINV>::tab.w[J];
        const int32_t t = odd ? mulb<18, W>(x[J]) : x[J];         // lane 1 sends alpha^-n' E1[n']
        const int32_t r = __shfl_xor_sync(0xffffffffu, t, 1);
        const int32_t v = join_value<DEC>(odd ? r - t : t + r);
        row[J] = DEC ? v * wgt : v;
        if constexpr (J + 1 < NA / 2) JoinBoth<NA, AINV, DEC, J + 1>::run(x, row, wgt, odd);
    }
};

template <int NA, int64_t AINV, bool DEC, int J>
struct JoinDiff {
    static __device__ __forceinline__ void run(const int32_t (&x)[NA / 2], int32_t *row, int32_t wgt, bool odd) {
        constexpr int H = kAeqK / 2;
        constexpr int32_t WA = TwTab<NA, AINV>::tab.w[J], WB = TwTab<NA, AINV>::tab.w[J + H];
        // lane 0 sends E0[j + H] and keeps E0[j]; lane 1 sends alpha^-j E1[j] and
        // keeps alpha^-(j + H) E1[j + H]
        const int32_t send = odd ? mulb<18, WA>(x[J]) : x[J + H];
        const int32_t own = odd ? mulb<18, WB>(x[J + H]) : x[J];
        const int32_t r = __shfl_xor_sync(0xffffffffu, send, 1);
        const int32_t v = join_value<DEC>(odd ? r - own : own - r);
        row[J] = DEC ? v * wgt : v;
        if constexpr (J + 1 < H) JoinDiff<NA, AINV, DEC, J + 1>::run(x, row, wgt, odd);
    }
};

// Gradient of eq. (6) on the tensor cores, exactly.  Per block and output o,
//   G[S1][k][o] = sum_i A[S1][k][i] B[i][o],  A[S1][k][i] = x_S1[t0 + i - k],
//   B[i][o] = e[i] z_o[i],
// a (4 x 16) x SA x 2 product.  |e z| <= 2^31 * 2^15 = 2^46, so e z is split
// into four balanced limbs c_l in [-2048, 2047] (e z = sum c_l 2^(12 l)); the
// limbs and the 5-bit x are exact in f16, every product and every partial sum
// of a block is an integer below 2^24 (2048 * 16 * 48 < 2^21), so the f32
// accumulation is exact and the limb sums are recombined in int64.
// Adding kLimbBias = 2048 (1 + 2^12 + 2^24 + 2^36) makes the limbs plain 12-bit
// digits d_l = c_l + 2048 of a value in [0, 2^48).
constexpr int64_t kLimbBias = 0x800800800800ll;

__device__ __forceinline__ __half limb_half(uint32_t d) {
    // d in [0, 4096): 2^23 + d exactly as f32, minus 2^23 + 2048, then to f16
    return __float2half_rn(__int_as_float(0x4B000000u | d) - 8390656.0f);
}

// Limbs c_0 .. c_3 of u - kLimbBias (u = e z + kLimbBias) to col[l * RSH].
template <int RSH>
__device__ __forceinline__ void ez_limbs(int64_t u, __half *col) {
    const uint32_t lo = (uint32_t)u, hi = (uint32_t)((uint64_t)u >> 32);
    col[0] = limb_half(lo & 0xFFFu);
    col[RSH] = limb_half((lo >> 12) & 0xFFFu);
    col[2 * RSH] = limb_half(__funnelshift_r(lo, hi, 24) & 0xFFFu);
    col[3 * RSH] = limb_half((hi >> 4) & 0xFFFu);
}

// f16 pair (x_S1[j], x_S1[j + 1]) from the staged words of symbols j, j + 1
// (one byte per stream): 0x6400 + (x + 128) is 1152 + x in f16, exact for
// any int8 x, and 1152 is subtracted exactly.
template <int S1>
__device__ __forceinline__ uint32_t x_pair(uint32_t wa, uint32_t wb) {
    constexpr uint32_t sel = S1 | (S1 << 4) | ((4 + S1) << 8) | ((4 + S1) << 12);
    uint32_t r = (__byte_perm(wa, wb, sel) & 0x00FF00FFu) ^ 0x64806480u;
    __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&r), __halves2half2(__ushort_as_half(0x6480),
                                                                                   __ushort_as_half(0x6480)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One m-tile (input stream S1, taps 0..15) of the gradient product; the lane
// holds rows k = gr, gr + 8 and limb columns 2 t, 2 t + 1 of the result.
// A[k][i] = x[i - k] is Toeplitz: register pairs p[j] = x(2t - gr + 8 (j - 1) + {0, 1})
// cover every fragment of the KT k-steps.
template <class C, int S1>
__device__ __forceinline__ void gradient_tile(const uint32_t (&wa)[2 * C::KT + 1], const uint32_t (&wb)[2 * C::KT + 1],
                                              const uint32_t (&b0)[C::KT], const uint32_t (&b1)[C::KT],
                                              int32_t *gs, int gr, int t) {
    uint32_t pr[2 * C::KT + 1];
#pragma unroll
    for (int j = 0; j < 2 * C::KT + 1; ++j) pr[j] = x_pair<S1>(wa[j], wb[j]);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < C::KT; ++kt)
        mma16816(d, pr[2 * kt + 1], pr[2 * kt], pr[2 * kt + 2], pr[2 * kt + 1], b0[kt], b1[kt]);
    // every sum is an integer below 2^24: exact in f32 and in the conversion
    *(int2 *)(gs + (S1 * C::K + gr) * 8 + 2 * t) = make_int2(__float2int_rn(d[0]), __float2int_rn(d[1]));
    *(int2 *)(gs + (S1 * C::K + gr + 8) * 8 + 2 * t) = make_int2(__float2int_rn(d[2]), __float2int_rn(d[3]));
}

// gs[S1][k][4 o + l] = sum_i x_S1[t0 + i - k] c_l(e z_o)[i] for the block at xw
// (xw[m] = staged word of symbol t0 + m, m >= -K).
template <class C>
__device__ __forceinline__ void gradient_mma(const uint32_t *xw, const uint32_t *ezh, int32_t *gs, int lane) {
    const int gr = lane >> 2, t = lane & 3;
    const uint32_t *xb = xw + 2 * t - gr - 8;
    uint32_t wa[2 * C::KT + 1], wb[2 * C::KT + 1];
#pragma unroll
    for (int j = 0; j < 2 * C::KT + 1; ++j) {
        wa[j] = xb[8 * j];
        wb[j] = xb[8 * j + 1];
    }
    uint32_t b0[C::KT], b1[C::KT];
#pragma unroll
    for (int kt = 0; kt < C::KT; ++kt) {
        b0[kt] = ezh[gr * C::EZ_ROW + 8 * kt + t];
        b1[kt] = ezh[gr * C::EZ_ROW + 8 * kt + 4 + t];
    }
    gradient_tile<C, 0>(wa, wb, b0, b1, gs, gr, t);
    gradient_tile<C, 1>(wa, wb, b0, b1, gs, gr, t);
    gradient_tile<C, 2>(wa, wb, b0, b1, gs, gr, t);
    gradient_tile<C, 3>(wa, wb, b0, b1, gs, gr, t);
}

// PER: update period P > 1 (gradient summed over P blocks, tap spectra cached);
// the P = 1 instance is the per-block update with no period bookkeeping.
// MMA: the gradient on the tensor cores (exact, opt-in); otherwise int32 x
// int32 -> int64 multiply-adds on the integer pipes.
// FS: frequency-domain summation over the inputs is compiled in (freq_sum 1 or 2).
template <int NA, int64_t ALPHA, bool PER, bool MMA, bool FS>
__global__ void __launch_bounds__(128) aeq_kernel(const DevFrame *__restrict__ frames,
                                                  const AeqChain *__restrict__ chains, int n_items,
                                                  AeqParams prm) {
    using C = AeqCfg<NA, ALPHA>;
    constexpr int K = C::K;
    constexpr int M = C::M;
    constexpr int SA = C::SA;
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int period = PER ? prm.period : 1;
    const int words = C::WORDS + (PER ? C::WCACHE : C::TAPS);
    uint32_t *xs2 = smem + warp * words;          // two staging buffers of C::XS words
    int32_t *xf = (int32_t *)(xs2 + 2 * C::XS);
    int32_t *red = xf + C::XF;
    uint32_t *ezh = (uint32_t *)(red + C::RED);
    int2 *ezl = (int2 *)ezh;                      // integer gradient: e z_o as limbs (c0, c1) [o][SA]
    int32_t *tsm = (int32_t *)(ezh + C::EZ);             // P = 1: the warp's master taps, [filter][TROW]
    int32_t *wcache = tsm + lane;                         // P > 1: stride 32, conflict-free

    const int h = lane & 1;                   // frequency parity held by this lane
    const int task = lane >> 1;
    const int o = task >> 3;                  // output within the polarisation pair
    const int s1 = (task >> 1) & 3;
    const int g = task & 1;                   // 0: hi group (weight 128), 1: lo group
    const int k0 = 8 * g + 4 * h;             // this lane's 4 gradient taps
    // the 16 master taps of this lane's filter S1 -> S2 live in the warp's tap
    // table; the filter's four lanes (g, h) each own and update 4 of them
    int32_t *trow = tsm + (task >> 1) * C::TROW;
    const bool odd = h != 0;
    const int64_t A2 = (int64_t)prm.rde_a * prm.rde_a;
    const int mu = prm.mu_shift;

    for (int item = blockIdx.x * wpb + warp; item < n_items; item += gridDim.x * wpb) {
        const AeqChain ch = chains[item >> 1];
        const int p = item & 1;
        const int s2 = 2 * p + o;
        const DevFrame &fr = frames[ch.frame];
        const uint32_t *xin = (const uint32_t *)fr.aeq_in;
        int16_t *out = (int16_t *)fr.out;

        // P = 1: this lane's taps k0 .. k0 + 3 (T[0..3]), the filter's 16 in the
        // table; P > 1: all 16 of the filter in registers
        int32_t T[PER ? K : 4];
        if constexpr (PER) {
#pragma unroll
            for (int k = 0; k < K; ++k) T[k] = ch.init[(s2 * 4 + s1) * K + k];
        } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) T[kk] = ch.init[(s2 * 4 + s1) * K + k0 + kk];
            __syncwarp();                         // the previous item's last reads of the table
            *(int4 *)(trow + k0) = make_int4(T[0], T[1], T[2], T[3]);
        }

        const int64_t nblk = (ch.end - ch.begin + SA - 1) / SA;
        int64_t acc[4] = {0, 0, 0, 0};            // gradient of taps k0 .. k0 + 3 over the period
        int in_period = 0;                        // blocks of the current period done
        bool fsum = FS && prm.freq_sum == 1;      // this block sums the inputs in Z_F
        // input symbols of batch 0 (PRE blocks + K history); later batches are
        // prefetched one batch ahead into the other buffer
        __syncwarp();
        stage_async<C::XS>(xs2, xin, ch.begin - K, ch.lo, ch.end, lane);
        const uint32_t *xs = xs2;
        for (int64_t blk = 0; blk < nblk; ++blk) {
            const int bb = (int)(blk % C::PRE);
            const int64_t t0 = ch.begin + blk * SA;
            if (bb == 0) {
                const int64_t batch = blk / C::PRE;
                xs = xs2 + (batch & 1) * C::XS;
                cp_async_wait_all();
                __syncwarp();
                if (blk + C::PRE < nblk)
                    stage_async<C::XS>(xs2 + ((batch + 1) & 1) * C::XS, xin, t0 + C::PRE * SA - K, ch.lo, ch.end,
                                       lane);
                {
                    // N-point spectra of the batch's inputs, N^-1 folded in, as even
                    // and odd halves in bit-reversed order: row (block, input) holds
                    // X[2k'+hh] at hh HALF + bitrev_M(k')
                    if constexpr (C::FULL_INPUT) {
                        // lane = 4 block + input: one N-point transform, whose
                        // register hh M + j holds X[2 bitrev_M(j) + hh]
                        const int bq = lane >> 2, sq = lane & 3;
                        const uint32_t *xw = xs + bq * SA;
                        int32_t *row = xf + (bq * 4 + sq) * C::XF_ROW;
                        int32_t xv[NA];
#pragma unroll
                        for (int j = 0; j < NA; ++j) xv[j] = sx8(xw[j], 8 * sq);
                        fnt_fwd<NA, ALPHA, 5>(xv);                   // |x| <= 16
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                            for (int j = 0; j < M; ++j)
                                row[hh * C::HALF + j] = rhoc(rho(rhoc(xv[hh * M + j]) * C::NINV));
                    } else {
                        // X[2k'+hh] = FNT_{N/2, alpha^2} of a_j + a_{j+N/2} (hh = 0) or
                        // (a_j - a_{j+N/2}) alpha^j (hh = 1); lane = 8 block + 2 input + hh
                        static_assert(C::PRE == 4, "one half-transform per lane");
                        const int hb = lane >> 3, hs = (lane >> 1) & 3, hh = lane & 1;
                        int32_t y[M];
                        SplitInput<NA, ALPHA, 0>::run(y, xs + hb * SA, 8 * hs, hh != 0);
                        fnt_fwd<M, C::ALPHA2, 17>(y);
                        int32_t *hrow = xf + (hb * 4 + hs) * C::XF_ROW + hh * C::HALF;
#pragma unroll
                        for (int j = 0; j < M; ++j) hrow[j] = rhoc(rho(rhoc(y[j]) * C::NINV));
                    }
                }
                __syncwarp();
            }

            // tap group -> even / odd half spectrum in this lane (once per period)
            int32_t y[M];
            if (!PER || in_period == 0) {
                int32_t wv[K];
                // tap group of a master tap T (W = T >> 16): hi W >> 7 = T >> 23
                // (arithmetic shifts compose), lo W & 127 = (T >> 16) & 127
                const int tsh = g ? 16 : 23;
                const int32_t tmask = g ? 127 : -1;
                if constexpr (PER) {
#pragma unroll
                    for (int k = 0; k < K; ++k) wv[k] = (T[k] >> tsh) & tmask;
                } else {
#pragma unroll
                    for (int q = 0; q < K / 4; ++q) {
                        const int4 t4 = *(const int4 *)(trow + 4 * q);
                        wv[4 * q] = (t4.x >> tsh) & tmask;
                        wv[4 * q + 1] = (t4.y >> tsh) & tmask;
                        wv[4 * q + 2] = (t4.z >> tsh) & tmask;
                        wv[4 * q + 3] = (t4.w >> tsh) & tmask;
                    }
                }
                if (FS && prm.freq_sum == 2) {
                    // guard: 16 sum |w| of every (output, group) over the four
                    // inputs within 32767, so every summed output decodes exactly
                    int32_t l1 = 0;
#pragma unroll
                    for (int k = 0; k < K; ++k) l1 += abs(wv[k]);
                    l1 += __shfl_xor_sync(0xffffffffu, l1, 4);
                    l1 += __shfl_xor_sync(0xffffffffu, l1, 8);
                    fsum = __all_sync(0xffffffffu, 16 * l1 <= 32767);
                }
                SplitTaps<NA, ALPHA, 0>::run(y, wv, odd);
#pragma unroll
                for (int j = K; j < M; ++j) y[j] = 0;
                if constexpr (M >= 2 * K)
                    fnt_fwd_halfzero<M, C::ALPHA2, 17>(y);
                else
                    fnt_fwd<M, C::ALPHA2, 17>(y);
                if constexpr (PER) {
#pragma unroll
                    for (int j = 0; j < M; ++j) wcache[32 * j] = y[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) y[j] = wcache[32 * j];
            }
            const int32_t *xrow = xf + (bb * 4 + s1) * C::XF_ROW + h * C::HALF;
            spectral_products(RedArith{}, y, xrow);
            if (FS && fsum) {
                // frequency-domain summation: the four input lanes of an (output,
                // group, half) all hold the sum of their products in Z_F
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    y[j] = rho(y[j] + __shfl_xor_sync(0xffffffffu, y[j], 4));
                    y[j] = rho(y[j] + __shfl_xor_sync(0xffffffffu, y[j], 8));
                }
            }
            fnt_inv<M, C::ALPHA2, 17>(y);
            {
                // kept outputs n >= K -> block position i = n - K of this task's row;
                // with summation only the first input lane contributes
                int32_t *rrow = red + task * C::RED_ROW;
                if (FS && fsum) {
                    // a summed output may exceed the per-pair bound (and wraps with
                    // freq_sum = 1): the exact signed decode of the residue
                    const int32_t wgt = s1 != 0 ? 0 : 1;
                    if constexpr (M > K) JoinBoth<NA, C::AINV, true, K>::run(y, rrow - K + (odd ? M : 0), wgt, odd);
                    JoinDiff<NA, C::AINV, true, 0>::run(y, rrow + (M - K) + (odd ? K / 2 : 0), wgt, odd);
                } else {
                    if constexpr (M > K) JoinBoth<NA, C::AINV, false, K>::run(y, rrow - K + (odd ? M : 0), 1, odd);
                    JoinDiff<NA, C::AINV, false, 0>::run(y, rrow + (M - K) + (odd ? K / 2 : 0), 1, odd);
                }
            }
            __syncwarp();

            // outputs and RDE error of this polarisation; e z of each output as
            // four balanced 12-bit limbs in f16 (the B operand of the gradient)
            for (int i = lane; i < SA; i += 32) {
                int32_t a0 = 0, a1 = 0;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    // task row m = 2 s1 + g: the hi group (g = 0) weighs 128
                    a0 += (m & 1 ? 1 : 128) * red[m * C::RED_ROW + i];
                    a1 += (m & 1 ? 1 : 128) * red[(8 + m) * C::RED_ROW + i];
                }
                const int32_t z0 = min(max(a0 >> 7, -32768), 32767);
                const int32_t z1 = min(max(a1 >> 7, -32768), 32767);
                const int64_t t = t0 + i;
                const bool valid = t < ch.end;
                const int64_t r2 = (int64_t)z0 * z0 + (int64_t)z1 * z1;
                const int64_t R = r2 < 6 * A2 ? 2 * A2 : (r2 < 14 * A2 ? 10 * A2 : 18 * A2);
                if (valid && t >= ch.keep)
                    *(uint32_t *)(out + t * 4 + 2 * p) = ((uint32_t)z0 & 0xFFFFu) | ((uint32_t)z1 << 16);
                const int32_t e = valid ? (int32_t)(R - r2) : 0;
                if constexpr (MMA) {
                    if (mu < 63) {
                        __half *col = (__half *)ezh + i;         // row 4 o + l, stride 2 EZ_ROW halves
                        ez_limbs<2 * C::EZ_ROW>(mad_wide(e, z0, kLimbBias), col);
                        ez_limbs<2 * C::EZ_ROW>(mad_wide(e, z1, kLimbBias), col + 8 * C::EZ_ROW);
                    }
                } else {
                    // e z_o (|e z| <= 2^46) = c1 2^23 + c0, 0 <= c0 < 2^23, |c1| <= 2^23
                    const int64_t ez0 = (int64_t)e * z0, ez1 = (int64_t)e * z1;
                    ezl[i] = make_int2((int32_t)(ez0 & 0x7FFFFF), (int32_t)(ez0 >> 23));
                    ezl[SA + i] = make_int2((int32_t)(ez1 & 0x7FFFFF), (int32_t)(ez1 >> 23));
                }
            }
            __syncwarp();

            // eq. (6): G[k] = sum_i e[i] z_S2[i] x_S1[t0 + i - k], summed over the
            // blocks of the update period
            const bool apply = !PER || ++in_period == period || blk + 1 == nblk;
            if (PER && apply) in_period = 0;
            if (mu < 63) {
                if constexpr (MMA) {
                    gradient_mma<C>(xs + bb * SA + K, ezh, red, lane);
                    __syncwarp();
                    // this lane's taps k0 .. k0 + 3: G = sum_limb c_limb 2^(12 limb)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int4 c4 = *(const int4 *)(red + (s1 * K + k0 + kk) * 8 + 4 * o);
                        int64_t v = acc[kk] + c4.x;
                        v = mad_wide(c4.y, 1 << 12, v);
                        v = mad_wide(c4.z, 1 << 24, v);
                        acc[kk] = v + ((int64_t)c4.w << 36);
                    }
                    __syncwarp();                         // gs is rewritten by the next block
                } else {
                    // taps k0 .. k0 + 3 over a rolling window w0..w3 = x_S1[t0 + i - k0 - kk],
                    // read as sign-extending byte loads of stream s1 from the staged words;
                    // G = sum_i (c1_i 2^23 + c0_i) w: the limb sums run in int32 over 8
                    // symbols at a time (below 8 2^23 16 = 2^30, exact) and then fold
                    // into the int64 sums
                    const int8_t *xb = (const int8_t *)(xs + bb * SA + K - k0) + s1;
                    int32_t w1 = xb[-4], w2 = xb[-8], w3 = xb[-12];
                    const int2 *ezrow = ezl + o * SA;
#pragma unroll C::GRAD_OUTER
                    for (int i8 = 0; i8 < SA; i8 += 8) {
                        int32_t l0[4] = {0, 0, 0, 0}, l1[4] = {0, 0, 0, 0};
#pragma unroll
                        for (int ii = 0; ii < 8; ++ii) {
                            const int i = i8 + ii;
                            const int32_t w0 = xb[4 * i];
                            const int2 c = ezrow[i];
                            l0[0] += c.x * w0;
                            l1[0] += c.y * w0;
                            l0[1] += c.x * w1;
                            l1[1] += c.y * w1;
                            l0[2] += c.x * w2;
                            l1[2] += c.y * w2;
                            l0[3] += c.x * w3;
                            l1[3] += c.y * w3;
                            w3 = w2;
                            w2 = w1;
                            w1 = w0;
                        }
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) acc[kk] += ((int64_t)l1[kk] << 23) + l0[kk];
                    }
                }
                if (apply) {
                    int32_t nv[4];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        // T[k0 + kk], by selects (no dynamic register indexing)
                        const int32_t cur =
                            PER ? (h ? (g ? T[(12 + kk) % (PER ? K : 4)] : T[(4 + kk) % (PER ? K : 4)])
                                     : (g ? T[(8 + kk) % (PER ? K : 4)] : T[kk]))
                                : T[kk];
                        int64_t v = (int64_t)cur + (acc[kk] >> mu);
                        v = v < -(1ll << 29) ? -(1ll << 29) : (v > (1ll << 29) - 1 ? (1ll << 29) - 1 : v);
                        nv[kk] = (int32_t)v;
                        acc[kk] = 0;
                    }
                    if constexpr (PER) {
                        // gather the filter's 16 taps from its four lanes (lane bit 0 = h,
                        // bit 1 = g); once per period
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const int32_t a = nv[kk];                                 // (g, h)
                            const int32_t b = __shfl_xor_sync(0xffffffffu, a, 1);     // (g, 1-h)
                            const int32_t c2 = __shfl_xor_sync(0xffffffffu, a, 2);    // (1-g, h)
                            const int32_t d = __shfl_xor_sync(0xffffffffu, b, 2);     // (1-g, 1-h)
                            T[kk] = g ? (h ? d : c2) : (h ? b : a);                   // g=0, h=0
                            T[4 + kk] = g ? (h ? c2 : d) : (h ? a : b);               // g=0, h=1
                            T[8 + kk] = g ? (h ? b : a) : (h ? d : c2);               // g=1, h=0
                            T[12 + kk] = g ? (h ? a : b) : (h ? c2 : d);              // g=1, h=1
                        }
                    } else {
                        // publish this lane's quarter of the filter's taps; the next
                        // block's tap transform reads all 16 from the table
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) T[kk] = nv[kk];
                        *(int4 *)(trow + k0) = make_int4(T[0], T[1], T[2], T[3]);
                        __syncwarp();
                    }
                }
            }
        }
        if (ch.write_state) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int32_t v = PER ? (h ? (g ? T[(12 + kk) % (PER ? K : 4)] : T[(4 + kk) % (PER ? K : 4)])
                                           : (g ? T[(8 + kk) % (PER ? K : 4)] : T[kk]))
                                      : T[kk];
                fr.state[(s2 * 4 + s1) * K + k0 + kk] = v;
            }
        }
        __syncwarp();
    }
}

}  // namespace

// Pointwise products mod F per AEQ block of both polarisations: every lane of
// a polarisation's warp runs the product stage of its task's N/2-point half
// once per block (16 tasks x 2 halves = 32 lanes); the stage is the kernel's
// own spectral_products, executed on the host with the counting policy.
template <int NA>
static int aeq_lane_products() {
    int mults = 0, shifts = 0;
    int32_t y[NA / 2] = {}, x[NA / 2] = {};
    spectral_products(CountArith{&mults, &shifts}, y, x);
    return mults;
}

int aeq_mults_per_block(int na) {
    constexpr int kLanesPerPol = 32;
    return 2 * kLanesPerPol * (na == 64 ? aeq_lane_products<64>() : aeq_lane_products<32>());
}

size_t aeq_smem_bytes(int na, int warps, int period) {
    const int words = na == 64 ? AeqCfg<64, 4080>::WORDS + (period > 1 ? AeqCfg<64, 4080>::WCACHE : AeqCfg<64, 4080>::TAPS)
                               : AeqCfg<32, 2>::WORDS + (period > 1 ? AeqCfg<32, 2>::WCACHE : AeqCfg<32, 2>::TAPS);
    return (size_t)warps * words * sizeof(uint32_t);
}

template <int NA, int64_t ALPHA, bool PER, bool MMA, bool FS>
static cudaError_t aeq_configure_one(int max_smem) {
    // up to the device's opt-in maximum: launches may reserve more than they use
    // to cap the CTAs per SM
    return cudaFuncSetAttribute(aeq_kernel<NA, ALPHA, PER, MMA, FS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                std::max(max_smem, (int)aeq_smem_bytes(NA, 4, PER ? 2 : 1)));
}

template <int NA, int64_t ALPHA, bool PER, bool MMA>
static cudaError_t aeq_configure_fs(int max_smem) {
    cudaError_t e = aeq_configure_one<NA, ALPHA, PER, MMA, false>(max_smem);
    return e == cudaSuccess ? aeq_configure_one<NA, ALPHA, PER, MMA, true>(max_smem) : e;
}

template <int NA, int64_t ALPHA>
static cudaError_t aeq_configure_n(int max_smem) {
    cudaError_t e = aeq_configure_fs<NA, ALPHA, false, false>(max_smem);
    if (e == cudaSuccess) e = aeq_configure_fs<NA, ALPHA, true, false>(max_smem);
    if (e == cudaSuccess) e = aeq_configure_fs<NA, ALPHA, false, true>(max_smem);
    if (e == cudaSuccess) e = aeq_configure_fs<NA, ALPHA, true, true>(max_smem);
    return e;
}

cudaError_t aeq_configure() {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = aeq_configure_n<64, 4080>(max_smem);
    return e == cudaSuccess ? aeq_configure_n<32, 2>(max_smem) : e;
}

template <int NA, int64_t ALPHA, bool PER, bool MMA>
static void aeq_launch_fs(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const DevFrame *frames,
                          const AeqChain *chains, int n_items, AeqParams prm) {
    if (prm.freq_sum != 0)
        aeq_kernel<NA, ALPHA, PER, MMA, true><<<grid, block, smem, stream>>>(frames, chains, n_items, prm);
    else
        aeq_kernel<NA, ALPHA, PER, MMA, false><<<grid, block, smem, stream>>>(frames, chains, n_items, prm);
}

template <int NA, int64_t ALPHA>
static void aeq_launch_n(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const DevFrame *frames,
                         const AeqChain *chains, int n_items, AeqParams prm, bool mma) {
    const bool per = prm.period > 1;
    if (mma) {
        if (per)
            aeq_launch_fs<NA, ALPHA, true, true>(grid, block, smem, stream, frames, chains, n_items, prm);
        else
            aeq_launch_fs<NA, ALPHA, false, true>(grid, block, smem, stream, frames, chains, n_items, prm);
    } else {
        if (per)
            aeq_launch_fs<NA, ALPHA, true, false>(grid, block, smem, stream, frames, chains, n_items, prm);
        else
            aeq_launch_fs<NA, ALPHA, false, false>(grid, block, smem, stream, frames, chains, n_items, prm);
    }
}

cudaError_t aeq_launch(int na, const DevFrame *frames, const AeqChain *chains, int n_chains, AeqParams prm,
                       int warps, int grid, cudaStream_t stream, size_t min_smem) {
    if (n_chains <= 0) return cudaSuccess;
    const dim3 block(32 * warps);
    // min_smem reserves extra shared memory to cap the CTAs resident per SM
    const size_t smem = std::max(aeq_smem_bytes(na, warps, prm.period), min_smem);
    const int n_items = 2 * n_chains;
    if (grid <= 0) grid = (n_items + warps - 1) / warps;
    if (na == 64)
        aeq_launch_n<64, 4080>(dim3(grid), block, smem, stream, frames, chains, n_items, prm, prm.tensor_gradient != 0);
    else
        aeq_launch_n<32, 2>(dim3(grid), block, smem, stream, frames, chains, n_items, prm, prm.tensor_gradient != 0);
    return cudaGetLastError();
}

}  // namespace fnt
