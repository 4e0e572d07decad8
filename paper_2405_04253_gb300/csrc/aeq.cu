// aeq.cu -- FNT-AEQ kernel: 4x4 real-valued MIMO equaliser with two 7-bit tap
// groups and the RDE tap update of eq. (6) (section "Proposed FNT-CDC&AEQ
// structure"), over Z_65537 with N = 32 / radix 2 or N = 64 / radix 4080.
//
// One warp runs one AEQ chain (a frame, or one segment of a long frame).  The
// tap update makes consecutive blocks of a chain a serial recurrence, so the
// parallelism inside a block is spread over the lanes:
//   lane = 16 p + 8 o + 2 s1 + g   (p: output polarisation, S2 = 2p + o,
//                                   s1: input stream, g: tap group hi / lo)
// Each lane owns the 16 master taps of filter S1 -> S2 in registers and, per
// block, runs the forward transform of its tap group, the product with the
// block's input spectrum, and the inverse transform -- one length-N transform
// pair per lane, 32 per block, as in the paper's per-pair convolution.  The
// four input spectra of 8 blocks at a time are computed by the 32 lanes
// together (one transform each) ahead of use, since they do not depend on the
// taps.  Results are combined through shared memory: y_S2 = sum over S1 of
// 128 c_hi + c_lo, z = sat16(y >> 7), e = R - |z|^2 per polarisation, then each
// lane accumulates the gradient of its 8 taps and the two lanes of a filter
// swap halves so both hold all 16 updated taps.
#include <cuda_runtime.h>

#include "internal.h"
#include "zf.cuh"

namespace fnt {

namespace {

template <int NA>
struct AeqCfg {
    static constexpr int K = kAeqK;
    static constexpr int SA = NA - K;                        // symbols per block
    static constexpr int PRE = 8;                            // blocks per input-spectrum batch
    static constexpr int XS = PRE * SA + K;                  // staged input symbols (char4 words)
    static constexpr int XF_ROW = NA + 1;
    static constexpr int XF = PRE * 4 * XF_ROW;              // input spectra [PRE][4][NA]
    static constexpr int RED_ROW = SA + 1;
    static constexpr int RED = 32 * RED_ROW;                 // per-lane weighted outputs
    static constexpr int ZS = 4 * SA;
    static constexpr int ES = 2 * SA;
    static constexpr int WORDS = XS + XF + RED + ZS + ES;
    static constexpr int32_t NINV = zcent(zinv(NA));
};

__device__ __forceinline__ int32_t sx8(uint32_t w, int sh) { return (int32_t)(w << (24 - sh)) >> 24; }

template <int NA, int64_t ALPHA>
__global__ void __launch_bounds__(128) aeq_kernel(const DevFrame *__restrict__ frames,
                                                  const AeqChain *__restrict__ chains, int n_chains,
                                                  AeqParams prm) {
    using C = AeqCfg<NA>;
    constexpr int K = C::K;
    constexpr int SA = C::SA;
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint32_t *xs = smem + warp * C::WORDS;
    int32_t *xf = (int32_t *)(xs + C::XS);
    int32_t *red = xf + C::XF;
    int32_t *zs = red + C::RED;
    int32_t *es = zs + C::ZS;

    const int p = lane >> 4;
    const int s2 = 2 * p + ((lane >> 3) & 1);
    const int s1 = (lane >> 1) & 3;
    const int g = lane & 1;                   // 0: hi group (weight 128), 1: lo group
    const int64_t A2 = (int64_t)prm.rde_a * prm.rde_a;
    const int mu = prm.mu_shift;

    for (int c = blockIdx.x * wpb + warp; c < n_chains; c += gridDim.x * wpb) {
        const AeqChain ch = chains[c];
        const DevFrame &fr = frames[ch.frame];
        const uint32_t *xin = (const uint32_t *)fr.aeq_in;
        int16_t *out = (int16_t *)fr.out;

        int32_t T[K];
#pragma unroll
        for (int k = 0; k < K; ++k) T[k] = ch.init[(s2 * 4 + s1) * K + k];

        const int64_t nblk = (ch.end - ch.begin + SA - 1) / SA;
        for (int64_t blk = 0; blk < nblk; ++blk) {
            const int bb = (int)(blk % C::PRE);
            const int64_t t0 = ch.begin + blk * SA;
            if (bb == 0) {
                __syncwarp();
                // symbols t0 - K + q of the next PRE blocks, zero outside [begin, end)
                for (int q = lane; q < C::XS; q += 32) {
                    const int64_t t = t0 - K + q;
                    xs[q] = (t >= ch.begin && t < ch.end) ? __ldg(xin + t) : 0u;
                }
                __syncwarp();
                {
                    const int bq = lane >> 2, sq = lane & 3;
                    int32_t x[NA];
#pragma unroll
                    for (int j = 0; j < NA; ++j) x[j] = sx8(xs[bq * SA + j], 8 * sq);
                    fnt_fwd<NA, ALPHA>(x);
                    int32_t *row = xf + (bq * 4 + sq) * C::XF_ROW;
#pragma unroll
                    for (int i = 0; i < NA; ++i) row[i] = rhoc(rho(rhoc(x[i]) * C::NINV));
                }
                __syncwarp();
            }

            // this lane's tap group, zero-padded to NA, through the transform pair
            int32_t y[NA];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int32_t W = T[k] >> 16;
                y[k] = g ? (W & 127) : (W >> 7);
            }
#pragma unroll
            for (int k = K; k < NA; ++k) y[k] = 0;
            fnt_fwd_halfzero<NA, ALPHA>(y);
            const int32_t *xrow = xf + (bb * 4 + s1) * C::XF_ROW;
#pragma unroll
            for (int i = 0; i < NA; ++i) y[i] = rho(rhoc(y[i]) * xrow[i]);
            fnt_inv<NA, ALPHA>(y);
            const int32_t wgt = g ? 1 : 128;
#pragma unroll
            for (int i = 0; i < SA; ++i) red[lane * C::RED_ROW + i] = decode(y[K + i]) * wgt;
            __syncwarp();

            // outputs, RDE error
            for (int q = lane; q < 2 * SA; q += 32) {
                const int pp = q >= SA ? 1 : 0;
                const int i = q - pp * SA;
                int32_t z0, z1;
                {
                    int32_t a0 = 0, a1 = 0;
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        a0 += red[(16 * pp + m) * C::RED_ROW + i];
                        a1 += red[(16 * pp + 8 + m) * C::RED_ROW + i];
                    }
                    z0 = min(max(a0 >> 7, -32768), 32767);
                    z1 = min(max(a1 >> 7, -32768), 32767);
                }
                const int64_t t = t0 + i;
                const bool valid = t < ch.end;
                const int64_t r2 = (int64_t)z0 * z0 + (int64_t)z1 * z1;
                const int64_t R = r2 < 6 * A2 ? 2 * A2 : (r2 < 14 * A2 ? 10 * A2 : 18 * A2);
                if (valid && t >= ch.keep)
                    *(uint32_t *)(out + t * 4 + 2 * pp) = ((uint32_t)z0 & 0xFFFFu) | ((uint32_t)z1 << 16);
                zs[(2 * pp) * SA + i] = valid ? z0 : 0;
                zs[(2 * pp + 1) * SA + i] = valid ? z1 : 0;
                es[pp * SA + i] = valid ? (int32_t)(R - r2) : 0;
            }
            __syncwarp();

            // eq. (6): G[k] = sum_i e_p[i] z_S2[i] x_S1[t0 + i - k], taps k = 8g + kk
            if (mu < 63) {
                int64_t acc[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) acc[kk] = 0;
                const uint32_t *xb = xs + bb * SA + K - 8 * g;
#pragma unroll 4
                for (int i = 0; i < SA; ++i) {
                    const int32_t e = es[p * SA + i];
                    const int32_t z = zs[s2 * SA + i];
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const int32_t xv = sx8(xb[i - kk], 8 * s1);
                        acc[kk] += (int64_t)e * (int64_t)(z * xv);
                    }
                }
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int32_t mine = g ? T[8 + kk] : T[kk];
                    int64_t v = (int64_t)mine + (acc[kk] >> mu);
                    v = v < -(1ll << 29) ? -(1ll << 29) : (v > (1ll << 29) - 1 ? (1ll << 29) - 1 : v);
                    const int32_t nv = (int32_t)v;
                    const int32_t other = __shfl_xor_sync(0xffffffffu, nv, 1);
                    T[kk] = g ? other : nv;
                    T[8 + kk] = g ? nv : other;
                }
            }
        }
        if (ch.write_state && g == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) fr.state[(s2 * 4 + s1) * K + k] = T[k];
        }
        __syncwarp();
    }
}

}  // namespace

size_t aeq_smem_bytes(int na, int warps) {
    return (size_t)warps * (na == 64 ? AeqCfg<64>::WORDS : AeqCfg<32>::WORDS) * sizeof(uint32_t);
}

cudaError_t aeq_configure() {
    cudaError_t e = cudaFuncSetAttribute(aeq_kernel<64, 4080>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)aeq_smem_bytes(64, 4));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(aeq_kernel<32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)aeq_smem_bytes(32, 4));
}

cudaError_t aeq_launch(int na, const DevFrame *frames, const AeqChain *chains, int n_chains, AeqParams prm,
                       int warps, int grid, cudaStream_t stream) {
    if (n_chains <= 0) return cudaSuccess;
    const dim3 block(32 * warps);
    const size_t smem = aeq_smem_bytes(na, warps);
    if (na == 64)
        aeq_kernel<64, 4080><<<grid, block, smem, stream>>>(frames, chains, n_chains, prm);
    else
        aeq_kernel<32, 2><<<grid, block, smem, stream>>>(frames, chains, n_chains, prm);
    return cudaGetLastError();
}

}  // namespace fnt
