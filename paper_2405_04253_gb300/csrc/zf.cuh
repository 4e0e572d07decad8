// zf.cuh -- arithmetic in Z_F, F = 2^16 + 1 = 65537, and per-thread length-N
// Fermat number transforms (eq. (1) / eq. (2) of the paper, section "Fermat
// number transform") for sm_103a.
//
// Representation.  Values are int32 "lazy residues": any x with x = v (mod F)
// and |x| < 2^17 stands for the residue v.  Reduction by a Fermat modulus is
// split-and-subtract: t = h * 2^16 + l  ==>  t = l - h (mod F), because
// 2^16 = -1 (mod F).  On the GPU that is one shift and one multiply-add:
//     rho(t)  = t - (t >> 16) * F                      -> [-32767, 98303]
//     rhoc(t) = t - ((t + 2^15) >> 16) * F             -> |r| <= 2^15 + |t| / 2^16
// (the multiply runs on the FMA pipe, the shift on the integer pipe).
//
// Transforms.  One thread owns a whole length-N transform in N registers; every
// index and twiddle is a compile-time constant after unrolling, so "bit-reversed
// order" costs nothing.  The radix-2 decimation-in-frequency network
// (a, b) -> (a + b, (a - b) w) takes natural order and leaves X[k] in register
// bitrev(k).  The inverse runs the same network with alpha^-1 through a
// bit-reversed view of the registers, which consumes bit-reversed spectra and
// leaves natural-order samples.  Twiddles are stored as centred residues
// (|w| <= 2^15); the powers of the radix sqrt(2) = 4080 or 2 make most of them
// small powers of two, which keeps most products inside 32 bits without a
// pre-reduction.
#pragma once

#include <cstdint>

#ifndef FNT_HD
#define FNT_HD __host__ __device__ __forceinline__
#endif

namespace fnt {

constexpr int32_t kF = 65537;

constexpr int64_t zmod(int64_t v) { return ((v % kF) + kF) % kF; }

constexpr int64_t zpow(int64_t a, int64_t e) {
    int64_t r = 1, b = zmod(a);
    while (e > 0) {
        if (e & 1) r = r * b % kF;
        b = b * b % kF;
        e >>= 1;
    }
    return r;
}

constexpr int64_t zinv(int64_t a) { return zpow(a, kF - 2); }   // F is prime

// Centred representative in [-32768, 32768].
constexpr int32_t zcent(int64_t v) {
    int64_t r = zmod(v);
    return r > 32768 ? (int32_t)(r - kF) : (int32_t)r;
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// Centred powers alpha^e, e in [0, N).
template <int N, int64_t ALPHA>
struct Twiddles {
    int32_t w[N];
    constexpr Twiddles() : w() {
        for (int e = 0; e < N; ++e) w[e] = zcent(zpow(ALPHA, e));
    }
};

template <int N, int64_t ALPHA>
struct TwTab {
    static constexpr Twiddles<N, ALPHA> tab{};
};

// ------------------------------------------------------------- reductions ----

FNT_HD int32_t rho(int32_t t) {
    // l - h with t = h * 2^16 + l; exact in wrapping 32-bit arithmetic because the
    // result fits in int32.
    return (int32_t)((uint32_t)t - (uint32_t)(t >> 16) * (uint32_t)kF);
}

FNT_HD int32_t rhoc(int32_t t) {
    // requires |t| < 2^31 - 2^15
    return (int32_t)((uint32_t)t - (uint32_t)((t + 32768) >> 16) * (uint32_t)kF);
}

// Exact signed value of a residue whose true integer value v satisfies
// |v| <= 32768 (constraint (5)), from any lazy x = v (mod F) with |x| < 2^24.
FNT_HD int32_t decode(int32_t x) {
    int32_t r = rhoc(x);                 // |r| <= 32768 + 256
    r = r > 32768 ? r - kF : r;
    r = r < -32768 ? r + kF : r;
    return r;
}

// Runtime variant for a centred constant w (|w| <= 2^15) and |x| < 2^30.
FNT_HD int32_t mulw(int32_t x, int32_t w) { return rho(rhoc(x) * w); }

// ------------------------------------------------------ spectral products ----
//
// The pointwise spectrum products of the kernels go through an arithmetic
// policy: ZArith is what the kernels run, and the host instantiates the same
// templates with a counting policy to report how many multiplications the
// kernels' product stages issue (the counts of Tab. 1).  mulmod is a product of
// two arbitrary residues; mulpow2 multiplies by a signed power of two (a shift
// in the paper's cost model, which Tab. 1 does not count).
struct ZArith {
    FNT_HD int32_t mulmod(int32_t a, int32_t h) const { return rho(rhoc(a) * h); }   // |a| < 2^30, |h| <= 2^15
    FNT_HD int32_t mulpow2(int32_t a, int32_t c) const { return rho(a * c); }         // |a c| < 2^31
};

// a b (mod F) as a lazy residue (|result| < 2^17) for |a| < 2^18, |b| <= 2^15 + 8:
// the 64-bit product is hi 2^32 + lo with 2^32 = 1 (mod F), and lo = l1 2^16 + l0
// with 2^16 = -1, so a b = hi + l0 - l1 (mod F).  Four instructions where
// rho(rhoc(a) b) takes six.
FNT_HD int32_t mulred(int32_t a, int32_t b) {
    const int64_t t = (int64_t)a * b;
    const uint32_t lo = (uint32_t)t;
    return (int32_t)(t >> 32) + (int32_t)(lo & 0xFFFFu) - (int32_t)(lo >> 16);
}

// The same products through mulred (operands within mulred's bounds).
struct RedArith {
    FNT_HD int32_t mulmod(int32_t a, int32_t h) const { return mulred(a, h); }
    FNT_HD int32_t mulpow2(int32_t a, int32_t c) const { return rho(a * c); }
};

// Host policy that counts, instead of computing: general products in *mults,
// power-of-two multiplications in *shifts.
struct CountArith {
    int *mults, *shifts;
    FNT_HD int32_t mulmod(int32_t, int32_t) const { return ++*mults, 0; }      // host use only
    FNT_HD int32_t mulpow2(int32_t, int32_t) const { return ++*shifts, 0; }
};

// x[i] <- x[i] h[i] (mod F), i < N: one transform's pointwise product.
template <class A, int N>
FNT_HD void spectral_products(const A &ar, int32_t (&x)[N], const int32_t *h) {
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = ar.mulmod(x[i], h[i]);
}

// -------------------------------------------------------------- transforms ----
//
// Lazy reduction.  Every register of a transform carries a compile-time bound
// b (|x| < 2^b), computed stage by stage in a constexpr plan from the bound of
// the inputs.  A butterfly reduces its sum only when the sum's bound would pass
// LIM, keeps a twiddle product unreduced while it stays under LIM, multiplies
// directly when |d| |w| < 2^31 and pre-reduces with rhoc only when it would
// not.  With LIM = 21 most butterflies cost 4-5 integer instructions instead
// of 8-10 for full reduction, and no intermediate ever leaves int32.

constexpr int bits_of(int64_t v) {   // smallest m with |v| <= 2^m
    int64_t a = v < 0 ? -v : v;
    int m = 0;
    while (((int64_t)1 << m) < a) ++m;
    return m;
}

constexpr int kLazyLim = 21;

enum : unsigned char { kSumLazy = 0, kSumRho = 1 };
enum : unsigned char { kDiffLazy = 0, kDiffRho = 1, kMulLazy = 2, kMulRho = 3, kMulRhoc = 4 };

template <int N, int64_t ALPHA, int INB, int OUTB>
struct LazyPlan {
    static constexpr int LOGN = ilog2(N);
    int b[LOGN + 1][N];                 // bound of position i at the input of stage s
    unsigned char ms[LOGN][N / 2];      // sum branch
    unsigned char md[LOGN][N / 2];      // difference branch
    constexpr LazyPlan() : b(), ms(), md() {
        for (int i = 0; i < N; ++i) b[0][i] = INB;
        for (int s = 0; s < LOGN; ++s) {
            const int half = N >> (s + 1);
            const int lim = (s + 1 == LOGN) ? (OUTB < kLazyLim ? OUTB : kLazyLim) : kLazyLim;
            for (int j = 0; j < N / 2; ++j) {
                const int blk = j / half, jj = j % half;
                const int i0 = blk * 2 * half + jj, i1 = i0 + half;
                const int bsum = (b[s][i0] > b[s][i1] ? b[s][i0] : b[s][i1]) + 1;
                if (bsum > lim) {
                    ms[s][j] = kSumRho;
                    b[s + 1][i0] = 17;
                } else {
                    ms[s][j] = kSumLazy;
                    b[s + 1][i0] = bsum;
                }
                const int64_t w = zcent(zpow(ALPHA, (int64_t)jj << s));
                if (w == 1) {
                    md[s][j] = bsum > lim ? kDiffRho : kDiffLazy;
                    b[s + 1][i1] = bsum > lim ? 17 : bsum;
                } else if (bsum + bits_of(w) <= 30) {
                    const int pb = bsum + bits_of(w);
                    md[s][j] = pb > lim ? kMulRho : kMulLazy;
                    b[s + 1][i1] = pb > lim ? 17 : pb;
                } else {
                    md[s][j] = kMulRhoc;
                    b[s + 1][i1] = 17;
                }
            }
        }
    }
};

template <int N, int64_t ALPHA, int INB, int OUTB>
struct LazyTab {
    static constexpr LazyPlan<N, ALPHA, INB, OUTB> plan{};
};

template <int N, int64_t ALPHA, int INB, int OUTB, bool BR, int S, int J>
struct DifStage {
    static FNT_HD void run(int32_t (&x)[N]) {
        constexpr int LOGN = ilog2(N);
        constexpr int HALF = N >> (S + 1);
        constexpr int BLK = J / HALF;
        constexpr int JJ = J % HALF;
        constexpr int I0 = BLK * 2 * HALF + JJ;
        constexpr int I1 = I0 + HALF;
        constexpr int R0 = BR ? bitrev(I0, LOGN) : I0;
        constexpr int R1 = BR ? bitrev(I1, LOGN) : I1;
        constexpr int32_t W = TwTab<N, ALPHA>::tab.w[JJ << S];
        constexpr unsigned char MS = LazyTab<N, ALPHA, INB, OUTB>::plan.ms[S][J];
        constexpr unsigned char MD = LazyTab<N, ALPHA, INB, OUTB>::plan.md[S][J];
        const int32_t a = x[R0], b = x[R1];
        const int32_t s = a + b;
        const int32_t d = a - b;
        x[R0] = MS == kSumRho ? rho(s) : s;
        if constexpr (MD == kDiffLazy) {
            x[R1] = d;
        } else if constexpr (MD == kDiffRho) {
            x[R1] = rho(d);
        } else if constexpr (MD == kMulLazy) {
            x[R1] = d * W;
        } else if constexpr (MD == kMulRho) {
            x[R1] = rho(d * W);
        } else {
            x[R1] = rho(rhoc(d) * W);
        }
        if constexpr (J + 1 < N / 2) DifStage<N, ALPHA, INB, OUTB, BR, S, J + 1>::run(x);
    }
};

template <int N, int64_t ALPHA, int INB, int OUTB, bool BR, int S>
struct Dif {
    static FNT_HD void run(int32_t (&x)[N]) {
        DifStage<N, ALPHA, INB, OUTB, BR, S, 0>::run(x);
        if constexpr (S + 1 < ilog2(N)) Dif<N, ALPHA, INB, OUTB, BR, S + 1>::run(x);
    }
};

// Forward transform, eq. (1) up to the final reduction: natural order in with
// |x| < 2^INB, X[k] in register bitrev(k) out with |X| < 2^18.
template <int N, int64_t ALPHA, int INB = 17, int OUTB = 18>
FNT_HD void fnt_fwd(int32_t (&x)[N]) {
    Dif<N, ALPHA, INB, OUTB, false, 0>::run(x);
}

// Inverse transform, eq. (2) without the factor N^-1: P[k] in register
// bitrev(k) in, p[n] in register n out; bounds as for fnt_fwd.
template <int N, int64_t ALPHA, int INB = 17, int OUTB = 18>
FNT_HD void fnt_inv(int32_t (&x)[N]) {
    Dif<N, zinv(ALPHA), INB, OUTB, true, 0>::run(x);
}

// Multiply a lazy value with |x| < 2^XB by a centred constant W, reduced.
template <int XB, int32_t W>
FNT_HD int32_t mulb(int32_t x) {
    if constexpr (W == 1) {
        return rho(x);
    } else if constexpr (XB + bits_of(W) <= 30) {
        return rho(x * W);
    } else {
        return rho(rhoc(x) * W);
    }
}

// Forward transform of a sequence whose entries N/2..N-1 are zero: the first
// stage reduces to (a, a * w); inputs |x| < 2^INB.
template <int N, int64_t ALPHA, int INB, int J>
struct DifFirstZeroPad {
    static FNT_HD void run(int32_t (&x)[N]) {
        constexpr int32_t W = TwTab<N, ALPHA>::tab.w[J];
        x[J + N / 2] = mulb<INB, W>(x[J]);
        if constexpr (J + 1 < N / 2) DifFirstZeroPad<N, ALPHA, INB, J + 1>::run(x);
    }
};

template <int N, int64_t ALPHA, int INB = 17, int OUTB = 18>
FNT_HD void fnt_fwd_halfzero(int32_t (&x)[N]) {
    DifFirstZeroPad<N, ALPHA, INB, 0>::run(x);
    if constexpr (N > 2) Dif<N, ALPHA, (INB > 17 ? INB : 17), OUTB, false, 1>::run(x);
}

}  // namespace fnt
