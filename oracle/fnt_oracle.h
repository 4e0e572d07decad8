/*
 * fnt_oracle.h -- declarations of the CPU reference (test infrastructure only).
 * This header belongs to the oracle alone; the CUDA library never includes it.
 */
#ifndef FNT_ORACLE_H
#define FNT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

long long orc_powmod(long long a, long long e, long long F);
long long orc_invmod(long long a, long long F);
long long orc_order(long long alpha, long long F);
int orc_check_transform(int N, long long alpha, long long F);
long long orc_decode(long long r, long long F);

void orc_fnt(const long long *x, long long *X, int N, long long alpha, long long F);
void orc_ifnt(const long long *X, long long *x, int N, long long alpha, long long F);

int orc_cdc(const int8_t *in, long long n, int n_pol, const int8_t *taps, int L,
            int N, long long alpha, int S, int32_t *out);

int orc_cdc_shift(const int8_t *taps, int L);
int orc_decim_phase(int L);
long long orc_requant_decimate(const int32_t *z, long long n, int shift, int phase, int8_t *x);

void orc_aeq_init_taps(int K, int w0, int32_t *T);
int orc_aeq(const int8_t *x, long long n_sym, int N, long long alpha, int K, int mu_shift,
            int rde_a, int32_t *T, int16_t *out, int use_fnt, int period, int freq_sum, int hist);
int orc_aeq_segmented(const int8_t *x, long long n_sym, int N, long long alpha, int K,
                      int mu_shift, int rde_a, const int32_t *T0, long long seg_len,
                      long long warmup, int32_t *T_out, int16_t *out, int use_fnt, int period,
                      int freq_sum);

#ifdef __cplusplus
}
#endif

#endif
