/*
 * Plain CPU oracle for the compression scheme of Masui et al.,
 * "A compression scheme for radio data in high performance computing"
 * (arXiv:1503.00638).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  The CUDA path shares
 * no code, header, table or constant with it.
 *
 * Everything here is written to be read against the paper, one element or one
 * bit at a time, with no blocking, fusion or reordering beyond what the paper's
 * definitions state.  Compile with -O2 -ffp-contract=off so that no multiply-add
 * is contracted (the float32 arithmetic of reading R1 below must be rounded
 * after every operation).
 *
 * Readings of the paper where it is silent (numbered R1, R2, ...):
 *   R1  q = 12 f s^2 is evaluated in float32, each operation rounded to
 *       nearest: c = fl32(6 f / N); cross q = (c * A_i) * A_j;
 *       auto q = ((2c) * A_i) * A_i.
 *   R2  no rounding when q is not a positive, finite, normal float32.
 *   R3  autos A_i are the unrounded real parts of product (i,i).
 *   R4  products are ordered upper-triangle row-major: (0,0),(0,1),..,(0,n-1),
 *       (1,1),(1,2),...
 *   R5  the sign of a value that rounds to zero is kept.
 *   R6  NaN and +-inf pass through; subnormals round like any other value.
 *   R7  rounding up past FLT_MAX gives +-inf.
 *   R9  a trailing partial block is shortened to a multiple of 8 elements and
 *       transposed like a full block; the last (n mod 8) elements are copied
 *       verbatim.
 *   R11 compressed framing: 8-byte big-endian uncompressed byte count, 4-byte
 *       big-endian block size in bytes, then per block a 4-byte big-endian
 *       compressed length followed by the LZ4 block, then the verbatim tail.
 *   R17 integer data: granularity 2^k with k <= 0 leaves the value alone; a
 *       nearest multiple above INT32_MAX is replaced by the lower multiple.
 *   R18 the compensated f of Sec. 3.2 is evaluated per (freq, time) sample,
 *       in float32 as stated at orc_compensation_min.
 *   R20 full-covariance noise: components after the redundancy removal of
 *       Sec. 3.1 in the order of orc_full_index; C from Eq. rad_full1-3 in
 *       fp64 from the float32 (or int32) values; s^2 = 1/(C^-1)_kk; a sample
 *       whose C is not positive definite is left unrounded; q = fl32(12 f s^2).
 */
#include <stddef.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#include <math.h>
#include <float.h>

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: noise from the radiometer equation                              */
/* ------------------------------------------------------------------------ */

/* Eq. rad_simple evaluated on its diagonal (g = i, h = j, beta = alpha):
 *   C_{aij,aij} = (1 + delta_ij) (1 - delta_ij delta_{a,Im}) V_ii V_jj / (2N).
 * For a diagonal covariance the unmarginalized noise of Eq. noise,
 * s^2 = 1 / (C^-1)_{aij,aij}, equals this diagonal entry.
 * alpha = 0 for the real part, 1 for the imaginary part.  fp64. */
double orc_rad_simple_var(int i, int j, int alpha, double Vii, double Vjj, double N)
{
    double d_ij = (i == j) ? 1.0 : 0.0;
    double d_aim = (alpha == 1) ? 1.0 : 0.0;
    return (1.0 + d_ij) * (1.0 - d_ij * d_aim) * Vii * Vjj / (2.0 * N);
}

/* Eq. rad_full1-3: covariance between component alpha of V_ij and component
 * beta of V_gh, from the complex correlation matrix V (n x n, row-major,
 * interleaved re/im, Hermitian).  fp64. */
double orc_rad_full_cov(const double *V, int n, int alpha, int i, int j,
                        int beta, int g, int h, double N)
{
#define VRE(a, b) V[2 * ((long)(a) * n + (b))]
#define VIM(a, b) V[2 * ((long)(a) * n + (b)) + 1]
    /* X = V_ig conj(V_jh),  Y = V_ih conj(V_jg) */
    double xr = VRE(i, g) * VRE(j, h) + VIM(i, g) * VIM(j, h);
    double xi = VIM(i, g) * VRE(j, h) - VRE(i, g) * VIM(j, h);
    double yr = VRE(i, h) * VRE(j, g) + VIM(i, h) * VIM(j, g);
    double yi = VIM(i, h) * VRE(j, g) - VRE(i, h) * VIM(j, g);
#undef VRE
#undef VIM
    if (alpha == 0 && beta == 0) return (xr + yr) / (2.0 * N);   /* rad_full1 */
    if (alpha == 1 && beta == 1) return (xr - yr) / (2.0 * N);   /* rad_full2 */
    if (alpha == 0 && beta == 1) return (-xi + yi) / (2.0 * N);  /* rad_full3 */
    /* C_{Im ij, Re gh} = C_{Re gh, Im ij}: rad_full3 with the pairs swapped */
    return orc_rad_full_cov(V, n, 0, g, h, 1, i, j, N);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: granularity and rounding                                        */
/* ------------------------------------------------------------------------ */

/* Reading R1: q = 12 f s^2 in float32 with a fixed operation order.
 * Cross (i != j): s^2 = A_i A_j / (2N)  =>  q = (6f/N) A_i A_j.
 * Auto real part: s^2 = A_i^2 / N     =>  q = (12f/N) A_i^2.          */
float orc_q32(int is_auto, float Ai, float Aj, double f, double N)
{
    float c = (float)(6.0 * f / N);
    if (is_auto) {
        float c2 = 2.0f * c;
        float t = c2 * Ai;
        return t * Ai;
    }
    float t = c * Ai;
    return t * Aj;
}

/* Eq. trunc_error: the granularity is the largest power of two g = 2^k with
 * g < sqrt(q), i.e. 4^k < q.  Found by exact comparisons in fp64 (q is a
 * float32, so it and every 4^k used here are exact doubles).
 * Returns 0 and leaves *k alone when reading R2 says "no rounding". */
int orc_granularity_exponent(float q, int *k)
{
    if (!(q > 0.0f) || !isfinite(q) || q < FLT_MIN) return 0;
    double qd = (double)q;
    int kk = 0;
    while (ldexp(1.0, 2 * kk) >= qd) kk--;
    while (ldexp(1.0, 2 * (kk + 1)) < qd) kk++;
    *k = kk;
    return 1;
}

/* Round x to the nearest multiple of 2^k, ties to the even multiple
 * (Sec. 3.2 and its footnote on IEEE 754 ties-to-even).  The scaling by 2^-k
 * and back is exact in fp64; nearbyint rounds half to even in the default
 * rounding mode; the final conversion is exact or overflows (R7). */
float orc_round_pow2(float x, int k)
{
    if (!isfinite(x)) return x;                       /* R6 */
    double y = nearbyint(ldexp((double)x, -k));
    return (float)ldexp(y, k);
}

/* One element: round x given its q (R2: no rounding when q is unusable). */
float orc_round_element(float x, float q)
{
    int k;
    if (!orc_granularity_exponent(q, &k)) return x;
    return orc_round_pow2(x, k);
}

/* Precision reduction of a visibility cube (Sec. 6, steps 1-3).
 * in/out: [n_freq][n_prod][n_time] complex64 stored as interleaved float32
 * (re, im), time fastest; n_prod = n_in (n_in + 1) / 2 in the order of R4.
 * Autos come from the unrounded input (R3).  Out of place. */
void orc_reduce_precision_c64(const float *in, float *out, long n_freq, long n_in,
                              long n_time, double N, double f)
{
    long n_prod = n_in * (n_in + 1) / 2;
    for (long fr = 0; fr < n_freq; fr++) {
        long p = 0;
        for (long i = 0; i < n_in; i++) {
            for (long j = i; j < n_in; j++, p++) {
                for (long t = 0; t < n_time; t++) {
                    long e = ((fr * n_prod + p) * n_time + t) * 2;
                    /* product (i,i) sits at index i*n_in - i*(i-1)/2 (R4) */
                    long pii = i * n_in - i * (i - 1) / 2;
                    long pjj = j * n_in - j * (j - 1) / 2;
                    float Ai = in[((fr * n_prod + pii) * n_time + t) * 2];
                    float Aj = in[((fr * n_prod + pjj) * n_time + t) * 2];
                    if (i == j) {
                        float q = orc_q32(1, Ai, Ai, f, N);
                        out[e] = orc_round_element(in[e], q);
                        out[e + 1] = in[e + 1];   /* s = 0 for Im V_ii */
                    } else {
                        float q = orc_q32(0, Ai, Aj, f, N);
                        out[e] = orc_round_element(in[e], q);
                        out[e + 1] = orc_round_element(in[e + 1], q);
                    }
                }
            }
        }
    }
}

/* ---- Integer visibilities (Sec. 3, Sec. 5: CHIME records int32 re/im) ---- */

/* Round an int32 to the nearest multiple of g = 2^k, ties to the even
 * multiple.  k <= 0 means g <= 1: no rounding (Sec. 5.1: a granularity of
 * unity implies no rounding for integers).  Reading R17: when the nearest
 * multiple is above INT32_MAX, the lower multiple is taken.  Exact in int64. */
int32_t orc_round_int(int32_t x, int k)
{
    if (k <= 0) return x;
    if (k > 62) return 0;            /* |x| < 2^31 < g/2 */
    int64_t g = (int64_t)1 << k;
    int64_t m = (int64_t)x / g;      /* toward zero; make it the floor */
    if ((int64_t)x - m * g < 0) m--;
    int64_t r = (int64_t)x - m * g;  /* 0 <= r < g */
    if (2 * r > g || (2 * r == g && (m & 1))) m++;
    int64_t y = m * g;
    if (y > INT32_MAX) y -= g;
    return (int32_t)y;
}

/* ---- Sec. 3.2: compensating f for correlated noise ----
 * f is multiplied by the minimum over cross products (i != j) of
 * 1 - V_ij V_ij^* / (V_ii V_jj).  Reading R18: per (freq, time) sample, with
 * rho = fl32(fl32(fl32(re re) + fl32(im im)) / fl32(A_i A_j)) and
 * 1 - rho in float32; a negative or NaN value counts as 0 (no rounding for
 * that sample), no cross product gives 1; the compensated constant is
 * c = fl32(6 f m / N) evaluated in fp64.  Values are float32 components, or
 * int32 components converted to float32 (round to nearest). */
static float comp_value(const void *in, int is_int, long idx)
{
    return is_int ? (float)((const int32_t *)in)[idx] : ((const float *)in)[idx];
}

float orc_compensation_min(const void *in, int is_int, long n_freq, long n_in, long n_time,
                           long fr, long t)
{
    long n_prod = n_in * (n_in + 1) / 2;
    float m = 1.0f;
    long p = 0;
    for (long i = 0; i < n_in; i++) {
        for (long j = i; j < n_in; j++, p++) {
            if (i == j) continue;
            long pii = i * n_in - i * (i - 1) / 2;
            long pjj = j * n_in - j * (j - 1) / 2;
            float Ai = comp_value(in, is_int, ((fr * n_prod + pii) * n_time + t) * 2);
            float Aj = comp_value(in, is_int, ((fr * n_prod + pjj) * n_time + t) * 2);
            float re = comp_value(in, is_int, ((fr * n_prod + p) * n_time + t) * 2);
            float im = comp_value(in, is_int, ((fr * n_prod + p) * n_time + t) * 2 + 1);
            float num = re * re + im * im;   /* each product rounded, then the sum */
            float den = Ai * Aj;
            float rho = num / den;
            float om = 1.0f - rho;
            if (!(om >= 0.0f)) om = 0.0f;
            if (om < m) m = om;
        }
    }
    (void)n_freq;
    return m;
}

/* Precision reduction of a cube of float32 (is_int = 0) or int32 (is_int = 1)
 * complex samples, optionally with the compensated f per (freq, time).
 * Otherwise as orc_reduce_precision_c64. */
void orc_reduce_precision(const void *in, void *out, int is_int, long n_freq, long n_in,
                          long n_time, double N, double f, int compensate)
{
    long n_prod = n_in * (n_in + 1) / 2;
    for (long fr = 0; fr < n_freq; fr++) {
        for (long t = 0; t < n_time; t++) {
            double fe = f;
            if (compensate) {
                float m = orc_compensation_min(in, is_int, n_freq, n_in, n_time, fr, t);
                fe = f * (double)m;
            }
            float c = (float)(6.0 * fe / N);   /* as orc_q32 with f = fe (fe = f when m = 1) */
            float c2 = 2.0f * c;
            long p = 0;
            for (long i = 0; i < n_in; i++) {
                for (long j = i; j < n_in; j++, p++) {
                    long e = ((fr * n_prod + p) * n_time + t) * 2;
                    long pii = i * n_in - i * (i - 1) / 2;
                    long pjj = j * n_in - j * (j - 1) / 2;
                    float Ai = comp_value(in, is_int, ((fr * n_prod + pii) * n_time + t) * 2);
                    float Aj = comp_value(in, is_int, ((fr * n_prod + pjj) * n_time + t) * 2);
                    float q = (i == j) ? (c2 * Ai) * Ai : (c * Ai) * Aj;
                    int k, ok = orc_granularity_exponent(q, &k);
                    for (int part = 0; part < 2; part++) {
                        int rounded = ok && !(i == j && part == 1);
                        if (is_int) {
                            int32_t x = ((const int32_t *)in)[e + part];
                            ((int32_t *)out)[e + part] = rounded ? orc_round_int(x, k) : x;
                        } else {
                            float x = ((const float *)in)[e + part];
                            ((float *)out)[e + part] = rounded ? orc_round_pow2(x, k) : x;
                        }
                    }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: noise from the full covariance (small arrays)                   */
/* ------------------------------------------------------------------------ */

/* After the redundancy removal of Sec. 3.1 (Re V_ji = Re V_ij, Im V_ji =
 * -Im V_ij, Im V_ii = 0 is dropped) the components of one (freq, time) sample
 * are, in this order: Re of every product p (p = 0 .. P-1, upper-triangle
 * row-major), then Im of every cross product (i < j) in the same order.
 * M = 2P - n = n^2 components.  Reading R20. */
long orc_full_index(long n, int i, int j, int alpha)
{
    long P = n * (n + 1) / 2;
    long p = (long)i * n - (long)i * (i - 1) / 2 + (j - i);
    return alpha == 0 ? p : P + p - i - 1;   /* i + 1 autos precede (i, j) */
}

/* The M x M covariance of Eq. rad_full1-3 (row-major) for the complex n x n
 * correlation matrix V (row-major, interleaved re/im, Hermitian). */
void orc_full_cov_matrix(const double *V, int n, double N, double *C)
{
    long M = (long)n * n;
    for (int i = 0; i < n; i++)
        for (int j = i; j < n; j++)
            for (int a = 0; a < 2; a++) {
                if (a == 1 && i == j) continue;
                long r = orc_full_index(n, i, j, a);
                for (int g = 0; g < n; g++)
                    for (int h = g; h < n; h++)
                        for (int b = 0; b < 2; b++) {
                            if (b == 1 && g == h) continue;
                            long c = orc_full_index(n, g, h, b);
                            C[r * M + c] = orc_rad_full_cov(V, n, a, i, j, b, g, h, N);
                        }
            }
}

/* Inverse of the M x M matrix A (destroyed) into Ainv by Gauss-Jordan
 * elimination without pivoting, which is exact arithmetic's route for a
 * positive definite matrix (every pivot is a Schur complement, hence > 0).
 * Returns 0, or -1 when a pivot is not positive and finite (the matrix is
 * not positive definite as far as fp64 can tell; reading R20). */
int orc_invert_spd(double *A, long M, double *Ainv)
{
    for (long r = 0; r < M; r++)
        for (long c = 0; c < M; c++) Ainv[r * M + c] = (r == c) ? 1.0 : 0.0;
    for (long k = 0; k < M; k++) {
        double piv = A[k * M + k];
        if (!(piv > 0.0) || !isfinite(piv)) return -1;
        for (long c = 0; c < M; c++) {
            A[k * M + c] /= piv;
            Ainv[k * M + c] /= piv;
        }
        for (long r = 0; r < M; r++) {
            if (r == k) continue;
            double m = A[r * M + k];
            if (m == 0.0) continue;
            for (long c = 0; c < M; c++) {
                A[r * M + c] -= m * A[k * M + c];
                Ainv[r * M + c] -= m * Ainv[k * M + c];
            }
        }
    }
    return 0;
}

/* Eq. noise: s^2 = 1 / (C^-1)_kk for every component of one sample, C from
 * Eq. rad_full1-3.  Returns 0, or -1 when C is not positive definite (s2 is
 * then all zero: no rounding for the sample).  fp64. */
int orc_full_noise_var(const double *V, int n, double N, double *s2)
{
    long M = (long)n * n;
    double *C = (double *)malloc(sizeof(double) * M * M);
    double *Ci = (double *)malloc(sizeof(double) * M * M);
    int rc = -1;
    if (C && Ci) {
        orc_full_cov_matrix(V, n, N, C);
        rc = orc_invert_spd(C, M, Ci);
        for (long k = 0; k < M; k++) s2[k] = rc == 0 ? 1.0 / Ci[k * M + k] : 0.0;
    }
    free(C);
    free(Ci);
    return rc;
}

/* Rounding of a float32 (is_int = 0) or int32 cube with the noise of Eq.
 * noise from the full covariance: per component q = fl32(12 f s^2) (the
 * product in fp64, rounded once), then the granularity and rounding of
 * orc_reduce_precision (R2-R7, R17).  Imaginary parts of autos stay. */
void orc_reduce_precision_full(const void *in, void *out, int is_int, long n_freq, long n_in,
                               long n_time, double N, double f)
{
    long n_prod = n_in * (n_in + 1) / 2, M = n_in * n_in;
    double *V = (double *)malloc(sizeof(double) * 2 * n_in * n_in);
    double *s2 = (double *)malloc(sizeof(double) * M);
    if (!V || !s2) {
        free(V);
        free(s2);
        return;
    }
    for (long fr = 0; fr < n_freq; fr++) {
        for (long t = 0; t < n_time; t++) {
            long p = 0;
            for (long i = 0; i < n_in; i++)
                for (long j = i; j < n_in; j++, p++) {
                    long e = ((fr * n_prod + p) * n_time + t) * 2;
                    double re = comp_value(in, is_int, e), im = comp_value(in, is_int, e + 1);
                    V[2 * (i * n_in + j)] = re;
                    V[2 * (i * n_in + j) + 1] = im;
                    V[2 * (j * n_in + i)] = re;
                    V[2 * (j * n_in + i) + 1] = -im;
                }
            orc_full_noise_var(V, (int)n_in, N, s2);
            p = 0;
            for (long i = 0; i < n_in; i++)
                for (long j = i; j < n_in; j++, p++)
                    for (int part = 0; part < 2; part++) {
                        long e = ((fr * n_prod + p) * n_time + t) * 2 + part;
                        int rounded = !(i == j && part == 1);
                        int k = 0, ok = 0;
                        if (rounded) {
                            float q = (float)(12.0 * f * s2[orc_full_index(n_in, (int)i, (int)j, part)]);
                            ok = orc_granularity_exponent(q, &k);
                        }
                        if (is_int) {
                            int32_t x = ((const int32_t *)in)[e];
                            ((int32_t *)out)[e] = ok ? orc_round_int(x, k) : x;
                        } else {
                            float x = ((const float *)in)[e];
                            ((float *)out)[e] = ok ? orc_round_pow2(x, k) : x;
                        }
                    }
        }
    }
    free(V);
    free(s2);
}

/* The granularity exponent chosen for every float of the cube (for tests of
 * Sec. 5.1's error distribution).  No rounding is marked as -1000. */
void orc_granularity_map_c64(const float *in, int32_t *kout, long n_freq, long n_in,
                             long n_time, double N, double f)
{
    long n_prod = n_in * (n_in + 1) / 2;
    for (long fr = 0; fr < n_freq; fr++) {
        long p = 0;
        for (long i = 0; i < n_in; i++) {
            for (long j = i; j < n_in; j++, p++) {
                for (long t = 0; t < n_time; t++) {
                    long e = ((fr * n_prod + p) * n_time + t) * 2;
                    long pii = i * n_in - i * (i - 1) / 2;
                    long pjj = j * n_in - j * (j - 1) / 2;
                    float Ai = in[((fr * n_prod + pii) * n_time + t) * 2];
                    float Aj = in[((fr * n_prod + pjj) * n_time + t) * 2];
                    int k;
                    float q = orc_q32(i == j, Ai, Aj, f, N);
                    int ok = orc_granularity_exponent(q, &k);
                    kout[e] = ok ? k : -1000;
                    kout[e + 1] = (ok && i != j) ? k : -1000;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2: the post-acquisition reorder                                       */
/* ------------------------------------------------------------------------ */

/* An instrument writes one time sample after another (time slowest); the
 * paper reorders after acquisition so that time varies fastest.  in holds
 * n_time rows of n_series elements of es bytes; out[s][t] = in[t][s]. */
void orc_reorder_time(const void *vin, void *vout, size_t n_time, size_t n_series, size_t es)
{
    const unsigned char *in = (const unsigned char *)vin;
    unsigned char *out = (unsigned char *)vout;
    for (size_t t = 0; t < n_time; t++)
        for (size_t s = 0; s < n_series; s++)
            memcpy(out + (s * n_time + t) * es, in + (t * n_series + s) * es, es);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2: Bitshuffle, the blocked bit transpose                           */
/* ------------------------------------------------------------------------ */

/* Bit r of element e (r = 8 * byte + bit, little-endian element, LSB = bit 0
 * as in the caption of Fig. f:bits) moves to bit-row r of the block:
 * byte r * (B/8) + e/8, bit e % 8.  Blocks of B elements, tail per R9. */
static void transpose_block(const uint8_t *in, uint8_t *out, size_t B, size_t es)
{
    memset(out, 0, B * es);
    for (size_t e = 0; e < B; e++) {
        for (size_t r = 0; r < 8 * es; r++) {
            unsigned bit = (in[e * es + r / 8] >> (r % 8)) & 1u;
            out[r * (B / 8) + e / 8] |= (uint8_t)(bit << (e % 8));
        }
    }
}

static void untranspose_block(const uint8_t *in, uint8_t *out, size_t B, size_t es)
{
    memset(out, 0, B * es);
    for (size_t e = 0; e < B; e++) {
        for (size_t r = 0; r < 8 * es; r++) {
            unsigned bit = (in[r * (B / 8) + e / 8] >> (e % 8)) & 1u;
            out[e * es + r / 8] |= (uint8_t)(bit << (r % 8));
        }
    }
}

static size_t default_block(size_t es, size_t block_elems)
{
    /* Sec. 4.2.1: the default block is 4096 bytes */
    return block_elems ? block_elems : 4096 / es;
}

int orc_bitshuffle(const void *vin, void *vout, size_t n, size_t es, size_t block_elems,
                   int inverse)
{
    const uint8_t *in = (const uint8_t *)vin;
    uint8_t *out = (uint8_t *)vout;
    if (!(es == 1 || es == 2 || es == 4 || es == 8)) return -1;
    size_t B = default_block(es, block_elems);
    if (B % 8 != 0) return -1;
    size_t done = 0;
    while (done < n) {
        size_t Bb = n - done >= B ? B : (n - done) - (n - done) % 8;
        if (Bb == 0) break;
        if (inverse) untranspose_block(in + done * es, out + done * es, Bb, es);
        else transpose_block(in + done * es, out + done * es, Bb, es);
        done += Bb;
    }
    memcpy(out + done * es, in + done * es, (n - done) * es);   /* R9 tail */
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1: LZ4 block codec (LZ77 class: literals + (offset, length) pairs) */
/* ------------------------------------------------------------------------ */

#define LZ4_MINMATCH 4
#define LZ4_LASTLITERALS 5    /* the last 5 bytes of a block are literals */
#define LZ4_MFLIMIT 12        /* a match starts at least 12 bytes before the end */

size_t orc_lz4_bound(size_t n) { return n + n / 255 + 16; }

static size_t put_len(uint8_t *op, size_t v)
{
    size_t w = 0;
    while (v >= 255) { op[w++] = 255; v -= 255; }
    op[w++] = (uint8_t)v;
    return w;
}

static uint32_t read32le(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
           ((uint32_t)p[3] << 24);
}

/* Greedy LZ4 encoder: a 4096-entry table of the last position of each 4-byte
 * hash, every position probed (step 1), the first verified match taken and
 * extended forward.  Returns the compressed size, or 0 if cap is too small. */
size_t orc_lz4_compress_block(const uint8_t *src, size_t n, uint8_t *dst, size_t cap)
{
    int32_t table[4096];
    for (int h = 0; h < 4096; h++) table[h] = -1;
    size_t anchor = 0, i = 0, o = 0;
    if (cap < orc_lz4_bound(n)) return 0;
    if (n >= LZ4_MFLIMIT + 1) {
        while (i + LZ4_MFLIMIT <= n) {
            uint32_t w = read32le(src + i);
            uint32_t h = (w * 2654435761u) >> 20;
            int32_t c = table[h];
            table[h] = (int32_t)i;
            if (c >= 0 && i - (size_t)c <= 65535 && read32le(src + c) == w) {
                size_t L = LZ4_MINMATCH;
                while (i + L < n - LZ4_LASTLITERALS && src[c + L] == src[i + L]) L++;
                size_t LL = i - anchor, ML = L - LZ4_MINMATCH;
                uint8_t *tok = dst + o++;
                *tok = (uint8_t)(((LL < 15 ? LL : 15) << 4) | (ML < 15 ? ML : 15));
                if (LL >= 15) o += put_len(dst + o, LL - 15);
                memcpy(dst + o, src + anchor, LL);
                o += LL;
                size_t off = i - (size_t)c;
                dst[o++] = (uint8_t)(off & 255);
                dst[o++] = (uint8_t)(off >> 8);
                if (ML >= 15) o += put_len(dst + o, ML - 15);
                i += L;
                anchor = i;
            } else {
                i++;
            }
        }
    }
    size_t LL = n - anchor;
    dst[o++] = (uint8_t)((LL < 15 ? LL : 15) << 4);
    if (LL >= 15) o += put_len(dst + o, LL - 15);
    memcpy(dst + o, src + anchor, LL);
    o += LL;
    return o;
}

/* Strict LZ4 block decoder.  Returns 0 when src decodes to exactly dst_len
 * bytes; a negative code otherwise:
 *   -1 input ended early       -2 literal run overruns the output
 *   -3 offset 0                -4 offset reaches before the block start
 *   -5 match overruns output   -6 output shorter than expected
 *   -7 a match breaks the end-of-block rules (starts later than 12 bytes
 *      before the end, or ends inside the last 5 bytes)                    */
int orc_lz4_decompress_block(const uint8_t *src, size_t src_len, uint8_t *dst, size_t dst_len)
{
    size_t ip = 0, op = 0;
    for (;;) {
        if (ip >= src_len) return -1;
        unsigned token = src[ip++];
        size_t LL = token >> 4;
        if (LL == 15) {
            unsigned b;
            do {
                if (ip >= src_len) return -1;
                b = src[ip++];
                LL += b;
            } while (b == 255);
        }
        if (LL > src_len - ip) return -1;
        if (LL > dst_len - op) return -2;
        memcpy(dst + op, src + ip, LL);
        ip += LL;
        op += LL;
        if (ip == src_len) break;              /* last sequence: literals only */
        if (src_len - ip < 2) return -1;
        size_t off = (size_t)src[ip] | ((size_t)src[ip + 1] << 8);
        ip += 2;
        if (off == 0) return -3;
        if (off > op) return -4;
        size_t ML = token & 15u;
        if (ML == 15) {
            unsigned b;
            do {
                if (ip >= src_len) return -1;
                b = src[ip++];
                ML += b;
            } while (b == 255);
        }
        ML += LZ4_MINMATCH;
        if (ML > dst_len - op) return -5;
        if (op + LZ4_MFLIMIT > dst_len || op + ML + LZ4_LASTLITERALS > dst_len) return -7;
        for (size_t k = 0; k < ML; k++) dst[op + k] = dst[op + k - off];   /* overlap = RLE */
        op += ML;
    }
    return op == dst_len ? 0 : -6;
}

/* ------------------------------------------------------------------------ */
/* Bitshuffle + LZ4 per block with the framing of reading R11                */
/* ------------------------------------------------------------------------ */

static void put_be64(uint8_t *p, uint64_t v) { for (int k = 7; k >= 0; k--) { p[k] = (uint8_t)v; v >>= 8; } }
static void put_be32(uint8_t *p, uint32_t v) { for (int k = 3; k >= 0; k--) { p[k] = (uint8_t)v; v >>= 8; } }
static uint64_t get_be64(const uint8_t *p) { uint64_t v = 0; for (int k = 0; k < 8; k++) v = (v << 8) | p[k]; return v; }
static uint32_t get_be32(const uint8_t *p) { uint32_t v = 0; for (int k = 0; k < 4; k++) v = (v << 8) | p[k]; return v; }

size_t orc_compress_bound(size_t n, size_t es, size_t block_elems)
{
    size_t B = default_block(es, block_elems);
    size_t nb = n / B, rem = n % B, last = rem - rem % 8;
    size_t bound = 12 + nb * (4 + orc_lz4_bound(B * es));
    if (last) bound += 4 + orc_lz4_bound(last * es);
    return bound + (rem % 8) * es;
}

/* Returns the compressed size, or 0 on a bad argument / small capacity.
 * block_sizes (may be NULL) receives the compressed length of every block. */
size_t orc_compress(const void *vin, size_t n, size_t es, size_t block_elems,
                    void *vout, size_t cap, uint32_t *block_sizes)
{
    const uint8_t *in = (const uint8_t *)vin;
    uint8_t *out = (uint8_t *)vout;
    if (!(es == 1 || es == 2 || es == 4 || es == 8)) return 0;
    size_t B = default_block(es, block_elems);
    if (B % 8 != 0 || B * es > 65536) return 0;
    if (cap < orc_compress_bound(n, es, block_elems)) return 0;
    put_be64(out, (uint64_t)(n * es));
    put_be32(out + 8, (uint32_t)(B * es));
    size_t o = 12, done = 0, b = 0;
    uint8_t shuf[65536];
    while (done < n) {
        size_t Bb = n - done >= B ? B : (n - done) - (n - done) % 8;
        if (Bb == 0) break;
        transpose_block(in + done * es, shuf, Bb, es);
        size_t c = orc_lz4_compress_block(shuf, Bb * es, out + o + 4, orc_lz4_bound(Bb * es));
        put_be32(out + o, (uint32_t)c);
        if (block_sizes) block_sizes[b] = (uint32_t)c;
        o += 4 + c;
        done += Bb;
        b++;
    }
    memcpy(out + o, in + done * es, (n - done) * es);
    return o + (n - done) * es;
}

/* Returns 0 on success, or a negative code: -10 bad argument, -11 header does
 * not match (n, es, block size), -12 stream truncated, -13 trailing bytes,
 * or the block decoder's code. */
int orc_decompress(const void *vin, size_t in_len, void *vout, size_t n, size_t es,
                   size_t block_elems)
{
    const uint8_t *in = (const uint8_t *)vin;
    uint8_t *out = (uint8_t *)vout;
    if (!(es == 1 || es == 2 || es == 4 || es == 8)) return -10;
    size_t B = default_block(es, block_elems);
    if (B % 8 != 0 || B * es > 65536) return -10;
    if (in_len < 12) return -12;
    if (get_be64(in) != (uint64_t)(n * es) || get_be32(in + 8) != (uint32_t)(B * es)) return -11;
    size_t ip = 12, done = 0;
    uint8_t shuf[65536];
    while (done < n) {
        size_t Bb = n - done >= B ? B : (n - done) - (n - done) % 8;
        if (Bb == 0) break;
        if (in_len - ip < 4) return -12;
        size_t c = get_be32(in + ip);
        ip += 4;
        if (c > in_len - ip) return -12;
        int rc = orc_lz4_decompress_block(in + ip, c, shuf, Bb * es);
        if (rc) return rc;
        untranspose_block(shuf, out + done * es, Bb, es);
        ip += c;
        done += Bb;
    }
    size_t tail = (n - done) * es;
    if (in_len - ip < tail) return -12;
    memcpy(out + done * es, in + ip, tail);
    if (ip + tail != in_len) return -13;
    return 0;
}
