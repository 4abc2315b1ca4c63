/*
 * dmas_oracle.c -- plain FP64 CPU oracle for n-th order Delay-Multiply-and-Sum
 * (DMAS) beamforming with Coherence Factor (CF) weighting and envelope detection.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to prove the CUDA path right.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant with the CUDA library
 * and includes nothing from it.
 *
 * Everything is double precision, written as plainly as the method allows:
 *
 *   directions   u(theta, phi) = (sin th cos ph, sin ph, cos th cos ph)
 *                (array in the z = 0 plane, broadside +z; Fig. 1 coordinate
 *                system, azimuth theta, elevation phi)
 *   delays       tau_{i,psi} = -((p_i - p_bar) . u_psi) / c  (Sec. II, the
 *                delay look-up table; far-field plane wave, centroid reference)
 *   pre-steering x_i(t, psi) = m_i(t + tau_{i,psi})          (Eq. signal_delay)
 *                ROUND: nearest sample, llround(tau * fs); LINEAR: every
 *                stored channel is linearly interpolated; samples outside the
 *                frame are zero.
 *   roots        s_i = sgn(x_i) |x_i|^(1/n), sgn(0) = 0        (Sec. II-B)
 *   DMAS         E_n(s_1..s_N), the n-th elementary symmetric polynomial
 *                (Eq. dmasn, Eq. dmas_as_En).  ROUND mode evaluates it as the
 *                coefficient of z^n in prod_i (1 + s_i z), which is the subset
 *                sum of Eq. dmasn expanded one factor at a time (no
 *                Newton-Girard cancellation).  LINEAR mode has no single value
 *                per microphone (each power channel is interpolated on its
 *                own), so there E_n is defined by the Newton-Girard partition
 *                formula (Eq. girard_newton_general) over the interpolated
 *                power sums P_k (Eq. power_sum).
 *   CF           (sum x_i)^2 / (N sum x_i^2 + eps)              (Eq. cf)
 *   weighting    y = E_n * CF (or E_n with CF off)             (Sec. II-D)
 *   envelope     |y| low-pass filtered along t: a zero-phase windowed-sinc
 *                FIR (Hamming window), zero padded at the frame ends
 *                (Sec. II step 3; 5 kHz cutoff in Sec. III-B).
 *   matched      optional, before everything above (Sec. II step 1): each
 *   filter       microphone signal correlated with the emitted signal e,
 *                mf_i(t) = sum_{k=0}^{L-1} e[k] m_i(t + k), m = 0 outside the
 *                frame, so an echo arriving at t0 peaks at t0.
 *
 * Compile: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_ORDER 16

/* ------------------------------------------------------------------------- */
/* threads                                                                    */
/* ------------------------------------------------------------------------- */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* geometry: unit vectors and the delay look-up table (Sec. II)               */
/* ------------------------------------------------------------------------- */

/* azel: [M][2] radians (azimuth theta, elevation phi) -> u: [M][3]. */
void oracle_unit_vectors(int M, const double *azel, double *u)
{
    for (int k = 0; k < M; ++k) {
        double th = azel[2 * k + 0];
        double ph = azel[2 * k + 1];
        u[3 * k + 0] = sin(th) * cos(ph);
        u[3 * k + 1] = sin(ph);
        u[3 * k + 2] = cos(th) * cos(ph);
    }
}

/* tau[M][N] seconds.  The centroid is the plain mean of the positions, summed
 * in microphone order; the projection is evaluated x, then y, then z. */
void oracle_geometric_delays(int N, const double *xyz, int M, const double *u,
                             double c, double *tau)
{
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int i = 0; i < N; ++i) {
        cx += xyz[3 * i + 0];
        cy += xyz[3 * i + 1];
        cz += xyz[3 * i + 2];
    }
    cx /= (double)N;
    cy /= (double)N;
    cz /= (double)N;
    for (int k = 0; k < M; ++k) {
        for (int i = 0; i < N; ++i) {
            double dx = xyz[3 * i + 0] - cx;
            double dy = xyz[3 * i + 1] - cy;
            double dz = xyz[3 * i + 2] - cz;
            double proj = dx * u[3 * k + 0];
            proj = proj + dy * u[3 * k + 1];
            proj = proj + dz * u[3 * k + 2];
            tau[(size_t)k * N + i] = -proj / c;
        }
    }
}

/* Nearest-sample shift of one delay: round half away from zero. */
long long oracle_round_shift(double tau, double fs)
{
    double delta = tau * fs;
    return llround(delta);
}

/* ------------------------------------------------------------------------- */
/* elementary symmetric polynomials                                           */
/* ------------------------------------------------------------------------- */

/* E_n of r[0..N-1]: coefficient of z^n in prod (1 + r_i z).  e[0] = 1 and each
 * factor (1 + r_i z) multiplies the running polynomial, highest degree first so
 * that e[k-1] still holds the previous factor's value. */
double oracle_esym_product(int N, const double *r, int n)
{
    double e[ORACLE_MAX_ORDER + 1];
    if (n < 0 || n > ORACLE_MAX_ORDER) return NAN;
    for (int k = 0; k <= n; ++k) e[k] = 0.0;
    e[0] = 1.0;
    for (int i = 0; i < N; ++i)
        for (int k = n; k >= 1; --k) e[k] += r[i] * e[k - 1];
    return e[n];
}

/* Eq. girard_newton_general: E_n as a sum over the integer partitions of n,
 * written as multiplicities k_1..k_n with k_1 + 2 k_2 + ... + n k_n = n:
 *     sign = (-1)^(n - sum k_i),  term = prod_i P_i^{k_i} / (k_i! i^{k_i}).
 * P[1..n] are the power sums (P[0] unused).  Partitions are enumerated
 * recursively, part size `i` from n down to 1, with `rest` still to place. */
static double ng_partitions(int n, const double *P, int i, int rest, int nparts,
                            double prod)
{
    if (rest == 0) {
        int sgn_exp = n - nparts;
        return (sgn_exp % 2 == 0) ? prod : -prod;
    }
    if (i == 0) return 0.0;
    double total = 0.0;
    /* choose multiplicity k of part size i */
    double factor = 1.0;  /* P_i^k / (k! i^k), built up for k = 0, 1, ... */
    for (int k = 0; k * i <= rest; ++k) {
        if (k > 0) factor = factor * P[i] / ((double)k * (double)i);
        total += ng_partitions(n, P, i - 1, rest - k * i, nparts + k, prod * factor);
    }
    return total;
}

double oracle_esym_newton_girard(int n, const double *P)
{
    if (n < 0 || n > ORACLE_MAX_ORDER) return NAN;
    if (n == 0) return 1.0;
    return ng_partitions(n, P, n, n, 0, 1.0);
}

/* Same formula, long double, for spot checks of the FP64 evaluation. */
static long double ng_partitions_ld(int n, const long double *P, int i, int rest,
                                    int nparts, long double prod)
{
    if (rest == 0) return ((n - nparts) % 2 == 0) ? prod : -prod;
    if (i == 0) return 0.0L;
    long double total = 0.0L, factor = 1.0L;
    for (int k = 0; k * i <= rest; ++k) {
        if (k > 0) factor = factor * P[i] / ((long double)k * (long double)i);
        total += ng_partitions_ld(n, P, i - 1, rest - k * i, nparts + k, prod * factor);
    }
    return total;
}

/* ------------------------------------------------------------------------- */
/* signed n-th root (Sec. II-B)                                               */
/* ------------------------------------------------------------------------- */
double oracle_signed_root(double x, int n)
{
    if (x > 0.0) return pow(x, 1.0 / (double)n);
    if (x < 0.0) return -pow(-x, 1.0 / (double)n);
    return 0.0;
}

/* ------------------------------------------------------------------------- */
/* envelope low-pass                                                          */
/* ------------------------------------------------------------------------- */

/* Default length: 2 * ceil(fs / fc) + 1 taps. */
int oracle_fir_length(double fs, double fc)
{
    return 2 * (int)ceil(fs / fc) + 1;
}

/* Windowed-sinc low-pass, Hamming window, L odd, H = (L-1)/2, normalised to a
 * unit DC gain:  h[k] = w[k] sin(2 pi fc k / fs) / (pi k), h[0] = 2 fc / fs,
 * w[k] = 0.54 + 0.46 cos(pi k / H), stored as h[k + H] for k = -H..H. */
int oracle_fir_taps(double fs, double fc, int L, double *h)
{
    if (L < 1 || (L % 2) == 0) return -1;
    int H = (L - 1) / 2;
    double sum = 0.0;
    for (int k = -H; k <= H; ++k) {
        double ideal;
        if (k == 0) ideal = 2.0 * fc / fs;
        else ideal = sin(2.0 * M_PI * fc * (double)k / fs) / (M_PI * (double)k);
        double w = (H == 0) ? 1.0 : 0.54 + 0.46 * cos(M_PI * (double)k / (double)H);
        h[k + H] = w * ideal;
        sum += h[k + H];
    }
    for (int k = 0; k < L; ++k) h[k] /= sum;
    return 0;
}

/* env[t] = sum_{k=-H..H} h[k] |y[t-k]|, |y| taken as zero outside [0, T). */
void oracle_envelope(int T, const double *y, int L, const double *h, double *env)
{
    int H = (L - 1) / 2;
    for (int t = 0; t < T; ++t) {
        double acc = 0.0;
        for (int k = -H; k <= H; ++k) {
            int s = t - k;
            if (s < 0 || s >= T) continue;
            acc += h[k + H] * fabs(y[s]);
        }
        env[t] = acc;
    }
}

/* mf[i][t] = sum_{k=0}^{L-1} e[k] frame[i][t + k], frame taken as zero past T. */
void oracle_matched_filter(int N, int T, const double *frame, int L, const double *e,
                           double *mf)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        const double *m = frame + (size_t)i * T;
        for (int t = 0; t < T; ++t) {
            double acc = 0.0;
            for (int k = 0; k < L && t + k < T; ++k) acc += e[k] * m[t + k];
            mf[(size_t)i * T + t] = acc;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* the beamformer                                                             */
/* ------------------------------------------------------------------------- */

/*
 * frame : [N][T] microphone samples m_i(t)
 * tau   : [M][N] delays in seconds (from oracle_geometric_delays or explicit)
 * order : n >= 1
 * delay_mode : 0 = nearest sample (ROUND), 1 = linear interpolation (LINEAR)
 * use_cf, cf_eps : CF weighting on/off and the denominator's small constant
 * L, taps : envelope FIR (taps == NULL or L == 0: no envelope, img = |y| is not
 *           formed and img_out is left untouched)
 * dir_begin, dir_end : directions [dir_begin, dir_end) are computed; output row
 *           psi is stored at (psi - dir_begin) * T.
 * y_out, cf_out, img_out : [dir_end - dir_begin][T] or NULL.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_dmas(int N, int T, const double *frame, int M, const double *tau,
                double fs, int order, int delay_mode, int use_cf, double cf_eps,
                int L, const double *taps, int dir_begin, int dir_end,
                double *y_out, double *cf_out, double *img_out)
{
    if (N < 1 || T < 1 || M < 1 || order < 1 || order > ORACLE_MAX_ORDER) return -1;
    if (dir_begin < 0 || dir_end > M || dir_begin > dir_end) return -1;
    if (delay_mode != 0 && delay_mode != 1) return -1;
    if (taps != NULL && (L < 1 || L % 2 == 0)) return -1;
    const int n = order;
    const int C = n + 2; /* channels per microphone: r^1..r^n, m, m^2 */

    /* Per-microphone channels.  The root of a delayed sample is the root of the
     * raw sample it points at, so roots (and their powers) are taken once per
     * raw sample.  ch[(i*C + c)*T + t]. */
    double *ch = (double *)malloc(sizeof(double) * (size_t)N * C * T);
    if (!ch) return -1;
    for (int i = 0; i < N; ++i) {
        for (int t = 0; t < T; ++t) {
            double m = frame[(size_t)i * T + t];
            double r = oracle_signed_root(m, n);
            double rk = 1.0;
            for (int k = 1; k <= n; ++k) {
                rk *= r;
                ch[((size_t)i * C + (k - 1)) * T + t] = rk;
            }
            ch[((size_t)i * C + n) * T + t] = m;
            ch[((size_t)i * C + n + 1) * T + t] = m * m;
        }
    }
    int err = 0;

#pragma omp parallel for schedule(dynamic, 1)
    for (int psi = dir_begin; psi < dir_end; ++psi) {
        double *y = (double *)malloc(sizeof(double) * (size_t)T);
        double *cfr = (double *)malloc(sizeof(double) * (size_t)T);
        double *rr = (double *)malloc(sizeof(double) * (size_t)N);
        long long *sh = (long long *)malloc(sizeof(long long) * (size_t)N);
        double *fr = (double *)malloc(sizeof(double) * (size_t)N);
        if (!y || !cfr || !rr || !sh || !fr) {
#pragma omp atomic write
            err = 1;
            free(y); free(cfr); free(rr); free(sh); free(fr);
            continue;
        }
        for (int i = 0; i < N; ++i) {
            double delta = tau[(size_t)psi * N + i] * fs;
            if (delay_mode == 0) {
                sh[i] = llround(delta);
                fr[i] = 0.0;
            } else {
                double j = floor(delta);
                sh[i] = (long long)j;
                fr[i] = delta - j;
            }
        }
        for (int t = 0; t < T; ++t) {
            double A = 0.0, B = 0.0, E;
            if (delay_mode == 0) {
                for (int i = 0; i < N; ++i) {
                    long long s = (long long)t + sh[i];
                    double x = 0.0, r = 0.0;
                    if (s >= 0 && s < T) {
                        x = ch[((size_t)i * C + n) * T + s];
                        r = ch[((size_t)i * C + 0) * T + s];
                    }
                    rr[i] = r;
                    A += x;
                    B += x * x;
                }
                E = oracle_esym_product(N, rr, n);
            } else {
                double P[ORACLE_MAX_ORDER + 1];
                for (int k = 0; k <= n; ++k) P[k] = 0.0;
                for (int i = 0; i < N; ++i) {
                    long long s0 = (long long)t + sh[i], s1 = s0 + 1;
                    double f = fr[i];
                    for (int c = 0; c < C; ++c) {
                        const double *row = ch + ((size_t)i * C + c) * T;
                        double v0 = (s0 >= 0 && s0 < T) ? row[s0] : 0.0;
                        double v1 = (s1 >= 0 && s1 < T) ? row[s1] : 0.0;
                        double v = (1.0 - f) * v0 + f * v1;
                        if (c < n) P[c + 1] += v;
                        else if (c == n) A += v;
                        else B += v;
                    }
                }
                E = oracle_esym_newton_girard(n, P);
            }
            double cf = (A * A) / ((double)N * B + cf_eps);
            cfr[t] = cf;
            y[t] = use_cf ? E * cf : E;
        }
        size_t row = (size_t)(psi - dir_begin) * T;
        if (y_out) memcpy(y_out + row, y, sizeof(double) * (size_t)T);
        if (cf_out) memcpy(cf_out + row, cfr, sizeof(double) * (size_t)T);
        if (img_out && taps) oracle_envelope(T, y, L, taps, img_out + row);
        free(y); free(cfr); free(rr); free(sh); free(fr);
    }
    free(ch);
    return err ? -1 : 0;
}

/* Long-double recomputation of one LINEAR-mode pixel's E_n (spot checks of the
 * FP64 evaluation's own rounding).  Same arguments as oracle_dmas for one
 * (psi, t); returns E_n. */
double oracle_linear_esym_ld(int N, int T, const double *frame, const double *tau_row,
                             double fs, int order, int t)
{
    const int n = order;
    long double P[ORACLE_MAX_ORDER + 1];
    if (n < 1 || n > ORACLE_MAX_ORDER) return NAN;
    for (int k = 0; k <= n; ++k) P[k] = 0.0L;
    for (int i = 0; i < N; ++i) {
        double delta = tau_row[i] * fs;
        double j = floor(delta);
        long double f = (long double)(delta - j);
        long long s0 = (long long)t + (long long)j;
        for (int w = 0; w < 2; ++w) {
            long long s = s0 + w;
            long double weight = (w == 0) ? (1.0L - f) : f;
            if (s < 0 || s >= T) continue;
            long double m = (long double)frame[(size_t)i * T + s];
            long double r = 0.0L;
            if (m > 0) r = powl(m, 1.0L / (long double)n);
            else if (m < 0) r = -powl(-m, 1.0L / (long double)n);
            long double rk = 1.0L;
            for (int k = 1; k <= n; ++k) {
                rk *= r;
                P[k] += weight * rk;
            }
        }
    }
    return (double)ng_partitions_ld(n, P, n, n, 0, 1.0L);
}
