/*
 * oracle.c -- plain, slow CPU oracle for brute-force incoherent dedispersion
 * and the boxcar single-pulse search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no source with the CUDA library.
 *
 * Every function writes out a definition directly, in the order the method
 * states it, with no blocking, fusion or reordering:
 *   - delay table:       dispersion delay law, Ch.1 Eq.1 (constant
 *                        4148.808 s MHz^2, i.e. 4.14881 ms GHz^2), rounded to
 *                        the nearest sample with ties away from zero;
 *   - dedispersion:      brute-force shift-and-sum over channels, Sec.3.2
 *                        ("brute-force dedispersion is O(m x N)");
 *   - window statistics: median and median absolute deviation, Sec.3.3
 *                        (median preferred for robustness to outliers);
 *   - boxcar S/N search: time-domain boxcar filtering above a user threshold,
 *                        Sec.2.1;
 *   - peaks filtering and clustering of the candidates: square DM-time
 *                        stencils, then DBSCAN in the DM-time plane keeping
 *                        the strongest candidate of each cluster, Sec.2.1;
 *   - downsampling of a dedispersed series by a user factor (Sec.3.2) and
 *                        running-median de-reddening (Sec.3.3);
 *   - the folding transform of a series by the fast folding algorithm and
 *                        the boxcar search of its folded profiles, Sec.3.5;
 *   - resampling for the frequency derivatives f1, f2, Sec.3.4;
 *   - gptool-style RFI mitigation of 8-bit spectra (bandpass, channel and
 *                        time flags), Sec.2.1.
 * Readings where the paper is silent (channel frequencies, output length,
 * boxcar alignment, window layout, even-count median, MAD = 0) are listed at
 * each function.
 *
 * Floating point is IEEE double; build with -ffp-contract=off so no fused
 * multiply-add changes the rounding of the delay expression.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_K_DISP 4148.808          /* s MHz^2 per (pc cm^-3), Ch.1 Eq.1 */
#define ORC_MAD_TO_SIGMA 1.482602218505602

/* ------------------------------------------------------------------------ */
/* Delay table (Ch.1 Eq.1).                                                 */
/* Reading: channel c is centred at f_c = f_top + c*chan_bw (first channel   */
/* at f_top); the reference frequency f_ref is the highest channel          */
/* frequency, so every delay is >= 0 for DM >= 0.                            */
/* d[k][c] = round_half_away(K * DM_k * (f_c^-2 - f_ref^-2) / tsamp).        */
/* Returns the largest delay D, or -1 on a bad argument.                    */
/* ------------------------------------------------------------------------ */
int32_t orc_delay_table(int nchan, double f_top, double chan_bw, double tsamp,
                        const double *dm, int ndm, int32_t *d)
{
    if (nchan <= 0 || ndm <= 0 || !(tsamp > 0.0) || chan_bw == 0.0) return -1;
    double f_last = f_top + (double)(nchan - 1) * chan_bw;
    double fr = f_top > f_last ? f_top : f_last;
    int32_t dmax = 0;
    for (int k = 0; k < ndm; ++k) {
        if (!(dm[k] >= 0.0) || !isfinite(dm[k])) return -1;
        for (int c = 0; c < nchan; ++c) {
            double f = f_top + c * chan_bw;
            double x = ORC_K_DISP * dm[k] * (1.0 / (f * f) - 1.0 / (fr * fr)) / tsamp;
            double r = round(x);               /* C round(): half away from zero */
            if (r > 2147483647.0) return -1;
            d[(int64_t)k * nchan + c] = (int32_t)r;
            if ((int32_t)r > dmax) dmax = (int32_t)r;
        }
    }
    return dmax;
}

/* Unrounded delay x = K*DM*(f^-2 - f_ref^-2)/tsamp, so a test can list the  */
/* entries that sit within a hair of a .5 tie.                               */
double orc_delay_exact(int nchan, double f_top, double chan_bw, double tsamp,
                       double dm, int c)
{
    double f_last = f_top + (double)(nchan - 1) * chan_bw;
    double fr = f_top > f_last ? f_top : f_last;
    double f = f_top + c * chan_bw;
    return ORC_K_DISP * dm * (1.0 / (f * f) - 1.0 / (fr * fr)) / tsamp;
}

/* ------------------------------------------------------------------------ */
/* Unpack: time-major spectra [nin][nchan] (the layout of a block of         */
/* spectra, Sec.2.2) to channel-major rows [nchan][nin].  A plain transpose. */
/* ------------------------------------------------------------------------ */
void orc_unpack_u8(const uint8_t *in, int64_t nin, int nchan, uint8_t *out)
{
    for (int c = 0; c < nchan; ++c)
        for (int64_t s = 0; s < nin; ++s)
            out[(int64_t)c * nin + s] = in[s * nchan + c];
}

void orc_unpack_u16(const uint16_t *in, int64_t nin, int nchan, uint16_t *out)
{
    for (int c = 0; c < nchan; ++c)
        for (int64_t s = 0; s < nin; ++s)
            out[(int64_t)c * nin + s] = in[s * nchan + c];
}

/* ------------------------------------------------------------------------ */
/* Brute-force dedispersion (Sec.3.2).                                       */
/* out[k][t] = sum_c in[t + d[k][c]][c], t in [0, nout), nout = nin - D.      */
/* The input is read in its time-major layout in[sample][chan].  Sums are    */
/* accumulated in int64 and must fit int32 (they do: 4096*65535 < 2^31).     */
/* The loop over DM trials may run on several cores (each trial is           */
/* independent); the arithmetic is the same triple loop either way.          */
/* ------------------------------------------------------------------------ */
static int64_t sample_at(const void *in, int nbits, int nchan, int64_t s, int c)
{
    if (nbits == 8) return ((const uint8_t *)in)[s * nchan + c];
    return ((const uint16_t *)in)[s * nchan + c];
}

int orc_dedisperse(const void *in, int nbits, int64_t nin, int nchan,
                   const int32_t *d, int ndm, int64_t nout, int32_t *out)
{
    if (nbits != 8 && nbits != 16) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int k = 0; k < ndm; ++k) {
        const int32_t *dk = d + (int64_t)k * nchan;
        for (int64_t t = 0; t < nout; ++t) {
            int64_t acc = 0;
            for (int c = 0; c < nchan; ++c) {
                int64_t s = t + dk[c];
                if (s < 0 || s >= nin) { bad = 1; continue; }
                acc += sample_at(in, nbits, nchan, s, c);
            }
            if (acc > INT32_MAX) bad = 1;
            out[(int64_t)k * nout + t] = (int32_t)acc;
        }
    }
    return bad ? -1 : 0;
}

/* One output sample out[k][t], for sampled checks at sizes where the full   */
/* triple loop would take too long.  Same definition as above.               */
int64_t orc_dedisperse_at(const void *in, int nbits, int64_t nin, int nchan,
                          const int32_t *dk, int64_t t)
{
    int64_t acc = 0;
    for (int c = 0; c < nchan; ++c) {
        int64_t s = t + dk[c];
        if (s < 0 || s >= nin) return INT64_MIN;
        acc += sample_at(in, nbits, nchan, s, c);
    }
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Window statistics (Sec.3.3: median-based noise estimate; MAD as the       */
/* robust spread).                                                           */
/* Readings: windows j = [jL, (j+1)L) for j < nwin-1 with                    */
/* nwin = max(1, floor(n/L)); the last window runs to n.  L = 0 means one    */
/* window over the whole series.  Median of an even count = mean of the two  */
/* middle order statistics, kept exact as m2 = 2*median.  MAD = median of    */
/* |x - median|, kept exact as mad4 = 4*MAD (u_i = |2x_i - m2|,              */
/* mad4 = 2*median(u)).  The order statistics come from a full sort (qsort). */
/* ------------------------------------------------------------------------ */
static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_num_windows(int64_t n, int64_t L)
{
    if (L <= 0) return 1;
    int64_t w = n / L;
    return w < 1 ? 1 : w;
}

void orc_window_bounds(int64_t n, int64_t L, int64_t j, int64_t *lo, int64_t *hi)
{
    int64_t nwin = orc_num_windows(n, L);
    if (L <= 0) { *lo = 0; *hi = n; return; }
    *lo = j * L;
    *hi = (j == nwin - 1) ? n : (j + 1) * L;
}

/* m2 = 2*median and mad4 = 4*MAD of x[0..n). */
void orc_median_mad(const int32_t *x, int64_t n, int64_t *m2, int64_t *mad4)
{
    int64_t *v = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) v[i] = x[i];
    qsort(v, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t med2 = (n & 1) ? 2 * v[n / 2] : v[n / 2 - 1] + v[n / 2];
    for (int64_t i = 0; i < n; ++i) {
        int64_t u = 2 * (int64_t)x[i] - med2;
        v[i] = u < 0 ? -u : u;
    }
    qsort(v, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t umed2 = (n & 1) ? 2 * v[n / 2] : v[n / 2 - 1] + v[n / 2];
    free(v);
    *m2 = med2;
    *mad4 = umed2;
}

void orc_window_stats(const int32_t *x, int64_t n, int64_t L,
                      int64_t *m2, int64_t *mad4)
{
    int64_t nwin = orc_num_windows(n, L);
    for (int64_t j = 0; j < nwin; ++j) {
        int64_t lo, hi;
        orc_window_bounds(n, L, j, &lo, &hi);
        orc_median_mad(x + lo, hi - lo, &m2[j], &mad4[j]);
    }
}

/* ------------------------------------------------------------------------ */
/* Boxcar (Sec.2.1).  Reading: left-aligned windows, B_w(t) = sum_{i<w}      */
/* x[t+i], defined for t <= n - w only.  Direct summation in int64.          */
/* Returns -1 if a sum leaves int32.                                         */
/* ------------------------------------------------------------------------ */
int orc_boxcar(const int32_t *x, int64_t n, int w, int64_t *out)
{
    for (int64_t t = 0; t + w <= n; ++t) {
        int64_t acc = 0;
        for (int i = 0; i < w; ++i) acc += x[t + i];
        out[t] = acc;
        if (acc > INT32_MAX || acc < INT32_MIN) return -1;
    }
    return 0;
}

/* S/N of B_w(t) against the statistics of the window holding t:             */
/* snr = (B_w - w*median) / (sigma*sqrt(w)), sigma = 1.4826*MAD, in FP64.     */
/* Reading: MAD = 0 gives S/N = 0 (no candidate from that window).            */
double orc_snr(int64_t B, int w, int64_t m2, int64_t mad4)
{
    if (mad4 == 0) return 0.0;
    double sigma = ORC_MAD_TO_SIGMA * ((double)mad4 / 4.0);
    double num = (double)B - (double)w * ((double)m2 / 2.0);
    return num / (sigma * sqrt((double)w));
}

typedef struct {
    int32_t dm_idx;
    int32_t w_idx;
    int64_t t;
    double snr;
} orc_cand;

static int cmp_cand(const void *a, const void *b)
{
    const orc_cand *x = (const orc_cand *)a, *y = (const orc_cand *)b;
    if (x->dm_idx != y->dm_idx) return (x->dm_idx > y->dm_idx) - (x->dm_idx < y->dm_idx);
    return (x->t > y->t) - (x->t < y->t);
}

/* Best width and S/N at one (series, t): widths scanned in the order given;   */
/* the first width reaching the maximum wins (ties go to the earlier width).  */
/* Only widths with t + w <= n take part.  Returns -1 if none does.           */
int orc_best_at(const int32_t *x, int64_t n, int64_t L, const int *widths,
                int nw, int64_t t, double *snr_out)
{
    int64_t j = (L <= 0) ? 0 : t / L;
    int64_t nwin = orc_num_windows(n, L);
    if (j > nwin - 1) j = nwin - 1;
    int64_t lo, hi, m2, mad4;
    orc_window_bounds(n, L, j, &lo, &hi);
    orc_median_mad(x + lo, hi - lo, &m2, &mad4);
    int best = -1;
    double bsnr = 0.0;
    for (int wi = 0; wi < nw; ++wi) {
        int w = widths[wi];
        if (t + w > n) continue;
        int64_t B = 0;
        for (int i = 0; i < w; ++i) B += x[t + i];
        double s = orc_snr(B, w, m2, mad4);
        if (best < 0 || s > bsnr) { best = wi; bsnr = s; }
    }
    *snr_out = bsnr;
    return best;
}

/* Single-pulse search over series[ndm][n]: per window the statistics, per    */
/* (k, t) the best width, and one candidate per (k, t) whose best S/N is      */
/* >= thr (reading: no peak merging).  Candidates come back sorted by (k, t). */
/* Returns the true count; at most cap records are written.                   */
int64_t orc_sps(const int32_t *series, int ndm, int64_t n, const int *widths,
                int nw, int64_t L, double thr, orc_cand *out, int64_t cap)
{
    int64_t nwin = orc_num_windows(n, L);
    int64_t count = 0;
    int64_t *m2 = (int64_t *)malloc((size_t)nwin * sizeof(int64_t));
    int64_t *mad4 = (int64_t *)malloc((size_t)nwin * sizeof(int64_t));
    for (int k = 0; k < ndm; ++k) {
        const int32_t *x = series + (int64_t)k * n;
        orc_window_stats(x, n, L, m2, mad4);
        for (int64_t t = 0; t < n; ++t) {
            int64_t j = (L <= 0) ? 0 : t / L;
            if (j > nwin - 1) j = nwin - 1;
            int best = -1;
            double bsnr = 0.0;
            for (int wi = 0; wi < nw; ++wi) {
                int w = widths[wi];
                if (t + w > n) continue;
                int64_t B = 0;
                for (int i = 0; i < w; ++i) B += x[t + i];
                double s = orc_snr(B, w, m2[j], mad4[j]);
                if (best < 0 || s > bsnr) { best = wi; bsnr = s; }
            }
            if (best >= 0 && bsnr >= thr) {
                if (count < cap) {
                    out[count].dm_idx = k;
                    out[count].w_idx = best;
                    out[count].t = t;
                    out[count].snr = bsnr;
                }
                ++count;
            }
        }
    }
    free(m2);
    free(mad4);
    int64_t nout = count < cap ? count : cap;
    qsort(out, (size_t)nout, sizeof(orc_cand), cmp_cand);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Peaks filtering (Sec.2.1): redundant candidates of one event are removed   */
/* with square stencils of different sizes in the DM-time plane.              */
/* Reading: the stencil of candidate i is the square |k - k_i| <= h,          */
/* |t - t_i| <= h (trial index and sample units) whose half-size              */
/* h = half[w_i] is set by the candidate's boxcar width; i is kept iff no     */
/* other candidate j inside its square is stronger: s_j > s_i, or s_j == s_i  */
/* and (k_j, t_j) precedes (k_i, t_i).  S/N values are compared exactly as    */
/* given (FP32, the search's output).  The (k, t) pairs must be distinct.     */
/* Direct loop over all other candidates for each decided one; idx lists the  */
/* candidates to decide (NULL: all n, m = n) and keep[q] answers for idx[q].  */
/* Returns -1 on a width index outside [0, nw) or a negative half-size.       */
/* ------------------------------------------------------------------------ */
static int orc_stronger(uint32_t kj, uint32_t tj, float sj, uint32_t ki,
                        uint32_t ti, float si)
{
    if (sj != si) return sj > si;
    return kj < ki || (kj == ki && tj < ti);
}

int orc_peaks(const uint32_t *k, const uint32_t *t, const uint32_t *w,
              const float *s, int64_t n, const int32_t *half, int nw,
              const int64_t *idx, int64_t m, uint8_t *keep)
{
    for (int64_t q = 0; q < m; ++q) {
        int64_t i = idx ? idx[q] : q;
        if (i < 0 || i >= n || w[i] >= (uint32_t)nw || half[w[i]] < 0) return -1;
        int64_t h = half[w[i]];
        int kept = 1;
        for (int64_t j = 0; j < n && kept; ++j) {
            if (j == i) continue;
            int64_t dk = (int64_t)k[j] - (int64_t)k[i];
            int64_t dt = (int64_t)t[j] - (int64_t)t[i];
            if (dk < -h || dk > h || dt < -h || dt > h) continue;
            if (orc_stronger(k[j], t[j], s[j], k[i], t[i], s[i])) kept = 0;
        }
        keep[q] = (uint8_t)kept;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* DBSCAN (density-based clustering, Ester et al. 1996) of the filtered       */
/* candidates in the DM-time plane (the clustering step of Sec.2.1).          */
/* Reading: the neighbourhood of point p is every point q with                */
/* |k_q - k_p| <= eps_dm and |t_q - t_p| <= eps_t, p itself included; p is a  */
/* core point if its neighbourhood holds >= min_pts points.  Points, sorted   */
/* by (k, t), are visited in that order.  An unvisited core point starts a    */
/* new cluster, expanded breadth-first: every point reached that is not yet   */
/* in a cluster joins it, and the neighbourhoods of the core points reached   */
/* are expanded in turn.  Border points therefore keep the first cluster that */
/* reaches them; points no cluster reaches are noise (label -1).  A cluster's */
/* label is the sorted index of the point that started it (its first core     */
/* point).  Region queries are linear scans.                                  */
/* Returns -1 if the points are not sorted by (k, t) and distinct, or if      */
/* eps_dm, eps_t < 0 or min_pts < 1; 0 otherwise.                             */
/* ------------------------------------------------------------------------ */
static int orc_near(const uint32_t *k, const uint32_t *t, int64_t p, int64_t q,
                    int64_t eps_dm, int64_t eps_t)
{
    int64_t dk = (int64_t)k[q] - (int64_t)k[p];
    int64_t dt = (int64_t)t[q] - (int64_t)t[p];
    return dk >= -eps_dm && dk <= eps_dm && dt >= -eps_t && dt <= eps_t;
}

static int64_t orc_region_count(const uint32_t *k, const uint32_t *t, int64_t n,
                                int64_t p, int64_t eps_dm, int64_t eps_t)
{
    int64_t c = 0;
    for (int64_t q = 0; q < n; ++q) c += orc_near(k, t, p, q, eps_dm, eps_t);
    return c;
}

int orc_dbscan(const uint32_t *k, const uint32_t *t, int64_t n, int64_t eps_dm,
               int64_t eps_t, int64_t min_pts, int64_t *label)
{
    const int64_t UNSET = -2, NOISE = -1;
    if (eps_dm < 0 || eps_t < 0 || min_pts < 1 || n < 0) return -1;
    for (int64_t i = 1; i < n; ++i)
        if (k[i] < k[i - 1] || (k[i] == k[i - 1] && t[i] <= t[i - 1])) return -1;
    uint8_t *visited = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *pushed = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *queue = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) { label[i] = UNSET; pushed[i] = -1; }
    for (int64_t p = 0; p < n; ++p) {
        if (visited[p]) continue;
        visited[p] = 1;
        if (orc_region_count(k, t, n, p, eps_dm, eps_t) < min_pts) {
            label[p] = NOISE;            /* may become a border point later */
            continue;
        }
        const int64_t c = p;             /* a new cluster, labelled by p */
        label[p] = c;
        int64_t qh = 0, qt = 0;
        pushed[p] = c;
        for (int64_t q = 0; q < n; ++q)
            if (pushed[q] != c && orc_near(k, t, p, q, eps_dm, eps_t)) {
                pushed[q] = c;
                queue[qt++] = q;
            }
        while (qh < qt) {
            int64_t q = queue[qh++];
            if (label[q] == UNSET || label[q] == NOISE) label[q] = c;
            if (visited[q]) continue;
            visited[q] = 1;
            if (orc_region_count(k, t, n, q, eps_dm, eps_t) < min_pts) continue;
            for (int64_t r = 0; r < n; ++r)
                if (pushed[r] != c && orc_near(k, t, q, r, eps_dm, eps_t)) {
                    pushed[r] = c;
                    queue[qt++] = r;
                }
        }
    }
    for (int64_t i = 0; i < n; ++i)
        if (label[i] == UNSET) label[i] = NOISE;
    free(visited);
    free(pushed);
    free(queue);
    return 0;
}

/* The strongest member of every cluster (Sec.2.1 keeps the highest-S/N       */
/* candidate of each cluster): rep[c] = the point with label c and the        */
/* largest S/N, ties to the smaller sorted index; rep[c] = -1 for every c     */
/* in [0, n) that is not a label.                                             */
void orc_cluster_reps(const int64_t *label, const float *s, int64_t n,
                      int64_t *rep)
{
    for (int64_t c = 0; c < n; ++c) rep[c] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = label[i];
        if (c < 0) continue;
        if (rep[c] < 0 || s[i] > s[rep[c]]) rep[c] = i;
    }
}

/* ------------------------------------------------------------------------ */
/* Downsampling of a dedispersed series by a user factor (Sec.3.2 ends with   */
/* it): y[j] = sum_{i<f} x[j*f + i] for j < floor(n / f); a trailing partial  */
/* group is dropped (reading).  Sums in int64; returns -1 if f < 1 or a sum   */
/* leaves int32, 0 otherwise.                                                 */
/* ------------------------------------------------------------------------ */
int orc_downsample(const int32_t *x, int64_t n, int64_t f, int32_t *y)
{
    if (f < 1 || n < 0) return -1;
    for (int64_t j = 0; j < n / f; ++j) {
        int64_t s = 0;
        for (int64_t i = 0; i < f; ++i) s += x[j * f + i];
        if (s < INT32_MIN || s > INT32_MAX) return -1;
        y[j] = (int32_t)s;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Running-median de-reddening (Sec.3.3): the slowly varying baseline of a    */
/* series is removed by subtracting a running median, z[t] = x[t] - m[t].     */
/* Reading: m[t] is the median of x over the window [t - h, t + h] clamped to */
/* [0, n) (2h + 1 samples away from the ends); windows cut by an end may hold */
/* an even count, and the median taken is then the lower middle order         */
/* statistic, so m[t] is always a sample value and z stays an exact integer.  */
/* Direct selection per output: copy the window, sort it, take element        */
/* (count - 1) / 2.  Returns -1 if h < 0 or a residual leaves int32.          */
/* ------------------------------------------------------------------------ */
static int orc_cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_running_median_at(const int32_t *x, int64_t n, int64_t h,
                              int64_t t, int32_t *work)
{
    int64_t a = t - h < 0 ? 0 : t - h;
    int64_t b = t + h > n - 1 ? n - 1 : t + h;
    int64_t m = b - a + 1;
    memcpy(work, x + a, (size_t)m * sizeof(int32_t));
    qsort(work, (size_t)m, sizeof(int32_t), orc_cmp_i32);
    return work[(m - 1) / 2];
}

int orc_running_median_subtract(const int32_t *x, int64_t n, int64_t h,
                                int32_t *z)
{
    if (h < 0 || n < 0) return -1;
    int64_t wmax = 2 * h + 1 < n ? 2 * h + 1 : n;
    int32_t *work = (int32_t *)malloc((size_t)(wmax > 0 ? wmax : 1) * sizeof(int32_t));
    int rc = 0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t r = (int64_t)x[t] - orc_running_median_at(x, n, h, t, work);
        if (r < INT32_MIN || r > INT32_MAX) { rc = -1; break; }
        z[t] = (int32_t)r;
    }
    free(work);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Folding transform (Sec.3.5): a series cut into m rows of p samples,        */
/* r_i[j] = x[i*p + j], is folded at the trial periods p + s/(m - 1),         */
/* s = 0 .. m - 1 (the paper's p_s = p^2 / (p - s/(m - 1)) to first order),   */
/* by the fast folding algorithm (Staelin 1969).  Reading: m is the largest   */
/* power of two with m*p <= n (whole rows), and the transform of rows         */
/* [i0, i0 + k) is, for k = 1, the row itself, else with A and B the          */
/* transforms of the first and second halves,                                 */
/*   F[s][j] = A[s/2][j] + B[s/2][(j + (s+1)/2) mod p]   (integer division),  */
/* so profile s drifts by s samples over the m - 1 row steps.  Exact int64.   */
/* out is [m][p]; returns m, or -1 if p < 1 or n < p.                         */
/* ------------------------------------------------------------------------ */
static void orc_ffa_rec(const int32_t *x, int64_t p, int64_t i0, int64_t k,
                        int64_t *out, int64_t *tmp)
{
    if (k == 1) {
        for (int64_t j = 0; j < p; ++j) out[j] = x[i0 * p + j];
        return;
    }
    int64_t h = k / 2;
    int64_t *A = tmp, *B = tmp + h * p;
    int64_t *sub = (int64_t *)malloc((size_t)(k * p) * sizeof(int64_t));
    orc_ffa_rec(x, p, i0, h, A, sub);
    orc_ffa_rec(x, p, i0 + h, h, B, sub);
    free(sub);
    for (int64_t s = 0; s < k; ++s) {
        const int64_t *a = A + (s / 2) * p, *b = B + (s / 2) * p;
        int64_t sh = (s + 1) / 2;
        for (int64_t j = 0; j < p; ++j) out[s * p + j] = a[j] + b[(j + sh) % p];
    }
}

int64_t orc_ffa(const int32_t *x, int64_t n, int64_t p, int64_t *out)
{
    if (p < 1 || n < p) return -1;
    int64_t m = 1;
    while (2 * m * p <= n) m *= 2;
    int64_t *tmp = (int64_t *)malloc((size_t)(m * p) * sizeof(int64_t));
    orc_ffa_rec(x, p, 0, m, out, tmp);
    free(tmp);
    return m;
}

/* Boxcar search of one folded profile P[0..p) of m summed rows (Sec.3.5: a   */
/* boxcar filter detects the pulse in the folded profile).  Reading: cyclic   */
/* boxcars B_w(j) = sum_{i<w} P[(j + i) mod p] for the widths w <= p, the     */
/* profile mean mu = sum(P) / p as the baseline, and                          */
/*   S/N_w(j) = (B_w(j) - w mu) / (sigma sqrt(m w)),                          */
/* sigma the noise of one series sample.  Best over (w, j): the largest S/N,  */
/* ties to the smaller width, then the smaller phase.  FP64.                  */
/* Returns the best width index (-1 if no width fits), best S/N and phase.    */
int orc_fold_snr(const int64_t *P, int64_t p, int64_t m, const int *widths,
                 int nw, double sigma, double *best_snr, int64_t *best_phase)
{
    double tot = 0.0;
    int64_t itot = 0;
    for (int64_t j = 0; j < p; ++j) itot += P[j];
    tot = (double)itot;
    int best = -1;
    double bs = 0.0;
    int64_t bj = 0;
    for (int wi = 0; wi < nw; ++wi) {
        int64_t w = widths[wi];
        if (w < 1 || w > p) continue;
        for (int64_t j = 0; j < p; ++j) {
            int64_t B = 0;
            for (int64_t i = 0; i < w; ++i) B += P[(j + i) % p];
            /* (B - w mu) = (p B - w sum) / p, the numerator exact in int64 */
            double num = (double)(p * B - w * itot) / (double)p;
            double snr = num / (sigma * sqrt((double)(m * w)));
            if (best < 0 || snr > bs) { best = wi; bs = snr; bj = j; }
        }
    }
    (void)tot;
    *best_snr = bs;
    *best_phase = bj;
    return best;
}

/* ------------------------------------------------------------------------ */
/* Resampling for a frequency derivative (Sec.3.4).  A signal of frequency    */
/* f = f0 + f1 t + f2 t^2/2 is brought to a constant frequency by resampling  */
/* the series with the Doppler-transformed sampling interval                  */
/*   tau = tau0 (1 + f' t / f0 + f'' t^2 / (2 f0)),                           */
/* where f' = -f1, f'' = -f2 when f1 <= 0.  When f1 > 0 the series is        */
/* reversed, transformed with f0~ = f0 + f1 T + f2 T^2/2, f' = f1 + f2 T and  */
/* f'' = -f2 (T = n tau0 the duration), and reversed back.                    */
/* Reading: output bin k starts at t_k and lasts tau evaluated at its         */
/* nominal time t = k tau0; t_0 = 0 and t_{k+1} = t_k + tau_k, accumulated    */
/* here bin by bin; the bins kept are those ending by T; out[k] sums the      */
/* input bins [i tau0, (i+1) tau0) weighted by their overlap with             */
/* [t_k, t_{k+1}) over tau0 (fractional powers).  FP64 throughout; times in   */
/* units of tau0.  Returns the number of output bins (at most cap), -1 on a   */
/* bad argument (f0 <= 0, n < 1, or an interval <= 0).                        */
/* ------------------------------------------------------------------------ */
int64_t orc_resample(const int32_t *x, int64_t n, double f0, double f1,
                     double f2, double tau0, double *out, int64_t cap)
{
    if (n < 1 || !(f0 > 0.0) || !(tau0 > 0.0)) return -1;
    const double T = (double)n * tau0;
    const int rev = f1 > 0.0;
    double F0 = f0, fp = -f1, fpp = -f2;
    if (rev) {
        F0 = f0 + f1 * T + f2 * T * T / 2.0;
        fp = f1 + f2 * T;
        fpp = -f2;
        if (!(F0 > 0.0)) return -1;
    }
    int64_t k = 0;
    double tk = 0.0;                    /* in units of tau0 */
    while (k < cap) {
        double t = (double)k * tau0;
        double w = 1.0 + fp * t / F0 + fpp * t * t / (2.0 * F0);  /* tau/tau0 */
        if (!(w > 0.0)) return -1;
        double te = tk + w;
        if (te > (double)n) break;
        double acc = 0.0;
        int64_t i0 = (int64_t)floor(tk), i1 = (int64_t)floor(te);
        for (int64_t i = i0; i <= i1 && i < n; ++i) {
            double lo = tk > (double)i ? tk : (double)i;
            double hi = te < (double)(i + 1) ? te : (double)(i + 1);
            if (hi > lo) {
                double xi = rev ? (double)x[n - 1 - i] : (double)x[i];
                acc += xi * (hi - lo);
            }
        }
        out[k] = acc;
        tk = te;
        ++k;
    }
    if (rev) {
        for (int64_t a = 0, b = k - 1; a < b; ++a, --b) {
            double t = out[a];
            out[a] = out[b];
            out[b] = t;
        }
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* RFI mitigation of a block of 8-bit spectra, gptool style (Sec.2.1 and the  */
/* figure of its steps: bandpass from the mean spectrum median-filtered over  */
/* 21 channels, channels beyond 4 sigma of the corrected mean spectrum and    */
/* time samples beyond 3 sigma of the frequency-averaged series flagged,      */
/* both done twice).  Readings, all in exact integer arithmetic:              */
/*   round r: s[c] = sum of x[t][c] over unflagged t; b[c] = lower median of  */
/*   s over channels [c - hw, c + hw] clamped (hw = 10: 21 channels); R =     */
/*   lower median of b over all channels; e[c] = round(s[c] R / b[c]) (0 if  */
/*   b[c] = 0); among unflagged channels, with (m2, mad4) = 2 median and 4    */
/*   MAD of e (orc_median_mad), channel c is flagged when                     */
/*   20000 |2 e[c] - m2| > kc 14826 mad4 (|e - median| > kc 1.4826 MAD) and   */
/*   mad4 > 0; y[t][c] = min(255, round(x[t][c] R / b[c])); u[t] = sum of    */
/*   y[t][c] over unflagged channels; among unflagged t, t is flagged when    */
/*   20000 |2 u[t] - m2| > kt 14826 mad4 with (m2, mad4) of u.  Flags only    */
/*   accumulate.  After the rounds, out = y of the last round, with every     */
/*   flagged channel and time sample set to the fill level                    */
/*   min(255, round(R / T')), T' the unflagged sample count of that round.    */
/* round(a / b) = floor((2a + b) / (2b)) for a >= 0, b > 0.                   */
/* x and out are time-major [nt][nc]; fc[nc], ft[nt] get the flags (0/1).     */
/* Returns 0, or -1 on a bad argument.                                        */
/* ------------------------------------------------------------------------ */
static int orc_cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int64_t orc_round_div(int64_t a, int64_t b)
{
    return (2 * a + b) / (2 * b);
}

/* 2 * median and 4 * MAD of v[0..n) (n >= 1), like orc_median_mad. */
static void orc_median_mad_i64(const int64_t *v, int64_t n, int64_t *m2,
                               int64_t *mad4)
{
    int64_t *w = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    memcpy(w, v, (size_t)n * sizeof(int64_t));
    qsort(w, (size_t)n, sizeof(int64_t), orc_cmp_i64);
    int64_t med2 = w[(n - 1) / 2] + w[n / 2];
    for (int64_t i = 0; i < n; ++i) {
        int64_t d = 2 * v[i] - med2;
        w[i] = d < 0 ? -d : d;
    }
    qsort(w, (size_t)n, sizeof(int64_t), orc_cmp_i64);
    *m2 = med2;
    *mad4 = w[(n - 1) / 2] + w[n / 2];
    free(w);
}

int orc_rfi_clean(const uint8_t *x, int64_t nt, int64_t nc, int hw, int kc,
                  int kt, int rounds, uint8_t *out, uint8_t *fc, uint8_t *ft)
{
    if (nt < 1 || nc < 1 || hw < 0 || kc < 0 || kt < 0 || rounds < 1) return -1;
    int64_t *s = (int64_t *)malloc((size_t)nc * sizeof(int64_t));
    int64_t *b = (int64_t *)malloc((size_t)nc * sizeof(int64_t));
    int64_t *e = (int64_t *)malloc((size_t)nc * sizeof(int64_t));
    int64_t *u = (int64_t *)malloc((size_t)nt * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)(nt > nc ? nt : nc) * sizeof(int64_t));
    int64_t *win = (int64_t *)malloc((size_t)(2 * hw + 1) * sizeof(int64_t));
    memset(fc, 0, (size_t)nc);
    memset(ft, 0, (size_t)nt);
    int64_t R = 0, tkeep = nt;
    for (int r = 0; r < rounds; ++r) {
        tkeep = 0;
        for (int64_t t = 0; t < nt; ++t) tkeep += !ft[t];
        for (int64_t c = 0; c < nc; ++c) {
            int64_t acc = 0;
            for (int64_t t = 0; t < nt; ++t)
                if (!ft[t]) acc += x[t * nc + c];
            s[c] = acc;
        }
        for (int64_t c = 0; c < nc; ++c) {
            int64_t lo = c - hw < 0 ? 0 : c - hw;
            int64_t hi = c + hw > nc - 1 ? nc - 1 : c + hw;
            int64_t m = hi - lo + 1;
            memcpy(win, s + lo, (size_t)m * sizeof(int64_t));
            qsort(win, (size_t)m, sizeof(int64_t), orc_cmp_i64);
            b[c] = win[(m - 1) / 2];
        }
        memcpy(tmp, b, (size_t)nc * sizeof(int64_t));
        qsort(tmp, (size_t)nc, sizeof(int64_t), orc_cmp_i64);
        R = tmp[(nc - 1) / 2];
        for (int64_t c = 0; c < nc; ++c)
            e[c] = b[c] > 0 ? orc_round_div(s[c] * R, b[c]) : 0;
        int64_t k = 0;
        for (int64_t c = 0; c < nc; ++c)
            if (!fc[c]) tmp[k++] = e[c];
        if (k > 0) {
            int64_t m2, mad4;
            orc_median_mad_i64(tmp, k, &m2, &mad4);
            if (mad4 > 0)
                for (int64_t c = 0; c < nc; ++c) {
                    int64_t d = 2 * e[c] - m2;
                    if (!fc[c] && 20000 * (d < 0 ? -d : d) > (int64_t)kc * 14826 * mad4)
                        fc[c] = 1;
                }
        }
        for (int64_t t = 0; t < nt; ++t) {
            int64_t acc = 0;
            for (int64_t c = 0; c < nc; ++c) {
                int64_t y = b[c] > 0 ? orc_round_div((int64_t)x[t * nc + c] * R, b[c]) : 0;
                if (y > 255) y = 255;
                if (!fc[c]) acc += y;
            }
            u[t] = acc;
        }
        k = 0;
        for (int64_t t = 0; t < nt; ++t)
            if (!ft[t]) tmp[k++] = u[t];
        if (k > 0) {
            int64_t m2, mad4;
            orc_median_mad_i64(tmp, k, &m2, &mad4);
            if (mad4 > 0)
                for (int64_t t = 0; t < nt; ++t) {
                    int64_t d = 2 * u[t] - m2;
                    if (!ft[t] && 20000 * (d < 0 ? -d : d) > (int64_t)kt * 14826 * mad4)
                        ft[t] = 1;
                }
        }
    }
    int64_t fill = tkeep > 0 ? orc_round_div(R, tkeep) : 0;
    if (fill > 255) fill = 255;
    for (int64_t t = 0; t < nt; ++t)
        for (int64_t c = 0; c < nc; ++c) {
            int64_t y;
            if (ft[t] || fc[c]) {
                y = fill;
            } else {
                y = b[c] > 0 ? orc_round_div((int64_t)x[t * nc + c] * R, b[c]) : 0;
                if (y > 255) y = 255;
            }
            out[t * nc + c] = (uint8_t)y;
        }
    free(s); free(b); free(e); free(u); free(tmp); free(win);
    return 0;
}

/* Number of OpenMP threads the DM loop of orc_dedisperse uses from now on
 * (timing only; results do not depend on it). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
