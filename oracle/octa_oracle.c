/*
 * FP64 CPU oracle of the angiography preprocessing of Ploner et al.
 * (arXiv 2010.06931): saccade validity of the B-scans (Sec. 2.2) and the
 * en-face OCTA projection (Sec. 2.3).
 *
 * TEST INFRASTRUCTURE ONLY.  The plain, slow reference the CUDA path is
 * checked against; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code with the CUDA library.
 *
 * Volumes are float32 [h][w][d] on the common grid (depth contiguous).  The
 * B-scans of an X-fast scan are the rows j (fast axis x = i), those of a
 * Y-fast scan the columns i (fast axis y = j).  Order statistics (median,
 * rank, percentile) are taken exactly by sorting; sums, means and the
 * normalisation are double precision.
 *
 * Readings (the paper states no formulas for these steps):
 *   - validity: m_b = mean of the OCTA volume over B-scan b; mu, sigma = mean
 *     and population standard deviation of the m_b; B-scan b is saturated if
 *     m_b > mu + 3 sigma; v_b = 0 if b or any B-scan within 2 of it is
 *     saturated, else 1;
 *   - all filters replicate the edge sample (clamped indices);
 *   - median filter "radius 1": the 27-voxel 3x3x3 neighbourhood, 14th
 *     smallest;
 *   - rank-3 filter of width 15: the 3rd smallest of the 15 samples at
 *     offsets -7..7 along one axis, first along the fast axis, then along the
 *     slow axis;
 *   - percentiles: linear interpolation between order statistics at
 *     position q (N - 1) of the N voxels of the valid B-scans (all B-scans if
 *     none is valid); the 5th maps to 0, the 95th to 1;
 *   - lateral-contrast mask: normalised filtered value < 0.1, i.e. filtered
 *     value < p5 + 0.1 (p95 - p5);
 *   - OCT mask: OCT value > t_oct, t_oct given or (NaN) the mean OCT value
 *     over the valid B-scans;
 *   - en-face value: mean of the OCTA voxels kept by both masks along depth
 *     (0 if none);
 *   - B-scan median subtraction: median of the B-scan's en-face values (mean
 *     of the two middle ones for an even count) subtracted from each;
 *   - invalid B-scans are replaced by the nearest valid one (the lower index
 *     on a tie); nothing is replaced if no B-scan is valid.
 *
 * Parity status: every function is pinned by tests/test_oracle_octa.py
 * (scipy.ndimage filters, numpy percentiles, closed forms, hand-built
 * volumes); none is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static long clampl(long i, long n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

static int cmp_float(const void *a, const void *b)
{
    const float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* number of B-scans and of A-scans per B-scan */
static int n_bscans(int w, int h, int fast_axis) { return fast_axis == 0 ? h : w; }

/* A-scan index p = j * w + i of position f along the fast axis in B-scan b */
static long ascan_of(int w, int fast_axis, int b, int f)
{
    return fast_axis == 0 ? (long)b * w + f : (long)f * w + b;
}

/* Sec. 2.2: per-B-scan mean decorrelation, saturation test, validity. */
void oracle_saccade_validity(const float *A, int w, int h, int d, int fast_axis, float *v_out,
                             double *means_out)
{
    const int nb = n_bscans(w, h, fast_axis), nf = fast_axis == 0 ? w : h;
    double *m = (double *)malloc(sizeof(double) * (size_t)nb);
    for (int b = 0; b < nb; b++) {
        double s = 0.0;
        for (int f = 0; f < nf; f++) {
            const float *col = A + ascan_of(w, fast_axis, b, f) * d;
            for (int k = 0; k < d; k++) s += col[k];
        }
        m[b] = s / ((double)nf * d);
    }
    double mu = 0.0;
    for (int b = 0; b < nb; b++) mu += m[b];
    mu /= nb;
    double var = 0.0;
    for (int b = 0; b < nb; b++) var += (m[b] - mu) * (m[b] - mu);
    const double sigma = sqrt(var / nb);
    for (int b = 0; b < nb; b++) {
        int ok = 1;
        for (int o = -2; o <= 2; o++) {
            const int c = b + o;
            if (c >= 0 && c < nb && m[c] > mu + 3.0 * sigma) ok = 0;
        }
        v_out[b] = ok ? 1.0f : 0.0f;
        if (means_out) means_out[b] = m[b];
    }
    free(m);
}

/* 3x3x3 median, edge samples replicated. */
void oracle_median3(const float *in, int w, int h, int d, float *out)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < h; j++) {
        float v[27];
        for (int i = 0; i < w; i++)
            for (int k = 0; k < d; k++) {
                int n = 0;
                for (int dj = -1; dj <= 1; dj++)
                    for (int di = -1; di <= 1; di++)
                        for (int dk = -1; dk <= 1; dk++)
                            v[n++] = in[(clampl(j + dj, h) * w + clampl(i + di, w)) * d + clampl(k + dk, d)];
                qsort(v, 27, sizeof(float), cmp_float);
                out[((long)j * w + i) * d + k] = v[13];
            }
    }
}

/* Rank filter along axis (0: x, 1: y): the rank-th smallest (1-based) of
 * the width samples centred on each voxel, edge samples replicated. */
void oracle_rank_filter(const float *in, int w, int h, int d, int axis, int width, int rank, float *out)
{
    const int r = width / 2;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < h; j++) {
        float *v = (float *)malloc(sizeof(float) * (size_t)width);
        for (int i = 0; i < w; i++)
            for (int k = 0; k < d; k++) {
                for (int o = -r; o <= r; o++) {
                    const long ii = axis == 0 ? clampl(i + o, w) : i;
                    const long jj = axis == 1 ? clampl(j + o, h) : j;
                    v[o + r] = in[(jj * w + ii) * d + k];
                }
                qsort(v, (size_t)width, sizeof(float), cmp_float);
                out[((long)j * w + i) * d + k] = v[rank - 1];
            }
        free(v);
    }
}

/* q-th quantile (0..1) of n values by linear interpolation between the
 * order statistics at q (n - 1); sorts a copy. */
double oracle_percentile(const float *x, long n, double q)
{
    float *c = (float *)malloc(sizeof(float) * (size_t)n);
    memcpy(c, x, sizeof(float) * (size_t)n);
    qsort(c, (size_t)n, sizeof(float), cmp_float);
    const double pos = q * (double)(n - 1);
    const long lo = (long)floor(pos);
    const long hi = lo + 1 < n ? lo + 1 : lo;
    const double r = (double)c[lo] + (pos - (double)lo) * ((double)c[hi] - (double)c[lo]);
    free(c);
    return r;
}

/* Subtracts from every en-face value the median of its B-scan. */
void oracle_bscan_median_subtract(float *E, int w, int h, int fast_axis)
{
    const int nb = n_bscans(w, h, fast_axis), nf = fast_axis == 0 ? w : h;
    float *v = (float *)malloc(sizeof(float) * (size_t)nf);
    for (int b = 0; b < nb; b++) {
        for (int f = 0; f < nf; f++) v[f] = E[ascan_of(w, fast_axis, b, f)];
        qsort(v, (size_t)nf, sizeof(float), cmp_float);
        const double med = (nf % 2) ? (double)v[nf / 2] : 0.5 * ((double)v[nf / 2 - 1] + (double)v[nf / 2]);
        for (int f = 0; f < nf; f++) {
            float *e = &E[ascan_of(w, fast_axis, b, f)];
            *e = (float)((double)*e - med);
        }
    }
    free(v);
}

/* Replaces every invalid B-scan of E by the nearest valid one. */
void oracle_replace_invalid(float *E, int w, int h, int fast_axis, const float *v)
{
    const int nb = n_bscans(w, h, fast_axis), nf = fast_axis == 0 ? w : h;
    int any = 0;
    for (int b = 0; b < nb; b++) any |= v[b] != 0.0f;
    if (!any) return;
    float *src = (float *)malloc(sizeof(float) * (size_t)nb * nf);
    for (int b = 0; b < nb; b++)
        for (int f = 0; f < nf; f++) src[(long)b * nf + f] = E[ascan_of(w, fast_axis, b, f)];
    for (int b = 0; b < nb; b++) {
        if (v[b] != 0.0f) continue;
        int best = -1;
        for (int dist = 1; best < 0; dist++) {
            if (b - dist >= 0 && v[b - dist] != 0.0f) best = b - dist;
            else if (b + dist < nb && v[b + dist] != 0.0f) best = b + dist;
        }
        for (int f = 0; f < nf; f++) E[ascan_of(w, fast_axis, b, f)] = src[(long)best * nf + f];
    }
    free(src);
}

/* Sec. 2.3: the en-face OCTA image of one scan.
 *   A, S      OCTA (decorrelation) and OCT volumes [h][w][d]
 *   v         B-scan validity (from oracle_saccade_validity)
 *   q_lo/q_hi percentiles mapped to 0 and 1 (0.05, 0.95); thresh 0.1
 *   t_oct     OCT threshold, NaN: the mean OCT value over the valid B-scans
 *   filtered  (may be NULL) receives the rank-filtered volume
 *   E         en-face image [h][w]
 *   info      [p_lo, p_hi, t_oct, kept voxels]                            */
void oracle_enface(const float *A, const float *S, int w, int h, int d, int fast_axis, const float *v,
                   double q_lo, double q_hi, double thresh, double t_oct, float *filtered, float *E,
                   double *info)
{
    const long nvox = (long)w * h * d;
    const int nb = n_bscans(w, h, fast_axis), nf = fast_axis == 0 ? w : h;
    float *m = (float *)malloc(sizeof(float) * (size_t)nvox);
    float *r1 = (float *)malloc(sizeof(float) * (size_t)nvox);
    float *r2 = filtered ? filtered : (float *)malloc(sizeof(float) * (size_t)nvox);
    oracle_median3(A, w, h, d, m);
    oracle_rank_filter(m, w, h, d, fast_axis, 15, 3, r1);
    oracle_rank_filter(r1, w, h, d, 1 - fast_axis, 15, 3, r2);
    free(m);
    free(r1);
    /* voxels of the valid B-scans (all if none is valid) */
    int any = 0;
    for (int b = 0; b < nb; b++) any |= v[b] != 0.0f;
    long nsel = 0;
    float *sel = (float *)malloc(sizeof(float) * (size_t)nvox);
    double ssum = 0.0;
    for (int b = 0; b < nb; b++) {
        if (any && v[b] == 0.0f) continue;
        for (int f = 0; f < nf; f++) {
            const long p = ascan_of(w, fast_axis, b, f);
            for (int k = 0; k < d; k++) {
                sel[nsel++] = r2[p * d + k];
                ssum += S[p * d + k];
            }
        }
    }
    const double p_lo = oracle_percentile(sel, nsel, q_lo);
    const double p_hi = oracle_percentile(sel, nsel, q_hi);
    free(sel);
    if (isnan(t_oct)) t_oct = ssum / (double)nsel;
    const double cut = p_lo + thresh * (p_hi - p_lo);
    double kept_total = 0.0;
    for (long p = 0; p < (long)w * h; p++) {
        double s = 0.0;
        long kept = 0;
        for (int k = 0; k < d; k++) {
            if ((double)r2[p * d + k] < cut && (double)S[p * d + k] > t_oct) {
                s += A[p * d + k];
                kept++;
            }
        }
        E[p] = kept ? (float)(s / (double)kept) : 0.0f;
        kept_total += (double)kept;
    }
    if (!filtered) free(r2);
    oracle_bscan_median_subtract(E, w, h, fast_axis);
    oracle_replace_invalid(E, w, h, fast_axis, v);
    if (info) {
        info[0] = p_lo;
        info[1] = p_hi;
        info[2] = t_oct;
        info[3] = kept_total;
    }
}
