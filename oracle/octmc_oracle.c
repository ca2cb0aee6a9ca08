/*
 * FP64 CPU oracle for the joint orthogonal-raster OCT/OCTA registration
 * objective of Ploner et al., "Efficient and high accuracy 3-D OCT
 * angiography motion correction in pathology" (arXiv 2010.06931).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Everything is computed in double precision from the caller's float
 * volumes.  Every loop follows the definition it implements directly: no
 * blocking, no reordering beyond the sums the equations write.
 *
 * What is computed (paper section / equation in brackets):
 *   - the Hermite interpolator I with central-difference tangents
 *     (Catmull-Rom) and clamp-to-edge sampling               [Sec. 2.1, Eq. 2]
 *   - residuals R_ijk and the per-A-scan structural sum       [Eq. 2, 3, 5]
 *   - pseudo-Huber loss L (and the squared-difference loss)  [Eq. 4]
 *   - resampled validity v~ and the angio weight delta       [Eq. 7, 8]
 *   - en-face angio residual and S^ang                       [Eq. 6]
 *   - combined similarity with eta, and eta itself           [Eq. 9, 10]
 *   - temporal regulariser R and mean term M (readings: the  [Sec. 2.1]
 *     paper defers their exact form to earlier work; R carries the
 *     level depth d like the angio term of Eq. 6)
 *   - validity resampled by a Hermite interpolant without      [Eq. 7, 8]
 *     overshoot, so that 0 <= delta <= delta_0
 *   - the analytic gradient of all of the above (chain rule)
 *   - factor-2 pyramid, displacement prolongation, and the   [Sec. 2.1]
 *     L-BFGS solve with a weak-Wolfe bisection line search
 *
 * Parity status: every function here is pinned by tests under tests/ that
 * check it against closed forms, invariants, brute force or finite
 * differences; none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LOSS_PSEUDO_HUBER 0
#define OR_LOSS_SSD 1

/* One pyramid level of the problem.  Layouts: volumes [h][w][d] with depth
 * contiguous, en-face images and time maps [h][w], validity vx[h] (the
 * X-fast scan's slow axis is y) and vy[w].  Pointers ax/ay may be NULL (no
 * angiography: delta is then 0); vx/vy may be NULL (every B-scan valid). */
typedef struct {
    int w, h, d;
    const float *sx, *sy;
    const float *ax, *ay;
    const float *vx, *vy;
    const double *tx, *ty;
    double alpha;   /* weight of the temporal regulariser R            */
    double delta0;  /* default angio weight delta_0 (Eq. 8)            */
    double eps_h;   /* pseudo-Huber parameter of the data term (Eq. 4) */
    double eps_r;   /* pseudo-Huber parameter of R                     */
    double mu;      /* weight of the mean term M                       */
    double eta;     /* normalisation of Eq. 9                          */
    int loss;       /* OR_LOSS_PSEUDO_HUBER or OR_LOSS_SSD             */
} oracle_level;

/* ------------------------------------------------------------------ */
/* Interpolation (Sec. 2.1: "Hermitian interpolation"; Eq. 7 requires   */
/* continuous first derivatives).  Reading: cubic Hermite spline whose  */
/* node tangents are central differences, m_n = (p_{n+1} - p_{n-1})/2,  */
/* samples outside the grid replicate the nearest edge sample.          */
/* ------------------------------------------------------------------ */

static long clampl(long i, long n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

/* Weights of p_{n-1}, p_n, p_{n+1}, p_{n+2} for a point at n + t, obtained
 * by writing the Hermite form
 *     p(t) = h00 p_n + h10 m_n + h01 p_{n+1} + h11 m_{n+1}
 * with the central-difference tangents substituted; dw = d w / d t. */
void oracle_cr_weights(double t, double w[4], double dw[4])
{
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t;
    double h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
    double d00 = 6 * t2 - 6 * t, d10 = 3 * t2 - 4 * t + 1;
    double d01 = -6 * t2 + 6 * t, d11 = 3 * t2 - 2 * t;
    /* m_n = (p_{n+1} - p_{n-1})/2 , m_{n+1} = (p_{n+2} - p_n)/2 */
    w[0] = -0.5 * h10;
    w[1] = h00 - 0.5 * h11;
    w[2] = h01 + 0.5 * h10;
    w[3] = 0.5 * h11;
    dw[0] = -0.5 * d10;
    dw[1] = d00 - 0.5 * d11;
    dw[2] = d01 + 0.5 * d10;
    dw[3] = 0.5 * d11;
}

/* Integer base = floor(u) and fraction t for a sample at u on a grid of n
 * samples.  With edge replication the interpolant is constant for u < -1
 * and for u >= n, so clamping u into [-4, n+3] first changes neither value
 * nor derivative; it only keeps the integer conversion in range. */
static void split_coord(double u, long n, long *base, double *t)
{
    if (u < -4.0) u = -4.0;
    if (u > (double)n + 3.0) u = (double)n + 3.0;
    double f = floor(u);
    *base = (long)f;
    *t = u - f;
}

/* 1-D interpolation of v (n samples) at u; *du receives dI/du. */
double oracle_interp1(const float *v, int n, double u, double *du)
{
    long b;
    double t, w[4], dw[4], val = 0, der = 0;
    split_coord(u, n, &b, &t);
    oracle_cr_weights(t, w, dw);
    for (int a = 0; a < 4; a++) {
        double p = v[clampl(b - 1 + a, n)];
        val += w[a] * p;
        der += dw[a] * p;
    }
    if (du) *du = der;
    return val;
}

/* Validity resampling (Sec. 2.2, Eq. 7-8).  The paper asks for a Hermite
 * interpolant with continuous first derivatives, and states that delta is
 * delta_0 where both scans are valid, 0 where one is invalid, and fades
 * smoothly in between.  Central-difference tangents overshoot a 0/1 step
 * (delta would become negative next to an invalid band), so this reading
 * takes the cubic Hermite interpolant with zero tangents at the nodes: on
 * [n, n+1] the value is p_n + (p_{n+1} - p_n) (3 t^2 - 2 t^3).  It is C^1,
 * passes through the nodes and stays between the two node values.  Samples
 * outside the line replicate the edge value. */
double oracle_validity_interp(const float *v, int n, double u, double *du)
{
    long b;
    double t;
    split_coord(u, n, &b, &t);
    double p0 = v[clampl(b, n)], p1 = v[clampl(b + 1, n)];
    double h = t * t * (3.0 - 2.0 * t);   /* Hermite basis h01 */
    double dh = 6.0 * t * (1.0 - t);
    if (du) *du = (p1 - p0) * dh;
    return p0 + (p1 - p0) * h;
}

/* 2-D interpolation of an image img[h][w] at (x, y); gradient to g[2]. */
double oracle_interp2(const float *img, int w, int h, double x, double y, double g[2])
{
    long bx, by;
    double tx, ty, wx[4], dwx[4], wy[4], dwy[4];
    split_coord(x, w, &bx, &tx);
    split_coord(y, h, &by, &ty);
    oracle_cr_weights(tx, wx, dwx);
    oracle_cr_weights(ty, wy, dwy);
    double val = 0, gx = 0, gy = 0;
    for (int b = 0; b < 4; b++) {
        long jj = clampl(by - 1 + b, h);
        for (int a = 0; a < 4; a++) {
            long ii = clampl(bx - 1 + a, w);
            double p = img[jj * (long)w + ii];
            val += wx[a] * wy[b] * p;
            gx += dwx[a] * wy[b] * p;
            gy += wx[a] * dwy[b] * p;
        }
    }
    if (g) { g[0] = gx; g[1] = gy; }
    return val;
}

/* 3-D interpolation of vol[h][w][d] at (x, y, z); gradient to g[3].
 * This is the triple sum I = sum_abc wx_a wy_b wz_c S[.][.][.] of the
 * tensor-product Hermite interpolator, written out. */
double oracle_interp3(const float *vol, int w, int h, int d, double x, double y, double z,
                      double g[3])
{
    long bx, by, bz;
    double tx, ty, tz, wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
    split_coord(x, w, &bx, &tx);
    split_coord(y, h, &by, &ty);
    split_coord(z, d, &bz, &tz);
    oracle_cr_weights(tx, wx, dwx);
    oracle_cr_weights(ty, wy, dwy);
    oracle_cr_weights(tz, wz, dwz);
    double val = 0, gx = 0, gy = 0, gz = 0;
    for (int b = 0; b < 4; b++) {
        long jj = clampl(by - 1 + b, h);
        for (int a = 0; a < 4; a++) {
            long ii = clampl(bx - 1 + a, w);
            const float *col = vol + (jj * (long)w + ii) * (long)d;
            for (int c = 0; c < 4; c++) {
                double p = col[clampl(bz - 1 + c, d)];
                val += wx[a] * wy[b] * wz[c] * p;
                gx += dwx[a] * wy[b] * wz[c] * p;
                gy += wx[a] * dwy[b] * wz[c] * p;
                gz += wx[a] * wy[b] * dwz[c] * p;
            }
        }
    }
    if (g) { g[0] = gx; g[1] = gy; g[2] = gz; }
    return val;
}

/* ------------------------------------------------------------------ */
/* Loss (Eq. 4).  L(x) = eps (sqrt(1 + (x/eps)^2) - 1).  Evaluated in the */
/* algebraically identical form x^2 / (eps (sqrt(1+(x/eps)^2) + 1)),      */
/* which avoids the cancellation of "sqrt - 1" for |x| << eps.            */
/* The squared-difference loss is L(x) = x^2.                             */
/* ------------------------------------------------------------------ */
double oracle_loss(double x, double eps, int kind, double *dl)
{
    if (kind == OR_LOSS_SSD) {
        if (dl) *dl = 2.0 * x;
        return x * x;
    }
    double r = x / eps;
    double s = sqrt(1.0 + r * r);
    if (dl) *dl = r / s; /* dL/dx = (x/eps) / sqrt(1 + (x/eps)^2) */
    return (x * x / eps) / (s + 1.0);
}

/* ------------------------------------------------------------------ */
/* Data term, per A-scan (Eq. 2-10).                                    */
/* ------------------------------------------------------------------ */

/* Displacement layout: disp[V][c][j][i], V in {X=0, Y=1}, c in {x,y,z}. */
static inline double dget(const double *disp, int w, int h, int V, int c, int i, int j)
{
    return disp[(((long)V * 3 + c) * h + j) * (long)w + i];
}
static inline long didx(int w, int h, int V, int c, int i, int j)
{
    return (((long)V * 3 + c) * h + j) * (long)w + i;
}

/* Evaluates, for A-scan (i,j) and a given delta_0 and eta:
 *   str  = (1 - delta) sum_k L(R_ijk)                 (one term of Eq. 5)
 *   ang  = delta d L(R_ij(A^X, A^Y))                  (one term of Eq. 6)
 *   g6   = gradient of eta*str + ang/eta w.r.t. the 6 displacement values
 *          of this A-scan (X: dx,dy,dz then Y: dx,dy,dz)   (if g6 != NULL)
 */
static void ascan_terms(const oracle_level *P, const double *disp, int i, int j, double delta0,
                        double eta, double *str_out, double *ang_out, double *g6)
{
    const int w = P->w, h = P->h, d = P->d;
    double dX[3], dY[3];
    for (int c = 0; c < 3; c++) {
        dX[c] = dget(disp, w, h, 0, c, i, j);
        dY[c] = dget(disp, w, h, 1, c, i, j);
    }
    const int have_ang = (P->ax != NULL && P->ay != NULL);
    if (!have_ang) delta0 = 0.0;

    /* Eq. 7: validity resampled along each scan's slow axis. */
    double vtx = 1.0, dvtx = 0.0, vty = 1.0, dvty = 0.0;
    if (P->vx) vtx = oracle_validity_interp(P->vx, h, (double)j + dX[1], &dvtx);
    if (P->vy) vty = oracle_validity_interp(P->vy, w, (double)i + dY[0], &dvty);
    /* Eq. 8 */
    double delta = delta0 * vtx * vty;

    /* Eq. 2-3: structural residuals along depth. */
    double Lsum = 0.0, sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0};
    for (int k = 0; k < d; k++) {
        double gX[3], gY[3];
        double IX = oracle_interp3(P->sx, w, h, d, i + dX[0], j + dX[1], k + dX[2], gX);
        double IY = oracle_interp3(P->sy, w, h, d, i + dY[0], j + dY[1], k + dY[2], gY);
        double dl;
        Lsum += oracle_loss(IX - IY, P->eps_h, P->loss, &dl);
        for (int c = 0; c < 3; c++) {
            sx[c] += dl * gX[c];
            sy[c] += dl * gY[c];
        }
    }

    /* Eq. 6: en-face angio residual (Delta z plays no role in 2-D). */
    double La = 0.0, dla = 0.0, gAX[2] = {0, 0}, gAY[2] = {0, 0};
    if (have_ang) {
        double AX = oracle_interp2(P->ax, w, h, i + dX[0], j + dX[1], gAX);
        double AY = oracle_interp2(P->ay, w, h, i + dY[0], j + dY[1], gAY);
        La = oracle_loss(AX - AY, P->eps_h, P->loss, &dla);
    }

    *str_out = (1.0 - delta) * Lsum;
    *ang_out = delta * (double)d * La;
    if (!g6) return;

    /* Chain rule for eta*(1-delta)*Lsum + delta*d*La/eta. */
    const double cs = eta * (1.0 - delta);       /* weight of the structural sums */
    const double ca = delta * (double)d / eta;   /* weight of L'(Ra)               */
    const double ddelta = -eta * Lsum + (double)d * La / eta; /* d(...)/d delta  */
    g6[0] = cs * sx[0] + ca * dla * gAX[0];
    g6[1] = cs * sx[1] + ca * dla * gAX[1] + ddelta * delta0 * dvtx * vty;
    g6[2] = cs * sx[2];
    g6[3] = -cs * sy[0] - ca * dla * gAY[0] + ddelta * delta0 * vtx * dvty;
    g6[4] = -cs * sy[1] - ca * dla * gAY[1];
    g6[5] = -cs * sy[2];
}

/* Sums of Eq. 5 and Eq. 6 over rows j0 <= j < j1 (all i), with the given
 * delta_0.  Row partial sums are added in row order, so the result does not
 * depend on the number of threads. */
static void data_sums(const oracle_level *P, const double *disp, int j0, int j1, double delta0,
                      double eta, double *str_sum, double *ang_sum, double *grad)
{
    const int w = P->w, h = P->h;
    int nr = j1 - j0;
    double *rs = (double *)calloc((size_t)(nr > 0 ? nr : 1) * 2, sizeof(double));
    /* each row writes its own gradient entries and its own partial sums */
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = j0; j < j1; j++) {
        double s_str = 0, s_ang = 0;
        for (int i = 0; i < w; i++) {
            double st, an, g6[6];
            ascan_terms(P, disp, i, j, delta0, eta, &st, &an, grad ? g6 : NULL);
            s_str += st;
            s_ang += an;
            if (grad)
                for (int V = 0; V < 2; V++)
                    for (int c = 0; c < 3; c++) grad[didx(w, h, V, c, i, j)] = g6[3 * V + c];
        }
        rs[2 * (j - j0)] = s_str;
        rs[2 * (j - j0) + 1] = s_ang;
    }
    double a = 0, b = 0;
    for (int r = 0; r < nr; r++) {
        a += rs[2 * r];
        b += rs[2 * r + 1];
    }
    free(rs);
    *str_sum = a;
    *ang_sum = b;
}

/* ------------------------------------------------------------------ */
/* Temporal regulariser R (Sec. 2.1; the paper refers to Kraus et al.   */
/* for its exact form).  Reading: the A-scans of each volume are ordered */
/* by their sampling time t; each pair of consecutive samples n, n+1     */
/* contributes omega_n sum_c L_{eps_r}(d_{n+1,c} - d_{n,c}) ("absolute   */
/* displacement differences", smoothed), with omega_n = dt_min / dt_n so  */
/* that steps across the flyback between B-scans weigh less.            */
/* ------------------------------------------------------------------ */

static const double *g_sort_keys;
static int cmp_time(const void *a, const void *b)
{
    long ia = *(const long *)a, ib = *(const long *)b;
    double ta = g_sort_keys[ia], tb = g_sort_keys[ib];
    if (ta < tb) return -1;
    if (ta > tb) return 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0); /* ties: by index */
}

/* Builds the time-ordered chain of n samples: order[0..n-1] (indices into
 * the [h][w] map) and omega[0..n-2] (weight of pair order[m], order[m+1]). */
void oracle_chain(const double *t, long n, long *order, double *omega)
{
    for (long m = 0; m < n; m++) order[m] = m;
    g_sort_keys = t;
    qsort(order, (size_t)n, sizeof(long), cmp_time);
    double dtmin = INFINITY;
    for (long m = 0; m + 1 < n; m++) {
        double dt = t[order[m + 1]] - t[order[m]];
        if (dt > 0 && dt < dtmin) dtmin = dt;
    }
    for (long m = 0; m + 1 < n; m++) {
        double dt = t[order[m + 1]] - t[order[m]];
        if (!(dtmin < INFINITY)) omega[m] = 1.0;           /* all times equal */
        else omega[m] = dtmin / (dt > dtmin ? dt : dtmin); /* ties weigh 1    */
    }
}

/* R(D) and, if grad != NULL, adds alpha * dR/dD into grad.
 *
 * Scale reading: each pair's penalty is multiplied by the depth d of the
 * level.  The structural data term sums d voxels per A-scan (Eq. 3, 5), and
 * Eq. 6 multiplies the per-A-scan angiographic loss by d for exactly this
 * reason; R is a per-A-scan quantity as well, so it carries the same factor.
 * Then alpha weighs the regulariser against the data term in the same ratio
 * on every pyramid level (d halves with the voxel count per A-scan), and
 * the paper's alpha values (0.001 ... 1, Sec. 4) change the result, which
 * they do not with an unscaled R (its size is that of one voxel per A-scan). */
static double regulariser(const oracle_level *P, const double *disp, double *grad)
{
    const int w = P->w, h = P->h;
    const long n = (long)w * h;
    long *order = (long *)malloc(sizeof(long) * (size_t)n);
    double *omega = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
    double R = 0.0;
    for (int V = 0; V < 2; V++) {
        oracle_chain(V == 0 ? P->tx : P->ty, n, order, omega);
        for (long m = 0; m + 1 < n; m++) {
            long p = order[m], q = order[m + 1];
            for (int c = 0; c < 3; c++) {
                long ip = ((long)V * 3 + c) * n + p, iq = ((long)V * 3 + c) * n + q;
                double dl;
                R += P->d * omega[m] * oracle_loss(disp[iq] - disp[ip], P->eps_r, OR_LOSS_PSEUDO_HUBER, &dl);
                if (grad) {
                    grad[iq] += P->alpha * P->d * omega[m] * dl;
                    grad[ip] -= P->alpha * P->d * omega[m] * dl;
                }
            }
        }
    }
    free(order);
    free(omega);
    return R;
}

/* Mean term M (Sec. 2.1: penalises the sum of displacements, fixing the
 * three translational degrees of freedom).  Reading:
 *     M = mu sum_c ( sum_V sum_ij d^V_ij,c )^2 .
 * Adds dM/dD into grad when grad != NULL. */
static double mean_term(const oracle_level *P, const double *disp, double *grad)
{
    const long n = (long)P->w * P->h;
    double M = 0.0;
    for (int c = 0; c < 3; c++) {
        double s = 0.0;
        for (int V = 0; V < 2; V++)
            for (long p = 0; p < n; p++) s += disp[((long)V * 3 + c) * n + p];
        M += P->mu * s * s;
        if (grad)
            for (int V = 0; V < 2; V++)
                for (long p = 0; p < n; p++) grad[((long)V * 3 + c) * n + p] += 2.0 * P->mu * s;
    }
    return M;
}

/* ------------------------------------------------------------------ */
/* Objective (Eq. 1 with Eq. 9 replacing the structural term).          */
/*   f = eta S^str + S^ang / eta + alpha R + M                           */
/* terms (optional, 6 values): [S^str, S^ang, R, M, f, eta].              */
/* grad (optional): 6*w*h values, layout disp[V][c][j][i].                */
/* ------------------------------------------------------------------ */
int oracle_eval(const oracle_level *P, const double *disp, double *f_out, double *grad,
                double *terms)
{
    double Sstr, Sang;
    data_sums(P, disp, 0, P->h, P->delta0, P->eta, &Sstr, &Sang, grad);
    double R = regulariser(P, disp, grad);
    double M = mean_term(P, disp, grad);
    double f = P->eta * Sstr + Sang / P->eta + P->alpha * R + M;
    if (terms) {
        terms[0] = Sstr;
        terms[1] = Sang;
        terms[2] = R;
        terms[3] = M;
        terms[4] = f;
        terms[5] = P->eta;
    }
    if (f_out) *f_out = f;
    return isfinite(f) ? 0 : -4;
}

/* Data-term sums over rows [j0, j1) only, no gradient: used to time a
 * bounded sample of a full-size evaluation. */
void oracle_data_rows(const oracle_level *P, const double *disp, int j0, int j1, double *sums2)
{
    data_sums(P, disp, j0, j1, P->delta0, P->eta, &sums2[0], &sums2[1], NULL);
}

/* Eq. 10: eta = sqrt(S^ang_0.5(D0) / S^str_0.5(D0)), always with delta_0 =
 * 0.5 (the subscript of Eq. 10).  Reading for the degenerate cases: eta = 1
 * when there is no angiography, or either sum is zero or not finite. */
double oracle_eta(const oracle_level *P, const double *disp0)
{
    if (!P->ax || !P->ay) return 1.0;
    double Sstr, Sang;
    data_sums(P, disp0, 0, P->h, 0.5, 1.0, &Sstr, &Sang, NULL);
    double e = sqrt(Sang / Sstr);
    if (!(Sstr > 0) || !(Sang > 0) || !isfinite(e)) return 1.0;
    return e;
}

/* ------------------------------------------------------------------ */
/* Factor-2 pyramid (Sec. 2.1) and its validity (Sec. 2.2: downsampled  */
/* "in the same way").  Reading: box mean over 2 samples per downsampled */
/* axis; an odd size rounds up and the missing sample repeats the edge.  */
/* ------------------------------------------------------------------ */
static int half_up(int n) { return (n + 1) / 2; }

void oracle_pyramid_volume(const float *in, int w, int h, int d, float *out)
{
    int w2 = half_up(w), h2 = half_up(h), d2 = half_up(d);
    for (int j = 0; j < h2; j++)
        for (int i = 0; i < w2; i++)
            for (int k = 0; k < d2; k++) {
                double s = 0.0;
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++)
                        for (int c = 0; c < 2; c++)
                            s += in[(clampl(2 * j + b, h) * (long)w + clampl(2 * i + a, w)) * (long)d +
                                    clampl(2 * k + c, d)];
                out[((long)j * w2 + i) * d2 + k] = (float)(s / 8.0);
            }
}

void oracle_pyramid_image(const float *in, int w, int h, float *out)
{
    int w2 = half_up(w), h2 = half_up(h);
    for (int j = 0; j < h2; j++)
        for (int i = 0; i < w2; i++) {
            double s = 0.0;
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) s += in[clampl(2 * j + b, h) * (long)w + clampl(2 * i + a, w)];
            out[(long)j * w2 + i] = (float)(s / 4.0);
        }
}

void oracle_pyramid_line(const float *in, int n, float *out)
{
    for (int i = 0; i < half_up(n); i++)
        out[i] = (float)((in[clampl(2 * i, n)] + (double)in[clampl(2 * i + 1, n)]) / 2.0);
}

void oracle_pyramid_time(const double *in, int w, int h, double *out)
{
    int w2 = half_up(w), h2 = half_up(h);
    for (int j = 0; j < h2; j++)
        for (int i = 0; i < w2; i++) {
            double s = 0.0;
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) s += in[clampl(2 * j + b, h) * (long)w + clampl(2 * i + a, w)];
            out[(long)j * w2 + i] = s / 4.0;
        }
}

/* Displacement prolongation from a coarse level (wc x hc) to the next finer
 * level (wf x hf).  Reading: a fine A-scan centre i sits at (i - 0.5)/2 on
 * the coarse grid (box-filter centres); the coarse field is interpolated
 * bilinearly there (coordinates clamped to the grid) and, since pixel units
 * halve, every component is doubled. */
void oracle_prolong(const double *coarse, int wc, int hc, double *fine, int wf, int hf)
{
    for (int V = 0; V < 2; V++)
        for (int c = 0; c < 3; c++) {
            const double *src = coarse + ((long)V * 3 + c) * wc * (long)hc;
            double *dst = fine + ((long)V * 3 + c) * wf * (long)hf;
            for (int j = 0; j < hf; j++)
                for (int i = 0; i < wf; i++) {
                    double x = (i - 0.5) / 2.0, y = (j - 0.5) / 2.0;
                    if (x < 0) x = 0;
                    if (y < 0) y = 0;
                    if (x > wc - 1) x = wc - 1;
                    if (y > hc - 1) y = hc - 1;
                    long x0 = (long)floor(x), y0 = (long)floor(y);
                    long x1 = x0 + 1 < wc ? x0 + 1 : x0, y1 = y0 + 1 < hc ? y0 + 1 : y0;
                    double fx = x - x0, fy = y - y0;
                    double v = (1 - fx) * (1 - fy) * src[y0 * wc + x0] + fx * (1 - fy) * src[y0 * wc + x1] +
                               (1 - fx) * fy * src[y1 * wc + x0] + fx * fy * src[y1 * wc + x1];
                    dst[(long)j * wf + i] = 2.0 * v;
                }
        }
}

/* ------------------------------------------------------------------ */
/* L-BFGS (Sec. 2.1: "gradient-based L-BFGS solver").  The paper gives no */
/* details; reading: history m, two-loop recursion with the scaling       */
/* gamma = s'y / y'y, pairs with s'y <= 1e-12 * y'y are not stored, and a */
/* weak-Wolfe bisection line search (c1 = 1e-4, c2 = 0.9).               */
/* ------------------------------------------------------------------ */
static double dot(const double *a, const double *b, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Two-loop recursion: dir = -H g for the stored pairs (oldest first:
 * S[0..k-1], Y[0..k-1]).  With k == 0 the direction is -g. */
void oracle_lbfgs_direction(long n, int k, const double *const *S, const double *const *Y,
                            const double *g, double *dir)
{
    double *q = dir;
    double alpha[64];
    for (long i = 0; i < n; i++) q[i] = g[i];
    for (int m = k - 1; m >= 0; m--) {
        double rho = 1.0 / dot(Y[m], S[m], n);
        alpha[m] = rho * dot(S[m], q, n);
        for (long i = 0; i < n; i++) q[i] -= alpha[m] * Y[m][i];
    }
    double gamma = 1.0;
    if (k > 0) gamma = dot(S[k - 1], Y[k - 1], n) / dot(Y[k - 1], Y[k - 1], n);
    for (long i = 0; i < n; i++) q[i] *= gamma;
    for (int m = 0; m < k; m++) {
        double rho = 1.0 / dot(Y[m], S[m], n);
        double beta = rho * dot(Y[m], q, n);
        for (long i = 0; i < n; i++) q[i] += S[m][i] * (alpha[m] - beta);
    }
    for (long i = 0; i < n; i++) dir[i] = -q[i];
}

typedef struct {
    int m;          /* history length                                  */
    int max_iter;   /* iteration cap                                   */
    int max_ls;     /* evaluations per line search                     */
    double gtol;    /* stop when max|g| <= gtol                        */
    double ftol;    /* stop when the relative decrease stays below ftol */
                    /* for 3 consecutive iterations                    */
} oracle_solver;

typedef struct {
    int iters, evals, status; /* status 0: converged, 1: iteration cap, 2: line search failed */
    double f;
} oracle_stats;

/* Minimises fg (objective and gradient of n values) from x (in/out).
 * Line search (weak Wolfe, bisection/doubling): start at a = 1, or at
 * a = 1/||g||_2 when the history is empty; a trial that fails the Armijo
 * test (c1 = 1e-4) or is not finite halves the bracket; one that passes it
 * but fails the curvature test (c2 = 0.9) raises the lower end (doubling a
 * while no upper end exists); otherwise it is accepted.  After max_ls
 * trials the best Armijo point so far is taken; with none, the history is
 * dropped and the iteration retried once from -g, and then the solve stops
 * (status 2).  Other stops: max|g| <= gtol (status 0), a relative decrease
 * (f_old - f_new) / max(|f_old|, |f_new|, 1) below ftol for 3 iterations in
 * a row (status 0), max_iter iterations (status 1). */
typedef void (*oracle_fg)(void *ctx, const double *x, double *f, double *g);

static int lbfgs_minimize(long n, double *x, oracle_fg fg, void *ctx, const oracle_solver *opt,
                          oracle_stats *st)
{
    const int m = opt->m > 0 ? (opt->m < 64 ? opt->m : 64) : 1;
    const size_t nb = sizeof(double) * (size_t)n;
    double *g = (double *)malloc(nb), *gt = (double *)malloc(nb), *xt = (double *)malloc(nb);
    double *dir = (double *)malloc(nb), *gb = (double *)malloc(nb), *xb = (double *)malloc(nb);
    double *sn = (double *)malloc(nb), *yn = (double *)malloc(nb);
    double *S[64], *Y[64];
    const double *So[64], *Yo[64];
    for (int i = 0; i < m; i++) {
        S[i] = (double *)malloc(nb);
        Y[i] = (double *)malloc(nb);
    }
    int k = 0, head = 0, evals = 0, iters = 0, status = 1, small = 0, retried = 0;
    double f;
    fg(ctx, x, &f, g);
    evals++;
    while (iters < opt->max_iter) {
        double gmax = 0;
        for (long i = 0; i < n; i++) gmax = fmax(gmax, fabs(g[i]));
        if (gmax <= opt->gtol) { status = 0; break; }
        for (int t = 0; t < k; t++) {
            So[t] = S[(head + t) % m];
            Yo[t] = Y[(head + t) % m];
        }
        oracle_lbfgs_direction(n, k, So, Yo, g, dir);
        double dg0 = dot(g, dir, n);
        if (!(dg0 < 0)) { /* not a descent direction: restart from -g */
            k = 0;
            head = 0;
            for (long i = 0; i < n; i++) dir[i] = -g[i];
            dg0 = dot(g, dir, n);
        }
        double a = (k == 0) ? 1.0 / sqrt(dot(g, g, n)) : 1.0;
        double lo = 0.0, hi = INFINITY, ft = 0.0, fb = 0.0;
        int accepted = 0, have_lo = 0;
        for (int ls = 0; ls < opt->max_ls; ls++) {
            for (long i = 0; i < n; i++) xt[i] = x[i] + a * dir[i];
            fg(ctx, xt, &ft, gt);
            evals++;
            double dgt = dot(gt, dir, n);
            if (!(ft <= f + 1e-4 * a * dg0)) {
                hi = a;
                a = 0.5 * (lo + hi);
            } else if (dgt < 0.9 * dg0) {
                lo = a;
                have_lo = 1;
                fb = ft;
                memcpy(xb, xt, nb);
                memcpy(gb, gt, nb);
                a = isinf(hi) ? 2.0 * a : 0.5 * (lo + hi);
            } else {
                accepted = 1;
                break;
            }
        }
        if (!accepted) {
            if (have_lo) {
                memcpy(xt, xb, nb);
                memcpy(gt, gb, nb);
                ft = fb;
            } else if (k > 0 && !retried) {
                k = 0;
                head = 0;
                retried = 1;
                continue;
            } else {
                status = 2;
                break;
            }
        }
        retried = 0;
        /* history pair s = x_new - x, y = g_new - g (kept if s'y > 1e-12 y'y) */
        for (long i = 0; i < n; i++) {
            sn[i] = xt[i] - x[i];
            yn[i] = gt[i] - g[i];
        }
        double sy = dot(sn, yn, n), yy = dot(yn, yn, n);
        if (sy > 1e-12 * yy) {
            int slot;
            if (k < m) {
                slot = (head + k) % m;
                k++;
            } else {
                slot = head;
                head = (head + 1) % m;
            }
            memcpy(S[slot], sn, nb);
            memcpy(Y[slot], yn, nb);
        }
        double rel = (f - ft) / fmax(fmax(fabs(f), fabs(ft)), 1.0);
        memcpy(x, xt, nb);
        memcpy(g, gt, nb);
        f = ft;
        iters++;
        small = (rel < opt->ftol) ? small + 1 : 0;
        if (small >= 3) { status = 0; break; }
    }
    for (int i = 0; i < m; i++) {
        free(S[i]);
        free(Y[i]);
    }
    free(g); free(gt); free(xt); free(dir); free(gb); free(xb); free(sn); free(yn);
    st->iters = iters;
    st->evals = evals;
    st->status = status;
    st->f = f;
    return 0;
}

static void level_fg(void *ctx, const double *x, double *f, double *g)
{
    oracle_eval((const oracle_level *)ctx, x, f, g, NULL);
}

/* Minimises the level objective from x (in/out), eta fixed in P (the
 * minimiser above on oracle_eval). */
int oracle_solve_level(const oracle_level *P, double *x, const oracle_solver *opt,
                       oracle_stats *st)
{
    return lbfgs_minimize(6L * P->w * P->h, x, level_fg, (void *)P, opt, st);
}

/* The minimiser above on a caller-supplied objective fn(n, x, f, g), so the
 * L-BFGS and its line search (Sec. 2.1) can be checked on their own. */
typedef struct {
    void (*fn)(long n, const double *x, double *f, double *g);
    long n;
} fn_ctx;

static void fn_fg(void *ctx, const double *x, double *f, double *g)
{
    const fn_ctx *c = (const fn_ctx *)ctx;
    c->fn(c->n, x, f, g);
}

int oracle_lbfgs_minimize_fn(long n, double *x, void (*fn)(long, const double *, double *, double *),
                             const oracle_solver *opt, oracle_stats *st)
{
    fn_ctx c = {fn, n};
    return lbfgs_minimize(n, x, fn_fg, (void *)&c, opt, st);
}

/* Number of threads the OpenMP loops use (1 without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Final resampling and merging (Sec. 2.1, last paragraphs; Sec. 2.5).   */
/* Readings (the paper gives no constants or formulas):                  */
/*  - motion-corrected volume C^V = I(S^V, p_ijk + d^V_ij) (the same      */
/*    Hermite interpolator);                                             */
/*  - sampling density: every motion-corrected A-scan deposits weight 1   */
/*    at its transverse sampling position (i + dx, j + dy), clamped into  */
/*    the grid, split bilinearly over the 4 surrounding input A-scans;    */
/*    the density of A-scan (i,j) is that map read back bilinearly at its */
/*    own sampling position (1 without motion);                          */
/*  - weight exp(-beta * max(0, density - 1)) ("exponentially decaying   */
/*    for a density higher than normal"), set to 0 below tau; the two    */
/*    volumes' weights are normalised to sum 1; where both are clipped   */
/*    the volume with the larger weight is kept alone ("the B-scan with  */
/*    less oversampling remains");                                       */
/*  - en-face angiography: weights multiplied by the resampled validity  */
/*    (Eq. 7, Sec. 2.5), normalised; 0 where both products are 0.        */
/* ------------------------------------------------------------------ */
static double density_at(const double *map, int w, int h, double x, double y)
{
    if (x < 0) x = 0;
    if (y < 0) y = 0;
    if (x > w - 1) x = w - 1;
    if (y > h - 1) y = h - 1;
    long x0 = (long)floor(x), y0 = (long)floor(y);
    long x1 = x0 + 1 < w ? x0 + 1 : x0, y1 = y0 + 1 < h ? y0 + 1 : y0;
    double fx = x - x0, fy = y - y0;
    return (1 - fx) * (1 - fy) * map[y0 * w + x0] + fx * (1 - fy) * map[y0 * w + x1] +
           (1 - fx) * fy * map[y1 * w + x0] + fx * fy * map[y1 * w + x1];
}

static void splat(double *map, int w, int h, double x, double y)
{
    if (x < 0) x = 0;
    if (y < 0) y = 0;
    if (x > w - 1) x = w - 1;
    if (y > h - 1) y = h - 1;
    long x0 = (long)floor(x), y0 = (long)floor(y);
    long x1 = x0 + 1 < w ? x0 + 1 : x0, y1 = y0 + 1 < h ? y0 + 1 : y0;
    double fx = x - x0, fy = y - y0;
    map[y0 * w + x0] += (1 - fx) * (1 - fy);
    map[y0 * w + x1] += fx * (1 - fy);
    map[y1 * w + x0] += (1 - fx) * fy;
    map[y1 * w + x1] += fx * fy;
}

/* Outputs (any may be NULL): merged[h][w][d], corrected X / Y [h][w][d],
 * weights[2][h][w] (normalised structural weights), angio[h][w],
 * density[2][h][w]. */
void oracle_merge(const oracle_level *P, const double *disp, double beta, double tau, float *merged,
                  float *cx, float *cy, float *weights, float *angio, double *density)
{
    const int w = P->w, h = P->h, d = P->d;
    const long n = (long)w * h;
    double *map = (double *)calloc((size_t)(2 * n), sizeof(double));
    for (int V = 0; V < 2; V++)
        for (int j = 0; j < h; j++)
            for (int i = 0; i < w; i++)
                splat(map + V * n, w, h, i + dget(disp, w, h, V, 0, i, j), j + dget(disp, w, h, V, 1, i, j));
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < h; j++)
        for (int i = 0; i < w; i++) {
            const long p = (long)j * w + i;
            double wt[2], rho[2], va[2] = {1.0, 1.0};
            for (int V = 0; V < 2; V++) {
                double x = i + dget(disp, w, h, V, 0, i, j), y = j + dget(disp, w, h, V, 1, i, j);
                rho[V] = density_at(map + V * n, w, h, x, y);
                wt[V] = exp(-beta * fmax(0.0, rho[V] - 1.0));
                if (density) density[V * n + p] = rho[V];
            }
            double c0 = wt[0] >= tau ? wt[0] : 0.0, c1 = wt[1] >= tau ? wt[1] : 0.0;
            if (c0 == 0.0 && c1 == 0.0) {
                if (wt[0] >= wt[1]) c0 = 1.0;
                else c1 = 1.0;
            }
            const double wx = c0 / (c0 + c1), wy = c1 / (c0 + c1);
            if (weights) {
                weights[p] = (float)wx;
                weights[n + p] = (float)wy;
            }
            for (int k = 0; k < d; k++) {
                double IX = oracle_interp3(P->sx, w, h, d, i + dget(disp, w, h, 0, 0, i, j),
                                           j + dget(disp, w, h, 0, 1, i, j), k + dget(disp, w, h, 0, 2, i, j), NULL);
                double IY = oracle_interp3(P->sy, w, h, d, i + dget(disp, w, h, 1, 0, i, j),
                                           j + dget(disp, w, h, 1, 1, i, j), k + dget(disp, w, h, 1, 2, i, j), NULL);
                if (merged) merged[p * d + k] = (float)(wx * IX + wy * IY);
                if (cx) cx[p * d + k] = (float)IX;
                if (cy) cy[p * d + k] = (float)IY;
            }
            if (angio && P->ax && P->ay) {
                double gdummy[2], AXv, AYv;
                AXv = oracle_interp2(P->ax, w, h, i + dget(disp, w, h, 0, 0, i, j), j + dget(disp, w, h, 0, 1, i, j), gdummy);
                AYv = oracle_interp2(P->ay, w, h, i + dget(disp, w, h, 1, 0, i, j), j + dget(disp, w, h, 1, 1, i, j), gdummy);
                if (P->vx) va[0] = oracle_validity_interp(P->vx, h, j + dget(disp, w, h, 0, 1, i, j), NULL);
                if (P->vy) va[1] = oracle_validity_interp(P->vy, w, i + dget(disp, w, h, 1, 0, i, j), NULL);
                double a0 = fmax(0.0, c0 * va[0]), a1 = fmax(0.0, c1 * va[1]);
                angio[p] = (a0 + a1 > 0) ? (float)((a0 * AXv + a1 * AYv) / (a0 + a1)) : 0.0f;
            }
        }
    free(map);
}

/* ------------------------------------------------------------------ */
/* Rough axial prealignment (stage 1, Sec. 2.1 / Fig. 1).               */
/* Readings (the paper gives the parameterisation in words and defers  */
/* the tilt term T to earlier work):                                    */
/*  - parameters per B-scan b of each scan: axial offset a_b and tilt   */
/*    t_b; the A-scan at fast-axis position f of B-scan b is displaced  */
/*    axially by a_b + t_b (f - c), c = (n_f - 1) / 2, transversally by */
/*    0.  Layout [aX(h), tX(h), aY(w), tY(w)]: X-fast B-scans are rows  */
/*    j (f = i), Y-fast B-scans columns i (f = j);                      */
/*  - objective S_0^str + alpha R + M + T (Eq. 1): the structural data  */
/*    term alone (no angiography: delta_0 = 0, eta = 1), R and M of the */
/*    induced field;                                                    */
/*  - T fixes the tilt modes the data cannot see.  A deformation of the */
/*    common frame z = f(x, y) that both parameterisations can express  */
/*    (f in span{1, x, y, x y}) leaves the objective unchanged; M fixes */
/*    the constant, T the other three: a common x tilt (equal tilts of  */
/*    the X-fast B-scans, Y-fast offsets linear in i), a common y tilt, */
/*    and the twist x y (X tilts linear in j, Y tilts linear in i).     */
/*    Each term is the square of the linear functional the mode moves,  */
/*    weighted so that a mode of the frame costs what M charges for a   */
/*    shift of the same displacement energy (both volumes' squared      */
/*    displacements, 2 w h c^2 for a shift c).  With vx = (w^2 - 1)/12, */
/*    vy = (h^2 - 1)/12, sX = sum tX, sY = sum tY,                      */
/*    sT = sum_j tX_j (j - cy) + sum_i tY_i (i - cx), nT = h vy + w vx:  */
/*    T = 2 w vx sX^2 / h + 2 h vy sY^2 / w + 2 w h vx vy sT^2 / nT^2.  */
/*  - between levels: fine B-scan b sits at (b - 1/2) / 2 on the coarse */
/*    level (clamped, linear); offsets double, tilts are kept.          */
/* ------------------------------------------------------------------ */
void oracle_prealign_disp(const oracle_level *P, const double *prm, double *disp)
{
    const int w = P->w, h = P->h;
    const double cx = 0.5 * (w - 1), cy = 0.5 * (h - 1);
    const double *aX = prm, *tX = prm + h, *aY = prm + 2 * h, *tY = prm + 2 * h + w;
    memset(disp, 0, sizeof(double) * 6 * (size_t)w * h);
    for (int j = 0; j < h; j++)
        for (int i = 0; i < w; i++) {
            disp[didx(w, h, 0, 2, i, j)] = aX[j] + tX[j] * (i - cx);
            disp[didx(w, h, 1, 2, i, j)] = aY[i] + tY[i] * (j - cy);
        }
}

/* f and df/dprm of the stage-1 objective; terms (may be NULL) receives
 * [S^str, R, M, T, f]. */
void oracle_prealign_eval(const oracle_level *P, const double *prm, double *f_out, double *gprm, double *terms)
{
    const int w = P->w, h = P->h;
    const double cx = 0.5 * (w - 1), cy = 0.5 * (h - 1);
    oracle_level Q = *P;
    Q.delta0 = 0.0;
    Q.eta = 1.0;
    const size_t n = 6 * (size_t)w * h;
    double *disp = (double *)malloc(sizeof(double) * n), *g = (double *)malloc(sizeof(double) * n);
    double t6[6], f;
    oracle_prealign_disp(P, prm, disp);
    oracle_eval(&Q, disp, &f, g, t6);
    const double *tX = prm + h, *tY = prm + 2 * h + w;
    double sX = 0.0, sY = 0.0, sT = 0.0, nT = 0.0;
    for (int j = 0; j < h; j++) {
        sX += tX[j];
        sT += tX[j] * (j - cy);
        nT += (j - cy) * (j - cy);
    }
    for (int i = 0; i < w; i++) {
        sY += tY[i];
        sT += tY[i] * (i - cx);
        nT += (i - cx) * (i - cx);
    }
    const double vx = (w * (double)w - 1.0) / 12.0, vy = (h * (double)h - 1.0) / 12.0;
    const double lx = 2.0 * w * vx / h, ly = 2.0 * h * vy / w;
    const double lt = nT > 0 ? 2.0 * w * h * vx * vy / (nT * nT) : 0.0;
    const double T = lx * sX * sX + ly * sY * sY + lt * sT * sT;
    f += T;
    if (gprm) {
        for (int j = 0; j < h; j++) {
            double ga = 0.0, gt = 0.0;
            for (int i = 0; i < w; i++) {
                const double gz = g[didx(w, h, 0, 2, i, j)];
                ga += gz;
                gt += gz * (i - cx);
            }
            gprm[j] = ga;
            gprm[h + j] = gt + 2.0 * lx * sX + 2.0 * lt * sT * (j - cy);
        }
        for (int i = 0; i < w; i++) {
            double ga = 0.0, gt = 0.0;
            for (int j = 0; j < h; j++) {
                const double gz = g[didx(w, h, 1, 2, i, j)];
                ga += gz;
                gt += gz * (j - cy);
            }
            gprm[2 * h + i] = ga;
            gprm[2 * h + w + i] = gt + 2.0 * ly * sY + 2.0 * lt * sT * (i - cx);
        }
    }
    if (terms) {
        terms[0] = t6[0];
        terms[1] = t6[2];
        terms[2] = t6[3];
        terms[3] = T;
        terms[4] = f;
    }
    if (f_out) *f_out = f;
    free(disp);
    free(g);
}

static void prealign_fg(void *ctx, const double *x, double *f, double *g)
{
    oracle_prealign_eval((const oracle_level *)ctx, x, f, g, NULL);
}

/* L-BFGS solve of the stage-1 objective of one level from prm (in/out). */
int oracle_prealign_level(const oracle_level *P, double *prm, const oracle_solver *opt, oracle_stats *st)
{
    return lbfgs_minimize(2L * (P->w + P->h), prm, prealign_fg, (void *)P, opt, st);
}

/* Parameters of the coarse level (wc, hc) to the fine level (wf, hf). */
void oracle_prealign_prolong(const double *pc, int wc, int hc, double *pf, int wf, int hf)
{
    for (int part = 0; part < 4; part++) {
        const int nc = part < 2 ? hc : wc, nf = part < 2 ? hf : wf;
        const double *c = pc + (part < 2 ? part * hc : 2 * hc + (part - 2) * wc);
        double *o = pf + (part < 2 ? part * hf : 2 * hf + (part - 2) * wf);
        const double scale = (part % 2 == 0) ? 2.0 : 1.0;  /* offsets double, tilts are kept */
        for (int b = 0; b < nf; b++) {
            double x = 0.5 * b - 0.25;
            if (x < 0) x = 0;
            if (x > nc - 1) x = nc - 1;
            const int x0 = (int)floor(x), x1 = x0 + 1 < nc ? x0 + 1 : x0;
            const double fx = x - x0;
            o[b] = scale * ((1.0 - fx) * c[x0] + fx * c[x1]);
        }
    }
}
