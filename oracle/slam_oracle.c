/*
 * slam_oracle.c -- plain CPU oracle of the batched SLAM-backbone primitives
 * (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA path).
 *
 * Correlative scan matching (Sec. III-D): every candidate pose of a
 * discretised (dx, dy, dth) neighbourhood of the predicted pose is scored
 * against the log-odds grid; the best one is an absolute pose measurement
 * whose information is scaled by the normalised match score and by the
 * ambiguity margin between the best and the second-best candidates.
 *
 * The candidate set and score (this project's reading):
 *   translations (i, j) in [-n, n]^2 whole cells, rotations k in [-m, m]
 *   steps of dth; th_k = th + k*dth in fp32; for each returned beam
 *   (z < r_max) with table direction (cb, sb): the rotated direction
 *   (c cb - s sb, s cb + c sb) with (s, c) = orc_sincosf(th_k), the endpoint
 *   (x + z*dx, y + z*dy), its cell (floor(x/res), floor(y/res)) shifted by
 *   (i, j); the score adds the cell's occupancy evidence
 *   min(255, max(L, 0) >> 4), or 0 outside the map.
 *   best = highest score, ties to the lowest index
 *   ((k+m)(2n+1) + (j+n))(2n+1) + (i+n); second = highest score among the
 *   candidates more than `sep` steps from the best in some coordinate.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_sincosf(float x, float *s, float *c);
void orc_beam_dirs(int B, double fov, float *cb, float *sb);

static int orc_evidence(int16_t L)
{
    int v = L > 0 ? (int)L >> 4 : 0;
    return v < 255 ? v : 255;
}

/* One env: belief [H*W], pose (x, y, th), ranges z [B] (beam layout of a
 * B-beam sensor over fov).  Writes pose_out[3], match[3], scores[3]. */
void orc_csm(const int16_t *belief, int32_t W, int32_t H, float res, float r_max, int32_t B,
             double fov, const float *z, float x, float y, float th, int32_t n, int32_t m,
             int32_t sep, float dth, float *pose_out, float *match, int64_t *scores)
{
    float cb[4096], sb[4096];
    if (B > 4096)
        return;
    orc_beam_dirs(B, fov, cb, sb);
    const int side = 2 * n + 1, nk = 2 * m + 1;
    int64_t best = -1, best_q = 0;
    int64_t score[17 * 17 * 17];
    int nret = 0;
    for (int b = 0; b < B; ++b)
        if (z[b] < r_max)
            ++nret;
    for (int k = -m; k <= m; ++k) {
        float thk = th + (float)k * dth;
        float s, c;
        orc_sincosf(thk, &s, &c);
        for (int j = -n; j <= n; ++j)
            for (int i = -n; i <= n; ++i) {
                int64_t sc = 0;
                for (int b = 0; b < B; ++b) {
                    if (!(z[b] < r_max))
                        continue;
                    float dx = c * cb[b] - s * sb[b];
                    float dy = s * cb[b] + c * sb[b];
                    float ex = x + z[b] * dx;
                    float ey = y + z[b] * dy;
                    int ci = (int)floorf(ex / res) + i;
                    int cj = (int)floorf(ey / res) + j;
                    if (ci >= 0 && ci < W && cj >= 0 && cj < H)
                        sc += orc_evidence(belief[(int64_t)cj * W + ci]);
                }
                int64_t q = ((int64_t)(k + m) * side + (j + n)) * side + (i + n);
                score[q] = sc;
                if (sc > best) {
                    best = sc;
                    best_q = q;
                }
            }
    }
    int ib = (int)(best_q % side), jb = (int)((best_q / side) % side), kb = (int)(best_q / (side * side));
    int64_t second = 0;
    for (int64_t q = 0; q < (int64_t)nk * side * side; ++q) {
        int i = (int)(q % side), j = (int)((q / side) % side), k = (int)(q / (side * side));
        int d = abs(i - ib);
        if (abs(j - jb) > d) d = abs(j - jb);
        if (abs(k - kb) > d) d = abs(k - kb);
        if (d > sep && score[q] > second)
            second = score[q];
    }
    double norm = nret > 0 ? (double)best / (255.0 * (double)nret) : 0.0;
    double margin = best > 0 ? (double)(best - second) / (double)best : 0.0;
    match[0] = (float)norm;
    match[1] = (float)margin;
    match[2] = (float)(norm * margin);
    scores[0] = best;
    scores[1] = second;
    scores[2] = best_q;
    const float pi_f = (float)3.14159265358979323846;
    const float two_pi_f = (float)(2.0 * 3.14159265358979323846);
    float tho = th + (float)(kb - m) * dth;
    if (tho >= pi_f) tho = tho - two_pi_f;
    if (tho < -pi_f) tho = tho + two_pi_f;
    pose_out[0] = x + (float)(ib - n) * res;
    pose_out[1] = y + (float)(jb - n) * res;
    pose_out[2] = tho;
}

/* ---- fixed-lag window Gauss-Newton (Sec. III-D, Eq. 5-6) ------------------
 *
 * Poses x_i = (x, y, th), i = 0..L-1.  Factors (this project's reading of the
 * sliding-window pose graph):
 *   prior      r = x_0 - p (angle wrapped), information diag(wp)
 *   odometry   r = (R(th_i)^T (t_{i+1} - t_i) - u_xy, wrap(th_{i+1} - th_i - u_th)),
 *              information diag(wo)
 *   unary      r = x_i - z_i (angle wrapped), information diag(wm_i) (0: none)
 * Gauss-Newton: H = sum J^T W J, g = sum J^T W r, H d = -g solved densely,
 * x <- x + d (angles wrapped).  After the iterations, Sigma_last = the last
 * 3x3 block of H^-1 at the final estimate (Eq. 6). */
static double orc_wrap(double a)
{
    const double pi = 3.14159265358979323846;
    for (int q = 0; q < 64 && a >= pi; ++q) a -= 2.0 * pi;
    for (int q = 0; q < 64 && a < -pi; ++q) a += 2.0 * pi;
    return a;
}

/* In-place Gauss-Jordan inverse of the n x n matrix A (partial pivoting). */
static int orc_invert(double *A, double *Ainv, int n)
{
    for (int i = 0; i < n * n; ++i)
        Ainv[i] = 0.0;
    for (int i = 0; i < n; ++i)
        Ainv[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c]))
                piv = r;
        if (A[piv * n + c] == 0.0)
            return -1;
        for (int k = 0; k < n; ++k) {
            double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
            t = Ainv[c * n + k]; Ainv[c * n + k] = Ainv[piv * n + k]; Ainv[piv * n + k] = t;
        }
        double d = A[c * n + c];
        for (int k = 0; k < n; ++k) {
            A[c * n + k] /= d;
            Ainv[c * n + k] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c)
                continue;
            double f = A[r * n + c];
            if (f == 0.0)
                continue;
            for (int k = 0; k < n; ++k) {
                A[r * n + k] -= f * A[c * n + k];
                Ainv[r * n + k] -= f * Ainv[c * n + k];
            }
        }
    }
    return 0;
}

/* One env.  x [L*3] in/out; odo [(L-1)*3]; meas [L*3]; wm [L*3]; prior [3];
 * wp [3]; wo [3]; cov_last [9] out.  Returns 0, or -1 if H is singular. */
int orc_fixed_lag_gn(int L, int iters, double *x, const double *odo, const double *meas,
                     const double *wm, const double *prior, const double *wp, const double *wo,
                     double *cov_last)
{
    enum { NMAX = 48 };
    const int n = 3 * L;
    if (L < 1 || n > NMAX)
        return -1;
    double H[NMAX * NMAX], Hi[NMAX * NMAX], g[NMAX];
    for (int it = 0; it <= iters; ++it) {
        for (int i = 0; i < n * n; ++i)
            H[i] = 0.0;
        for (int i = 0; i < n; ++i)
            g[i] = 0.0;
        /* prior and unary factors: J = I on the pose's block */
        for (int i = 0; i < L; ++i) {
            const double *z = i == 0 ? prior : NULL;
            for (int pass = 0; pass < 2; ++pass) {
                const double *zz = pass == 0 ? z : meas + 3 * i;
                const double *w = pass == 0 ? wp : wm + 3 * i;
                if (!zz)
                    continue;
                double r[3] = {x[3 * i] - zz[0], x[3 * i + 1] - zz[1],
                               orc_wrap(x[3 * i + 2] - zz[2])};
                for (int a = 0; a < 3; ++a) {
                    H[(3 * i + a) * n + 3 * i + a] += w[a];
                    g[3 * i + a] += w[a] * r[a];
                }
            }
        }
        /* odometry factors */
        for (int i = 0; i + 1 < L; ++i) {
            const double th = x[3 * i + 2], c = cos(th), s = sin(th);
            const double dx = x[3 * i + 3] - x[3 * i], dy = x[3 * i + 4] - x[3 * i + 1];
            double r[3] = {c * dx + s * dy - odo[3 * i], -s * dx + c * dy - odo[3 * i + 1],
                           orc_wrap(x[3 * i + 5] - th - odo[3 * i + 2])};
            /* J over (x_i, x_{i+1}): 3 x 6 */
            double J[3][6] = {
                {-c, -s, -s * dx + c * dy, c, s, 0.0},
                {s, -c, -c * dx - s * dy, -s, c, 0.0},
                {0.0, 0.0, -1.0, 0.0, 0.0, 1.0}};
            for (int a = 0; a < 6; ++a) {
                int ia = 3 * i + a;
                for (int b = 0; b < 6; ++b) {
                    int ib = 3 * i + b;
                    double v = 0.0;
                    for (int q = 0; q < 3; ++q)
                        v += J[q][a] * wo[q] * J[q][b];
                    H[ia * n + ib] += v;
                }
                double v = 0.0;
                for (int q = 0; q < 3; ++q)
                    v += J[q][a] * wo[q] * r[q];
                g[ia] += v;
            }
        }
        double Hc[NMAX * NMAX];
        memcpy(Hc, H, sizeof(double) * (size_t)(n * n));
        if (orc_invert(Hc, Hi, n) != 0)
            return -1;
        if (it == iters)
            break;
        for (int a = 0; a < n; ++a) {
            double d = 0.0;
            for (int b = 0; b < n; ++b)
                d -= Hi[a * n + b] * g[b];
            x[a] += d;
        }
        for (int i = 0; i < L; ++i)
            x[3 * i + 2] = orc_wrap(x[3 * i + 2]);
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            cov_last[3 * a + b] = Hi[(n - 3 + a) * n + (n - 3 + b)];
    return 0;
}
