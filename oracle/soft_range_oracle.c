/*
 * soft_range_oracle.c -- plain fp64 CPU oracle of the differentiable soft
 * expected-range raycaster and of batched scan-to-map Gauss-Newton
 * (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA path).
 *
 * Soft range of one beam from pose (x, y, th) at beam angle beta:
 *   samples s_k = (k+1)*ds, k = 0..K-1, at q_k = (x, y) + s_k (cos phi, sin phi),
 *   phi = th + beta;
 *   l_k = bilinear interpolation of the log-odds grid on cell centres
 *         (clamp-to-edge outside the map);   p_k = 1 / (1 + exp(-l_k));
 *   T_0 = 1, T_{k+1} = T_k (1 - p_k)         (transmittance);
 *   r = sum_k T_k p_k s_k + T_K * K*ds        (no return: K*ds).
 * Reverse-mode derivative (adjoint): with R_K = K*ds and
 *   R_k = p_k s_k + (1 - p_k) R_{k+1}  (expected range given the beam
 * reached sample k), dr/dp_k = T_k (s_k - R_{k+1}); then
 *   dr/dl_k = dr/dp_k * p_k (1 - p_k), spread over the four bilinear
 *   corners, and through q_k to (x, y, th).
 * Gauss-Newton (Sec. III-D, Eq. 5) on the residuals e_b = r_b(xi) - z_b:
 *   xi <- xi - (J^T J + mu I)^{-1} J^T e, J_b = dr_b/dxi;
 * the inverse of the damped normal matrix is the pose covariance block of
 * Eq. 6 up to the range variance sigma^2.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int32_t W, H, B, K;
    double res, ds, fov;
} orc_soft_cfg;

static double orc_soft_beam_angle(const orc_soft_cfg *c, int b)
{
    const double two_pi = 2.0 * 3.14159265358979323846;
    if (c->fov <= 0.0 || c->fov >= two_pi - 1e-9)
        return (two_pi * (double)b) / (double)c->B;
    if (c->B == 1)
        return 0.0;
    return -0.5 * c->fov + ((double)b * c->fov) / (double)(c->B - 1);
}

static int orc_clampi(int v, int lo, int hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Bilinear log-odds at (px, py) metres and its gradient in metres^-1.
 * The four corner cells and weights are returned for the map adjoint. */
static double orc_bilinear(const orc_soft_cfg *c, const float *L, double px, double py,
                           double *gx, double *gy, int idx[4], double w[4])
{
    double u = px / c->res - 0.5, v = py / c->res - 0.5;
    double fu = floor(u), fv = floor(v);
    double ax = u - fu, ay = v - fv;
    int i0 = (int)fu, j0 = (int)fv;
    int ia = orc_clampi(i0, 0, c->W - 1), ib = orc_clampi(i0 + 1, 0, c->W - 1);
    int ja = orc_clampi(j0, 0, c->H - 1), jb = orc_clampi(j0 + 1, 0, c->H - 1);
    double l00 = L[ja * c->W + ia], l10 = L[ja * c->W + ib];
    double l01 = L[jb * c->W + ia], l11 = L[jb * c->W + ib];
    idx[0] = ja * c->W + ia; w[0] = (1 - ax) * (1 - ay);
    idx[1] = ja * c->W + ib; w[1] = ax * (1 - ay);
    idx[2] = jb * c->W + ia; w[2] = (1 - ax) * ay;
    idx[3] = jb * c->W + ib; w[3] = ax * ay;
    *gx = ((1 - ay) * (l10 - l00) + ay * (l11 - l01)) / c->res;
    *gy = ((1 - ax) * (l01 - l00) + ax * (l11 - l10)) / c->res;
    return w[0] * l00 + w[1] * l10 + w[2] * l01 + w[3] * l11;
}

/* Soft range of beam b; if grad_pose != NULL adds gr * dr/d(x, y, th) to it,
 * if grad_map != NULL adds gr * dr/dL to it. */
double orc_soft_range(const orc_soft_cfg *c, const float *L, double x, double y, double th,
                      int b, double gr, double *grad_pose, double *grad_map)
{
    enum { KMAX = 1024 };
    double p[KMAX], T[KMAX + 1], gxk[KMAX], gyk[KMAX], s[KMAX], wk[KMAX][4];
    int ik[KMAX][4];
    const int K = c->K < KMAX ? c->K : KMAX;
    const double phi = th + orc_soft_beam_angle(c, b);
    const double cp = cos(phi), sp = sin(phi);
    const double r_far = (double)K * c->ds;
    double r = 0.0;
    T[0] = 1.0;
    for (int k = 0; k < K; ++k) {
        s[k] = (double)(k + 1) * c->ds;
        double l = orc_bilinear(c, L, x + s[k] * cp, y + s[k] * sp, &gxk[k], &gyk[k], ik[k], wk[k]);
        p[k] = 1.0 / (1.0 + exp(-l));
        r += T[k] * p[k] * s[k];
        T[k + 1] = T[k] * (1.0 - p[k]);
    }
    r += T[K] * r_far;
    if (!grad_pose && !grad_map)
        return r;
    double R = r_far;                         /* R_{k+1} while walking back */
    for (int k = K - 1; k >= 0; --k) {
        double dr_dp = T[k] * (s[k] - R);
        double dr_dl = gr * dr_dp * p[k] * (1.0 - p[k]);
        if (grad_map)
            for (int q = 0; q < 4; ++q)
                grad_map[ik[k][q]] += dr_dl * wk[k][q];
        if (grad_pose) {
            grad_pose[0] += dr_dl * gxk[k];
            grad_pose[1] += dr_dl * gyk[k];
            grad_pose[2] += dr_dl * (gxk[k] * (-s[k] * sp) + gyk[k] * (s[k] * cp));
        }
        R = p[k] * s[k] + (1.0 - p[k]) * R;
    }
    return r;
}

/* Gauss-Newton scan-to-map correction of one pose (Eq. 5) with `iters`
 * damped steps; writes the final pose and the damped normal matrix
 * A = J^T J + mu I at the final pose (row-major 3x3). */
void orc_gn(const orc_soft_cfg *c, const float *L, const double pose_in[3], const float *z,
            int iters, double mu, double pose_out[3], double A_out[9])
{
    double xi[3] = {pose_in[0], pose_in[1], pose_in[2]};
    for (int it = 0; it <= iters; ++it) {
        double A[9] = {0}, g[3] = {0};
        for (int b = 0; b < c->B; ++b) {
            double J[3] = {0, 0, 0};
            double r = orc_soft_range(c, L, xi[0], xi[1], xi[2], b, 1.0, J, NULL);
            double e = r - (double)z[b];
            for (int i = 0; i < 3; ++i) {
                g[i] += J[i] * e;
                for (int j = 0; j < 3; ++j)
                    A[3 * i + j] += J[i] * J[j];
            }
        }
        for (int i = 0; i < 3; ++i)
            A[4 * i] += mu;
        if (it == iters) {
            memcpy(A_out, A, sizeof(A));
            break;
        }
        /* solve A d = -g by Cramer's rule (3x3) */
        double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
        double d[3];
        for (int col = 0; col < 3; ++col) {
            double M[9];
            memcpy(M, A, sizeof(M));
            for (int row = 0; row < 3; ++row)
                M[3 * row + col] = -g[row];
            d[col] = (M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                      M[2] * (M[3] * M[7] - M[4] * M[6])) / det;
        }
        for (int i = 0; i < 3; ++i)
            xi[i] += d[i];
    }
    pose_out[0] = xi[0];
    pose_out[1] = xi[1];
    pose_out[2] = xi[2];
}

/* Batched helpers: E envs of identical W x H grids (env e at L + e*W*H). */
void orc_soft_ranges(const orc_soft_cfg *c, const float *L, const double *pose, int E,
                     const double *gr, double *ranges, double *grad_pose, double *grad_map)
{
    const int64_t n = (int64_t)c->W * c->H;
    for (int e = 0; e < E; ++e)
        for (int b = 0; b < c->B; ++b) {
            double g = gr ? gr[(int64_t)e * c->B + b] : 1.0;
            ranges[(int64_t)e * c->B + b] = orc_soft_range(
                c, L + e * n, pose[3 * e], pose[3 * e + 1], pose[3 * e + 2], b, g,
                grad_pose ? grad_pose + 3 * e : NULL, grad_map ? grad_map + e * n : NULL);
        }
}

void orc_gn_batch(const orc_soft_cfg *c, const float *L, const double *pose_in, const float *z,
                  int E, int iters, double mu, double *pose_out, double *A_out)
{
    const int64_t n = (int64_t)c->W * c->H;
    for (int e = 0; e < E; ++e)
        orc_gn(c, L + e * n, pose_in + 3 * e, z + (int64_t)e * c->B, iters, mu,
               pose_out + 3 * e, A_out + 9 * e);
}

/* Per-beam Jacobian dr_b/d(x, y, th) [E, B, 3] by the adjoint, one beam at a time. */
void orc_soft_jacobian(const orc_soft_cfg *c, const float *L, const double *pose, int E,
                       double *ranges, double *jac)
{
    const int64_t n = (int64_t)c->W * c->H;
    for (int e = 0; e < E; ++e)
        for (int b = 0; b < c->B; ++b) {
            double *J = jac + 3 * ((int64_t)e * c->B + b);
            J[0] = J[1] = J[2] = 0.0;
            ranges[(int64_t)e * c->B + b] = orc_soft_range(
                c, L + e * n, pose[3 * e], pose[3 * e + 1], pose[3 * e + 2], b, 1.0, J, NULL);
        }
}
