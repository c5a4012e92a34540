// window_gn.cuh -- the fixed-lag window Gauss-Newton solver shared by the
// batched entry point (flgn.cu) and the in-step SLAM backbone (slam2d.cu).
//
// A window of L planar poses x_i = (x, y, th) with a prior factor on x_0,
// odometry factors between consecutive poses,
//   r = (R(th_i)^T (t_{i+1} - t_i) - u_xy, wrap(th_{i+1} - th_i - u_th)),
// and absolute pose factors r = x_i - z_i, each with a diagonal
// information (Sec. III-D, Eq. 5).  The Gauss-Newton normal matrix is block
// tridiagonal (3x3 blocks); it is eliminated block by block in fp64
// (S_0 = D_0, S_i = D_i - C_{i-1}^T S_{i-1}^-1 C_{i-1}) and solved by back
// substitution.  After the last iteration S_{L-1}^-1 -- the inverse of the
// Schur complement left when every earlier pose is eliminated -- is the
// marginal covariance of the newest pose (Eq. 6, "last block").
#pragma once

#include <cmath>

namespace aslam {

constexpr int kMaxWindow = 16;

namespace wgn {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double wrap_pi(double a) {
    // bounded: inputs are angles within a few turns
    for (int q = 0; q < 64 && a >= kPi; ++q) a -= 2.0 * kPi;
    for (int q = 0; q < 64 && a < -kPi; ++q) a += 2.0 * kPi;
    return a;
}

__device__ __forceinline__ double det3(const double *M) {
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// Adjugate inverse (one reciprocal of the determinant); false when singular.
__device__ __forceinline__ bool inv3(const double *M, double *R) {
    const double d = det3(M);
    if (!(d != 0.0) || !isfinite(d)) return false;
    const double id = 1.0 / d;
    R[0] = (M[4] * M[8] - M[5] * M[7]) * id;
    R[1] = (M[2] * M[7] - M[1] * M[8]) * id;
    R[2] = (M[1] * M[5] - M[2] * M[4]) * id;
    R[3] = (M[5] * M[6] - M[3] * M[8]) * id;
    R[4] = (M[0] * M[8] - M[2] * M[6]) * id;
    R[5] = (M[2] * M[3] - M[0] * M[5]) * id;
    R[6] = (M[3] * M[7] - M[4] * M[6]) * id;
    R[7] = (M[1] * M[6] - M[0] * M[7]) * id;
    R[8] = (M[0] * M[4] - M[1] * M[3]) * id;
    return true;
}

__device__ __forceinline__ void mul3(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

}  // namespace wgn

// Residual and Jacobians (w.r.t. x_i and x_{i+1}) of the odometry factor
// between poses a and b with measured motion u.
__device__ __forceinline__ void odo_factor(const double *xa, const double *xb, const float *u,
                                           double r[3], double Ja[9], double Jb[9]) {
    using namespace wgn;
    double s, c;
    sincos(xa[2], &s, &c);
    const double dx = xb[0] - xa[0], dy = xb[1] - xa[1];
    r[0] = c * dx + s * dy - (double)u[0];
    r[1] = -s * dx + c * dy - (double)u[1];
    r[2] = wrap_pi(xb[2] - xa[2] - (double)u[2]);
    Ja[0] = -c; Ja[1] = -s; Ja[2] = -s * dx + c * dy;
    Ja[3] = s;  Ja[4] = -c; Ja[5] = -c * dx - s * dy;
    Ja[6] = 0.0; Ja[7] = 0.0; Ja[8] = -1.0;
    Jb[0] = c; Jb[1] = s; Jb[2] = 0.0;
    Jb[3] = -s; Jb[4] = c; Jb[5] = 0.0;
    Jb[6] = 0.0; Jb[7] = 0.0; Jb[8] = 1.0;
}

// One window: x [L*3] fp32 in/out (oldest first), odo [(L-1)*3], meas and
// meas_info [L*3], prior and prior_info [3].  Returns false when a pivot
// block is singular (x is then left at the last estimate); Sl receives the
// newest pose's marginal covariance.  The forward elimination streams over
// the poses with the running blocks in registers: at pose i the diagonal
// block D_i collects the prior (i = 0), the pose factor, the odometry factor
// behind (i-1, i) and the one ahead (i, i+1), whose off-diagonal block C_i
// is kept with S_i^-1 and the eliminated right-hand side for the back
// substitution.
static __device__ bool window_gn(int L, int iters, const double wo[3], float *xio,
                                 const float *odo, const float *meas, const float *meas_info,
                                 const float *prior, const float *prior_info, double Sl[9]) {
    using namespace wgn;
    double x[kMaxWindow][3];
    double Cs[kMaxWindow][9], Sis[kMaxWindow][9], rs[kMaxWindow][3];
    for (int i = 0; i < L; ++i)
        for (int q = 0; q < 3; ++q) x[i][q] = (double)xio[3 * i + q];
    bool ok = true;
    double Si_last[9];
    for (int it = 0; it <= iters && ok; ++it) {
        double Jb_prev[9], rb_prev[3];           // factor (i-1, i): its x_i Jacobian and residual
        double C_prev[9], Si_prev[9], r_prev[3];
        for (int i = 0; i < L && ok; ++i) {
            double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0};
            // prior (pose 0) and pose factors: J = I
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 0 && i != 0) continue;
                const float *z = pass == 0 ? prior : meas + 3 * i;
                const float *w = pass == 0 ? prior_info : meas_info + 3 * i;
                const double rr[3] = {x[i][0] - (double)z[0], x[i][1] - (double)z[1],
                                      wrap_pi(x[i][2] - (double)z[2])};
                for (int q = 0; q < 3; ++q) {
                    D[4 * q] += (double)w[q];
                    g[q] += (double)w[q] * rr[q];
                }
            }
            // the factor behind: Jb^T W Jb and Jb^T W r
            if (i > 0)
                for (int p = 0; p < 3; ++p) {
                    for (int q = 0; q < 3; ++q) {
                        double v = 0.0;
                        for (int k = 0; k < 3; ++k) v += Jb_prev[3 * k + p] * wo[k] * Jb_prev[3 * k + q];
                        D[3 * p + q] += v;
                    }
                    double v = 0.0;
                    for (int k = 0; k < 3; ++k) v += Jb_prev[3 * k + p] * wo[k] * rb_prev[k];
                    g[p] += v;
                }
            // the factor ahead: Ja^T W Ja, Ja^T W r and the block C_i = Ja^T W Jb
            double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (i + 1 < L) {
                double r[3], Ja[9], Jb[9];
                odo_factor(x[i], x[i + 1], odo + 3 * i, r, Ja, Jb);
                for (int p = 0; p < 3; ++p) {
                    for (int q = 0; q < 3; ++q) {
                        double daa = 0.0, dab = 0.0;
                        for (int k = 0; k < 3; ++k) {
                            daa += Ja[3 * k + p] * wo[k] * Ja[3 * k + q];
                            dab += Ja[3 * k + p] * wo[k] * Jb[3 * k + q];
                        }
                        D[3 * p + q] += daa;
                        C[3 * p + q] = dab;
                    }
                    double v = 0.0;
                    for (int k = 0; k < 3; ++k) v += Ja[3 * k + p] * wo[k] * r[k];
                    g[p] += v;
                }
                for (int q = 0; q < 9; ++q) Jb_prev[q] = Jb[q];
                for (int q = 0; q < 3; ++q) rb_prev[q] = r[q];
            }
            // eliminate: S_i = D_i - C_{i-1}^T S_{i-1}^-1 C_{i-1}, r_i = -g_i - C_{i-1}^T S_{i-1}^-1 r_{i-1}
            double S[9], r[3] = {-g[0], -g[1], -g[2]};
            for (int q = 0; q < 9; ++q) S[q] = D[q];
            if (i > 0) {
                double Ct[9], M[9], MC[9];
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q) Ct[3 * p + q] = C_prev[3 * q + p];
                mul3(Ct, Si_prev, M);
                mul3(M, C_prev, MC);
                for (int q = 0; q < 9; ++q) S[q] -= MC[q];
                for (int p = 0; p < 3; ++p)
                    r[p] -= M[3 * p] * r_prev[0] + M[3 * p + 1] * r_prev[1] + M[3 * p + 2] * r_prev[2];
            }
            double Si[9];
            ok = inv3(S, Si);
            for (int q = 0; q < 9; ++q) {
                Si_prev[q] = Si[q];
                C_prev[q] = C[q];
                Sis[i][q] = Si[q];
                Cs[i][q] = C[q];
            }
            for (int q = 0; q < 3; ++q) r_prev[q] = rs[i][q] = r[q];
            if (i == L - 1)
                for (int q = 0; q < 9; ++q) Si_last[q] = Si[q];
        }
        if (!ok || it == iters) break;
        // back substitution: d_{L-1} = S^-1 r, d_i = S_i^-1 (r_i - C_i d_{i+1})
        double dn[3] = {0.0, 0.0, 0.0};
        for (int i = L - 1; i >= 0; --i) {
            double v[3] = {rs[i][0], rs[i][1], rs[i][2]};
            if (i + 1 < L)
                for (int p = 0; p < 3; ++p)
                    v[p] -= Cs[i][3 * p] * dn[0] + Cs[i][3 * p + 1] * dn[1] + Cs[i][3 * p + 2] * dn[2];
            double d[3];
            for (int p = 0; p < 3; ++p)
                d[p] = Sis[i][3 * p] * v[0] + Sis[i][3 * p + 1] * v[1] + Sis[i][3 * p + 2] * v[2];
            x[i][0] += d[0];
            x[i][1] += d[1];
            x[i][2] = wrap_pi(x[i][2] + d[2]);
            dn[0] = d[0];
            dn[1] = d[1];
            dn[2] = d[2];
        }
    }
    for (int i = 0; i < L; ++i)
        for (int q = 0; q < 3; ++q) xio[3 * i + q] = (float)x[i][q];
    for (int q = 0; q < 9; ++q) Sl[q] = ok ? Si_last[q] : NAN;
    return ok;
}

}  // namespace aslam
