// window_gn.cuh -- the fixed-lag window Gauss-Newton solver shared by the
// batched entry point (flgn.cu) and the in-step SLAM backbone (slam2d.cu),
// one half-warp per window.
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

// Per-window workspace of window_gn_half (shared memory).
struct WgnShared {
    double x[kMaxWindow][3];     // estimates (fp64 between passes)
    double D[kMaxWindow][9];     // diagonal blocks of the normal matrix
    double C[kMaxWindow][9];     // off-diagonal block of factor (i, i+1): Ja^T W Jb
    double g[kMaxWindow][3];     // gradient J^T W r
    double Si[kMaxWindow][9];    // inverse Schur complements S_i^-1
    double r[kMaxWindow][3];     // eliminated right-hand sides
    double M[9], S[9], R[9];     // per-step scratch
    double v[3], d[3];
};

// One window, solved by the 16 lanes of a half-warp together (two windows
// per warp: sm_103a's fp64 pipe takes a warp instruction whatever its
// active lanes, so the two halves share each one): x [L*3] fp32
// in/out (oldest first), odo [(L-1)*3], meas and meas_info [L*3], prior and
// prior_info [3].  The Gauss-Newton normal matrix is block tridiagonal (3x3
// blocks).  Each pass:
//   * lanes 0..L-1 linearize their pose in parallel: the prior (pose 0), the
//     pose factor, the odometry factor behind (i-1, i) and the one ahead
//     (i, i+1), giving D_i, g_i and the off-diagonal block C_i;
//   * the block elimination S_0 = D_0, S_i = D_i - C_{i-1}^T S_{i-1}^-1
//     C_{i-1} runs over the poses in order with lane (p, q) < 9 holding
//     entry (p, q) of each 3x3 product and of the adjugate inverse;
//   * back substitution d_{L-1} = S^-1 r, d_i = S_i^-1 (r_i - C_i d_{i+1}) by
//     lanes 0..2.
// Each entry is the same sum of products, in the same order, as a
// one-thread solve; lanes only shorten the dependent chain, which sm_103a's
// fp64 latency makes the cost.  After the last pass ws->Si[L-1] (the inverse
// of the Schur complement left when every earlier pose is eliminated) is
// the newest pose's marginal covariance (Eq. 6).  Returns false (uniform
// over the half-warp) when a pivot block is singular; x then keeps the last
// estimate.  Every lane of the half-warp must call it.
static __device__ bool window_gn_half(int L, int iters, const double wo[3], float *xio,
                                      const float *odo, const float *meas,
                                      const float *meas_info, const float *prior,
                                      const float *prior_info, WgnShared *ws) {
    using namespace wgn;
    const int lane = threadIdx.x & 15;                   // lane within the half-warp
    const unsigned hm = 0xffffu << (threadIdx.x & 16);   // this half's lanes
    if (lane < L)
        for (int q = 0; q < 3; ++q) ws->x[lane][q] = (double)xio[3 * lane + q];
    __syncwarp(hm);
    // entry (p, q) of a 3x3 block for lanes < 9, and the adjugate's operands:
    // R[p][q] = S[q1][p1] S[q2][p2] - S[q1][p2] S[q2][p1], (k1, k2) = (k+1, k+2) mod 3
    const int ep = lane < 9 ? lane / 3 : 0, eq = lane < 9 ? lane % 3 : 0;
    const int p1 = (ep + 1) % 3, p2 = (ep + 2) % 3, q1 = (eq + 1) % 3, q2 = (eq + 2) % 3;
    bool ok = true;
    for (int it = 0; it <= iters && ok; ++it) {
        // ---- linearization, one lane per pose --------------------------------
        if (lane < L) {
            const int i = lane;
            double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0};
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 0 && i != 0) continue;
                const float *z = pass == 0 ? prior : meas + 3 * i;
                const float *w = pass == 0 ? prior_info : meas_info + 3 * i;
                const double rr[3] = {ws->x[i][0] - (double)z[0], ws->x[i][1] - (double)z[1],
                                      wrap_pi(ws->x[i][2] - (double)z[2])};
                for (int q = 0; q < 3; ++q) {
                    D[4 * q] += (double)w[q];
                    g[q] += (double)w[q] * rr[q];
                }
            }
            if (i > 0) {
                // the factor behind: Jb^T W Jb and Jb^T W r
                double rb[3], Ja[9], Jb[9];
                odo_factor(ws->x[i - 1], ws->x[i], odo + 3 * (i - 1), rb, Ja, Jb);
                for (int p = 0; p < 3; ++p) {
                    for (int q = 0; q < 3; ++q) {
                        double v = 0.0;
                        for (int k = 0; k < 3; ++k) v += Jb[3 * k + p] * wo[k] * Jb[3 * k + q];
                        D[3 * p + q] += v;
                    }
                    double v = 0.0;
                    for (int k = 0; k < 3; ++k) v += Jb[3 * k + p] * wo[k] * rb[k];
                    g[p] += v;
                }
            }
            double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (i + 1 < L) {
                // the factor ahead: Ja^T W Ja, Ja^T W r and C_i = Ja^T W Jb
                double r[3], Ja[9], Jb[9];
                odo_factor(ws->x[i], ws->x[i + 1], odo + 3 * i, r, Ja, Jb);
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
            }
            for (int q = 0; q < 9; ++q) {
                ws->D[i][q] = D[q];
                ws->C[i][q] = C[q];
            }
            for (int q = 0; q < 3; ++q) ws->g[i][q] = g[q];
        }
        __syncwarp(hm);
        // ---- block elimination, lane (p, q) per entry ------------------------
        for (int i = 0; i < L; ++i) {
            if (i == 0) {
                if (lane < 9) ws->S[lane] = ws->D[0][lane];
                if (lane < 3) ws->r[0][lane] = -ws->g[0][lane];
            } else {
                // M = C_{i-1}^T S_{i-1}^-1
                const double *Cp = ws->C[i - 1], *Sp = ws->Si[i - 1];
                if (lane < 9)
                    ws->M[lane] = Cp[ep] * Sp[eq] + Cp[3 + ep] * Sp[3 + eq] + Cp[6 + ep] * Sp[6 + eq];
                __syncwarp(hm);
                // S_i = D_i - M C_{i-1};  r_i = -g_i - M r_{i-1}
                const double *M = ws->M;
                if (lane < 9)
                    ws->S[lane] = ws->D[i][lane] -
                                  (M[3 * ep] * Cp[eq] + M[3 * ep + 1] * Cp[3 + eq] +
                                   M[3 * ep + 2] * Cp[6 + eq]);
                if (lane < 3) {
                    const double *rp = ws->r[i - 1];
                    ws->r[i][lane] = -ws->g[i][lane] -
                                     (M[3 * lane] * rp[0] + M[3 * lane + 1] * rp[1] +
                                      M[3 * lane + 2] * rp[2]);
                }
            }
            __syncwarp(hm);
            // S_i^-1: adjugate entry per lane, one reciprocal of the determinant
            const double *S = ws->S;
            if (lane < 9) ws->R[lane] = S[3 * q1 + p1] * S[3 * q2 + p2] - S[3 * q1 + p2] * S[3 * q2 + p1];
            __syncwarp(hm);
            const double *R = ws->R;
            const double det = S[0] * R[0] + S[1] * R[3] + S[2] * R[6];
            ok = det != 0.0 && isfinite(det);
            if (!ok) break;                              // uniform over the half
            const double id = 1.0 / det;
            if (lane < 9) ws->Si[i][lane] = R[lane] * id;
            __syncwarp(hm);
        }
        if (!ok || it == iters) break;
        // ---- back substitution, lanes 0..2 ------------------------------------
        for (int i = L - 1; i >= 0; --i) {
            if (lane < 3) {
                double v = ws->r[i][lane];
                if (i + 1 < L) {
                    const double *Ci = ws->C[i];
                    v -= Ci[3 * lane] * ws->d[0] + Ci[3 * lane + 1] * ws->d[1] +
                         Ci[3 * lane + 2] * ws->d[2];
                }
                ws->v[lane] = v;
            }
            __syncwarp(hm);
            if (lane < 3) {
                const double *Sii = ws->Si[i];
                const double dd = Sii[3 * lane] * ws->v[0] + Sii[3 * lane + 1] * ws->v[1] +
                                  Sii[3 * lane + 2] * ws->v[2];
                ws->d[lane] = dd;
                ws->x[i][lane] = lane == 2 ? wrap_pi(ws->x[i][2] + dd) : ws->x[i][lane] + dd;
            }
            __syncwarp(hm);
        }
    }
    __syncwarp(hm);
    if (lane < L)
        for (int q = 0; q < 3; ++q) xio[3 * lane + q] = (float)ws->x[lane][q];
    __syncwarp(hm);
    return ok;
}

}  // namespace aslam
