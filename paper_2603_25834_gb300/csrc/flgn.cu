// flgn.cu -- batched fixed-lag window Gauss-Newton (Sec. III-D, Eq. 5-6) on
// sm_103a.
//
// Per env a window of L planar poses x_i = (x, y, th) with a prior factor on
// x_0, odometry factors between consecutive poses,
//   r = (R(th_i)^T (t_{i+1} - t_i) - u_xy, wrap(th_{i+1} - th_i - u_th)),
// and optional absolute pose factors r = x_i - z_i (e.g. correlative scan
// matches), each with a diagonal information.  The Gauss-Newton normal
// matrix is block tridiagonal (3x3 blocks); one thread per env eliminates
// it block by block in fp64 (S_0 = D_0, S_i = D_i - C_{i-1}^T S_{i-1}^-1 C_{i-1})
// and substitutes back.  After the last iteration S_{L-1}^-1 -- the inverse
// of the Schur complement left when every earlier pose is eliminated -- is
// the marginal covariance of the newest pose (Eq. 6, "last block").
#include <cmath>

#include "aslam_internal.cuh"

namespace aslam {
namespace {

constexpr int kMaxWindow = 16;
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

// Adjugate inverse; false when singular.
__device__ __forceinline__ bool inv3(const double *M, double *R) {
    const double d = det3(M);
    if (!(d != 0.0) || !isfinite(d)) return false;
    R[0] = (M[4] * M[8] - M[5] * M[7]) / d;
    R[1] = (M[2] * M[7] - M[1] * M[8]) / d;
    R[2] = (M[1] * M[5] - M[2] * M[4]) / d;
    R[3] = (M[5] * M[6] - M[3] * M[8]) / d;
    R[4] = (M[0] * M[8] - M[2] * M[6]) / d;
    R[5] = (M[2] * M[3] - M[0] * M[5]) / d;
    R[6] = (M[3] * M[7] - M[4] * M[6]) / d;
    R[7] = (M[1] * M[6] - M[0] * M[7]) / d;
    R[8] = (M[0] * M[4] - M[1] * M[3]) / d;
    return true;
}

__device__ __forceinline__ void mul3(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

struct FlgnArgs {
    int E, L, iters;
    double wo[3];
    double u_scale;
    float *x;
    const float *odo, *meas, *meas_info, *prior, *prior_info;
    float *cov, *u;
    int *status;
};

__global__ void flgn_kernel(const FlgnArgs a) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E) return;
    const int L = a.L;
    double x[kMaxWindow][3], D[kMaxWindow][9], C[kMaxWindow][9], g[kMaxWindow][3];
    double S[kMaxWindow][9], Si[kMaxWindow][9], r[kMaxWindow][3];
    for (int i = 0; i < L; ++i)
        for (int q = 0; q < 3; ++q) x[i][q] = (double)a.x[((long long)e * L + i) * 3 + q];
    bool ok = true;
    for (int it = 0; it <= a.iters && ok; ++it) {
        for (int i = 0; i < L; ++i) {
            for (int q = 0; q < 9; ++q) D[i][q] = C[i][q] = 0.0;
            g[i][0] = g[i][1] = g[i][2] = 0.0;
        }
        // prior on x_0, unary factors on every pose (J = I)
        for (int i = 0; i < L; ++i) {
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 0 && i != 0) continue;
                const float *z = pass == 0 ? a.prior + 3 * (long long)e
                                           : a.meas + ((long long)e * L + i) * 3;
                const float *w = pass == 0 ? a.prior_info + 3 * (long long)e
                                           : a.meas_info + ((long long)e * L + i) * 3;
                const double rr[3] = {x[i][0] - (double)z[0], x[i][1] - (double)z[1],
                                      wrap_pi(x[i][2] - (double)z[2])};
                for (int q = 0; q < 3; ++q) {
                    D[i][4 * q] += (double)w[q];
                    g[i][q] += (double)w[q] * rr[q];
                }
            }
        }
        // odometry factors: J = [Ja | Jb] over (x_i, x_{i+1})
        for (int i = 0; i + 1 < L; ++i) {
            const double th = x[i][2], c = cos(th), s = sin(th);
            const double dx = x[i + 1][0] - x[i][0], dy = x[i + 1][1] - x[i][1];
            const float *u = a.odo + ((long long)e * (L - 1) + i) * 3;
            const double rr[3] = {c * dx + s * dy - (double)u[0], -s * dx + c * dy - (double)u[1],
                                  wrap_pi(x[i + 1][2] - th - (double)u[2])};
            const double Ja[3][3] = {{-c, -s, -s * dx + c * dy}, {s, -c, -c * dx - s * dy},
                                     {0.0, 0.0, -1.0}};
            const double Jb[3][3] = {{c, s, 0.0}, {-s, c, 0.0}, {0.0, 0.0, 1.0}};
            for (int p = 0; p < 3; ++p) {
                for (int q = 0; q < 3; ++q) {
                    double daa = 0.0, dbb = 0.0, dab = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        daa += Ja[k][p] * a.wo[k] * Ja[k][q];
                        dbb += Jb[k][p] * a.wo[k] * Jb[k][q];
                        dab += Ja[k][p] * a.wo[k] * Jb[k][q];
                    }
                    D[i][3 * p + q] += daa;
                    D[i + 1][3 * p + q] += dbb;
                    C[i][3 * p + q] += dab;            // block (i, i+1)
                }
                double ga = 0.0, gb = 0.0;
                for (int k = 0; k < 3; ++k) {
                    ga += Ja[k][p] * a.wo[k] * rr[k];
                    gb += Jb[k][p] * a.wo[k] * rr[k];
                }
                g[i][p] += ga;
                g[i + 1][p] += gb;
            }
        }
        // forward elimination of H d = -g
        for (int q = 0; q < 9; ++q) S[0][q] = D[0][q];
        for (int q = 0; q < 3; ++q) r[0][q] = -g[0][q];
        ok = inv3(S[0], Si[0]);
        for (int i = 1; i < L && ok; ++i) {
            double Ct[9], M[9], MC[9];
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) Ct[3 * p + q] = C[i - 1][3 * q + p];
            mul3(Ct, Si[i - 1], M);                      // C^T S^-1
            mul3(M, C[i - 1], MC);
            for (int q = 0; q < 9; ++q) S[i][q] = D[i][q] - MC[q];
            for (int p = 0; p < 3; ++p)
                r[i][p] = -g[i][p] - (M[3 * p] * r[i - 1][0] + M[3 * p + 1] * r[i - 1][1] +
                                      M[3 * p + 2] * r[i - 1][2]);
            ok = inv3(S[i], Si[i]);
        }
        if (!ok || it == a.iters) break;
        // back substitution, then the update
        double d[kMaxWindow][3];
        for (int i = L - 1; i >= 0; --i) {
            double v[3] = {r[i][0], r[i][1], r[i][2]};
            if (i + 1 < L)
                for (int p = 0; p < 3; ++p)
                    v[p] -= C[i][3 * p] * d[i + 1][0] + C[i][3 * p + 1] * d[i + 1][1] +
                            C[i][3 * p + 2] * d[i + 1][2];
            for (int p = 0; p < 3; ++p)
                d[i][p] = Si[i][3 * p] * v[0] + Si[i][3 * p + 1] * v[1] + Si[i][3 * p + 2] * v[2];
        }
        for (int i = 0; i < L; ++i) {
            x[i][0] += d[i][0];
            x[i][1] += d[i][1];
            x[i][2] = wrap_pi(x[i][2] + d[i][2]);
        }
    }
    if (a.status) a.status[e] = ok ? 0 : 1;
    for (int i = 0; i < L; ++i)
        for (int q = 0; q < 3; ++q) a.x[((long long)e * L + i) * 3 + q] = (float)x[i][q];
    const double *Sl = Si[L - 1];
    if (a.cov)
        for (int q = 0; q < 9; ++q) a.cov[9 * (long long)e + q] = ok ? (float)Sl[q] : NAN;
    if (a.u) a.u[e] = ok ? (float)(cbrt(det3(Sl)) / a.u_scale) : NAN;
}

}  // namespace

int flgn_max_window() { return kMaxWindow; }

cudaError_t launch_flgn(int E, int L, int iters, const float *wo, float u_scale, float *x,
                        const float *odo, const float *meas, const float *meas_info,
                        const float *prior, const float *prior_info, float *cov, float *u,
                        int *status, cudaStream_t s) {
    FlgnArgs a;
    a.E = E;
    a.L = L;
    a.iters = iters;
    for (int q = 0; q < 3; ++q) a.wo[q] = (double)wo[q];
    a.u_scale = (double)u_scale;
    a.x = x;
    a.odo = odo;
    a.meas = meas;
    a.meas_info = meas_info;
    a.prior = prior;
    a.prior_info = prior_info;
    a.cov = cov;
    a.u = u;
    a.status = status;
    flgn_kernel<<<(E + 63) / 64, 64, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace aslam
