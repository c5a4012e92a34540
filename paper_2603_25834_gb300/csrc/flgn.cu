// flgn.cu -- batched fixed-lag window Gauss-Newton (Sec. III-D, Eq. 5-6) on
// sm_103a: one half-warp per env runs window_gn_half (window_gn.cuh) in fp64 and
// reports the newest pose's marginal covariance and U = det^(1/3) / scale.
#include <cmath>

#include "aslam_internal.cuh"
#include "window_gn.cuh"

namespace aslam {
namespace {

struct FlgnArgs {
    int E, L, iters;
    double wo[3];
    double u_scale;
    float *x;
    const float *odo, *meas, *meas_info, *prior, *prior_info;
    float *cov, *u;
    int *status;
};

constexpr int kEnvsPerCta = 8;   // two per warp

__global__ void __launch_bounds__(16 * kEnvsPerCta) flgn_kernel(const FlgnArgs a) {
    __shared__ WgnShared s_ws[kEnvsPerCta];
    const int g = threadIdx.x >> 4, lane = threadIdx.x & 15;
    const int e = blockIdx.x * kEnvsPerCta + g;
    if (e >= a.E) return;                            // uniform over the half-warp
    const int L = a.L;
    const long long w = (long long)e * L * 3;
    WgnShared *ws = &s_ws[g];
    const bool ok = window_gn_half(L, a.iters, a.wo, a.x + w, a.odo + (long long)e * (L - 1) * 3,
                                   a.meas + w, a.meas_info + w, a.prior + 3 * (long long)e,
                                   a.prior_info + 3 * (long long)e, ws);
    const double *Sl = ws->Si[L - 1];
    if (a.cov && lane < 9) a.cov[9 * (long long)e + lane] = ok ? (float)Sl[lane] : NAN;
    if (lane == 0) {
        if (a.status) a.status[e] = ok ? 0 : 1;
        if (a.u) a.u[e] = ok ? (float)(cbrt(wgn::det3(Sl)) / a.u_scale) : NAN;
    }
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
    // one half-warp per env, few per CTA: the fp64 solves spread over every SM
    flgn_kernel<<<(E + kEnvsPerCta - 1) / kEnvsPerCta, 16 * kEnvsPerCta, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace aslam
