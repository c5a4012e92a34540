// slam2d.cu -- the SLAM backbone inside the 2-D step (Sec. III-D): pose
// prediction from odometry, correlative scan matching of this step's scan
// against the map before it is integrated, and a sliding fixed-lag window
// solved by Gauss-Newton, whose newest-pose marginal covariance gives U_t.
//
// Runs between the sensing and the update kernels:
//   slam_predict2d_kernel  one thread per env: window restart on reset, the
//                          odometry (v dt, 0, w dt) of this step and the pose
//                          predicted from the window's newest estimate;
//   csm2d_kernel           the batched scan matcher (csm2d.cu);
//   slam_window2d_kernel   one half-warp per env: slide the window, append the
//                          predicted pose, the odometry factor and the match
//                          (information w * meas_info), anchor the oldest
//                          pose at its current estimate, run window_gn_half
//                          in fp64, write Sigma_t and U_t, and the weight of
//                          this scan's map update: the normalised match
//                          score, or 1 for an episode's first scan (known
//                          pose, nothing to match against yet).
#include <cmath>

#include "aslam_internal.cuh"
#include "env_common.cuh"
#include "window_gn.cuh"

namespace aslam {
namespace {

__device__ __forceinline__ float wrap_f(float th) {
    const float pi_f = (float)3.14159265358979323846;
    const float two_pi_f = (float)(2.0 * 3.14159265358979323846);
    if (th >= pi_f) th = fsub(th, two_pi_f);
    if (th < -pi_f) th = fadd(th, two_pi_f);
    return th;
}

__global__ void slam_predict2d_kernel(const Step2DParams p) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.E; e += gridDim.x * blockDim.x) {
        const bool reset = p.done[e] != 0;           // reset at the start of this step
        if (reset) p.win_n[e] = 0;
        const int n = p.win_n[e];
        const float v = fminf(fmaxf(p.actions[2 * e], 0.0f), p.v_max);
        const float w = fminf(fmaxf(p.actions[2 * e + 1], -p.w_max), p.w_max);
        const float ux = fmul(v, p.dt), uth = fmul(w, p.dt);
        float px, py, pth;
        if (n == 0) {
            // a fresh window starts from the known pose: this step's start
            const EnvStart &st = reinterpret_cast<const EnvSense *>(p.env_sense)[e].start;
            px = st.x;
            py = st.y;
            pth = st.th;
        } else {
            const float *last = p.win_x + ((long long)e * p.slam_L + n - 1) * 3;
            float s, c;
            det_sincos(last[2], s, c);
            px = fadd(last[0], fmul(c, ux));
            py = fadd(last[1], fmul(s, ux));
            pth = wrap_f(fadd(last[2], uth));
        }
        p.slam_pred[3 * e] = px;
        p.slam_pred[3 * e + 1] = py;
        p.slam_pred[3 * e + 2] = pth;
        p.slam_odo[3 * e] = ux;
        p.slam_odo[3 * e + 1] = 0.0f;
        p.slam_odo[3 * e + 2] = uth;
    }
}

constexpr int kWinEnvs = 8;      // envs per CTA of the window kernel, two per warp

__global__ void __launch_bounds__(16 * kWinEnvs) slam_window2d_kernel(const Step2DParams p) {
    __shared__ WgnShared s_ws[kWinEnvs];
    __shared__ float s_prior[kWinEnvs][3];
    const int g = threadIdx.x >> 4, lane = threadIdx.x & 15;      // the env's half-warp
    const unsigned hm = 0xffffu << (threadIdx.x & 16);
    const int e = blockIdx.x * kWinEnvs + g;
    if (e >= p.E) return;                            // uniform over the half-warp
    const int L = p.slam_L;
    const long long w0 = (long long)e * L * 3;
    float *x = p.win_x + w0, *odo = p.win_odo + w0, *meas = p.win_meas + w0;
    float *minfo = p.win_minfo + w0;
    int n = p.win_n[e];
    if (n == L) {
        // slide: drop the oldest pose and the odometry factor behind it (lane
        // i moves entry i+1 to i; every read precedes every write; L <= 16)
        float xs[3], ms[3], is[3], os[3];
        const bool mv = lane + 1 < L, mvo = lane + 2 < L;
        for (int q = 0; q < 3; ++q) {
            if (mv) {
                xs[q] = x[3 * lane + 3 + q];
                ms[q] = meas[3 * lane + 3 + q];
                is[q] = minfo[3 * lane + 3 + q];
            }
            if (mvo) os[q] = odo[3 * lane + 3 + q];
        }
        __syncwarp(hm);
        for (int q = 0; q < 3; ++q) {
            if (mv) {
                x[3 * lane + q] = xs[q];
                meas[3 * lane + q] = ms[q];
                minfo[3 * lane + q] = is[q];
            }
            if (mvo) odo[3 * lane + q] = os[q];
        }
        n = L - 1;
    }
    __syncwarp(hm);
    // the first scan of an episode: the pose is known, the map it would be
    // matched against is empty (or stale): no pose factor, full weight
    const bool first = n == 0;
    const float wgt = first ? 0.0f : p.csm_match[3 * e + 2];
    if (lane == 0) p.slam_upd_w[e] = first ? 1.0f : p.csm_match[3 * e];
    if (lane < 3) {
        x[3 * n + lane] = p.slam_pred[3 * e + lane];
        meas[3 * n + lane] = p.csm_pose[3 * e + lane];
        minfo[3 * n + lane] = fmul(wgt, p.slam_meas_info[lane]);
        if (n > 0) odo[3 * (n - 1) + lane] = p.slam_odo[3 * e + lane];
    }
    ++n;
    if (lane == 0) p.win_n[e] = n;
    __syncwarp(hm);
    if (lane < 3) s_prior[g][lane] = x[lane];     // the oldest pose's current estimate
    __syncwarp(hm);
    WgnShared *ws = &s_ws[g];
    const bool ok = window_gn_half(n, p.slam_iters, p.slam_wo, x, odo, meas, minfo, s_prior[g],
                                   p.slam_prior_info, ws);
    if (lane == 0) {
        const double *Sl = ws->Si[n - 1];
        double *S = p.pose_cov + 6 * (long long)e;
        S[0] = ok ? Sl[0] : NAN;
        S[1] = ok ? 0.5 * (Sl[1] + Sl[3]) : NAN;
        S[2] = ok ? 0.5 * (Sl[2] + Sl[6]) : NAN;
        S[3] = ok ? Sl[4] : NAN;
        S[4] = ok ? 0.5 * (Sl[5] + Sl[7]) : NAN;
        S[5] = ok ? Sl[8] : NAN;
        p.u_scan[e] = ok ? (float)(cbrt(wgn::det3(Sl)) / p.uq_scale) : NAN;
        if (!ok) atomicOr(p.err, kErrChecks);          // singular window (never with a prior)
    }
}

}  // namespace

cudaError_t launch_slam2d(const Step2DParams &p, cudaStream_t s, const cudaEvent_t *ev) {
    const int grid = (p.E + 127) / 128;
    slam_predict2d_kernel<<<grid, 128, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], s);
    if (e != cudaSuccess) return e;
    e = launch_csm2d(p, p.csm_n_xy, p.csm_n_th, p.csm_sep, p.csm_dth, p.csm_map_bytes, p.csm_ws,
                     p.slam_pred, p.z, p.csm_pose, p.csm_match, p.csm_scores, true, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    if (e != cudaSuccess) return e;
    // one half-warp per env, few per CTA: the fp64 window solves spread over every
    // SM (the fp64 rate of one SM is small)
    slam_window2d_kernel<<<(p.E + kWinEnvs - 1) / kWinEnvs, 16 * kWinEnvs, 0, s>>>(p);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    return e;
}

}  // namespace aslam
