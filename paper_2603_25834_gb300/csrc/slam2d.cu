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
//   slam_correct2d_kernel  (slam_gn_iters > 0) one CTA per env: scan-to-map
//                          Gauss-Newton correction of the match on the soft
//                          expected-range model of the belief (Eq. 5);
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
#include "soft_model.cuh"
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

// Scan-to-map Gauss-Newton correction of the correlative match (Sec. III-D,
// Eq. 5), one CTA per env, threads over beams.  The model is the soft
// expected range of soft_model.cuh on the belief before this scan (K samples
// of ds, log-odds in nats), evaluated with fp64 directions and exact sample
// fractions; J^T J and J^T e are summed in fp64 and the 3x3 step is solved in
// fp64 by Cramer's rule on one thread:
//   xi <- xi - (J^T J + mu I)^-1 J^T e,   e_b = r_b(xi) - z_b,  mu = 1e-6,
// over the inliers fixed at the match: beams whose measured range is within
// the model's reach (z_b < K ds) and within two cells of the model's range
// there.  An iterate outside the matcher's search box keeps the match; an
// accepted result is reported on a 1 mm / 1 mrad lattice.  The CTA stages
// the belief window every sample can reach (the box plus K ds, one tap
// further) in shared memory when it fits.  An episode's first scan (an
// empty window) keeps the match.
constexpr int kCorrBlockMax = 512;
constexpr size_t kCorrWindowMax = 48 * 1024;     // staged window, no opt-in needed

__global__ void __launch_bounds__(kCorrBlockMax, 2) slam_correct2d_kernel(const Step2DParams p,
                                                                         int R, bool staged) {
    extern __shared__ __align__(16) short s_map[];
    __shared__ double red[9][32];
    __shared__ double s_xi[3];
    __shared__ double s_uv[2];
    __shared__ DF s_cs[2];
    __shared__ int s_ok;
    __shared__ unsigned char s_use[ASLAM_MAX_BEAMS];
    const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const float *pm = p.csm_pose + 3 * (long long)e;
    float *out = p.slam_gn_pose + 3 * (long long)e;
    if (p.win_n[e] == 0) {                       // uniform over the CTA
        if (tid < 3) out[tid] = pm[tid];
        return;
    }
    const int W = p.W[e], H = p.H[e], B = p.B[e];
    const short *Lq = p.belief + p.map_off[e];
    MapView m{Lq, W, H, 0, 0, W};
    if (staged) {
        // every tap of an accepted iterate lies within R cells of the match's cell
        const int ri = q16_of(pm[0], p.res) >> 16, rj = q16_of(pm[1], p.res) >> 16;
        const int x0 = min(max(ri - R, 0), W - 1), x1 = min(max(ri + R, 0), W - 1);
        const int y0 = min(max(rj - R, 0), H - 1), y1 = min(max(rj + R, 0), H - 1);
        const int ww = x1 - x0 + 1, wh = y1 - y0 + 1;
        for (int q = tid; q < ww * wh; q += nt) {
            const int jj = q / ww, ii = q - jj * ww;
            s_map[q] = __ldg(Lq + (long long)(y0 + jj) * W + x0 + ii);
        }
        m = MapView{s_map, W, H, x0, y0, ww};
    }
    if (tid == 0) {
        s_xi[0] = pm[0];
        s_xi[1] = pm[1];
        s_xi[2] = pm[2];
        s_ok = 1;
    }
    const float inv_res = 1.0f / p.res, scale = p.logodds_scale;
    const float r_far = (float)p.uq_K * p.uq_ds;
    const double gate = 2.0 * (double)p.res;
    const double box_xy = (double)(p.csm_n_xy + 1) * (double)p.res;
    const double box_th = (double)(p.csm_n_th + 1) * (double)p.csm_dth;
    const DF dsr = df_of((double)p.uq_ds / (double)p.res);
    const float *z = p.z + p.ray_off[e];
    const float4 *bdf = p.beam_df + p.ray_off[e];
    auto set_pose = [&]() {
        // the bilinear frame's origin and the heading's cos / sin, in fp64
        if (tid == 0) {
            s_uv[0] = s_xi[0] / (double)p.res - 0.5;
            s_uv[1] = s_xi[1] / (double)p.res - 0.5;
            double sd, cd;
            sincos(s_xi[2], &sd, &cd);
            s_cs[0] = df_of(cd);
            s_cs[1] = df_of(sd);
        }
        __syncthreads();
    };
    auto ray = [&](int b) {
        const float4 bd = bdf[b];
        return soft_ray(s_uv[0], s_uv[1], s_cs[0], s_cs[1], DF{bd.x, bd.y}, DF{bd.z, bd.w}, dsr);
    };
    __syncthreads();                             // staged map, s_xi
    set_pose();
    for (int b = tid; b < B; b += nt) {
        const float r0 = soft_range_q(m, inv_res, scale, ray(b), p.uq_K, p.uq_ds, r_far, nullptr);
        s_use[b] = z[b] < r_far && fabs((double)r0 - (double)z[b]) < gate;
    }
    for (int it = 0; it < p.slam_gn_iters; ++it) {
        if (it > 0) set_pose();
        // normal equations (xx, xy, xt, yy, yt, tt) and g = J^T e, in fp64
        double v[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int b = tid; b < B; b += nt) {
            if (!s_use[b]) continue;
            float J[3];
            const float r = soft_range_q(m, inv_res, scale, ray(b), p.uq_K, p.uq_ds, r_far, J);
            const double eb = (double)r - (double)z[b];
            const double J0 = J[0], J1 = J[1], J2 = J[2];
            v[0] += J0 * J0;
            v[1] += J0 * J1;
            v[2] += J0 * J2;
            v[3] += J1 * J1;
            v[4] += J1 * J2;
            v[5] += J2 * J2;
            v[6] += J0 * eb;
            v[7] += J1 * eb;
            v[8] += J2 * eb;
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            double a = v[q];
#pragma unroll
            for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[q][warp] = a;
        }
        __syncthreads();
        if (tid == 0) {
            double w[9];
            for (int q = 0; q < 9; ++q) {
                double a = 0.0;
                for (int k = 0; k < nw; ++k) a += red[q][k];
                w[q] = a;
            }
            const double mu = 1e-6;
            const double A[9] = {w[0] + mu, w[1], w[2], w[1], w[3] + mu, w[4], w[2], w[4], w[5] + mu};
            const double g[3] = {w[6], w[7], w[8]};
            const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                               A[2] * (A[3] * A[7] - A[4] * A[6]);
            for (int col = 0; col < 3; ++col) {
                double M[9];
                for (int q = 0; q < 9; ++q) M[q] = A[q];
                for (int row = 0; row < 3; ++row) M[3 * row + col] = -g[row];
                s_xi[col] += (M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                              M[2] * (M[3] * M[7] - M[4] * M[6])) / det;
            }
            s_ok = fabs(s_xi[0] - (double)pm[0]) <= box_xy && fabs(s_xi[1] - (double)pm[1]) <= box_xy &&
                   fabs(s_xi[2] - (double)pm[2]) <= box_th;      // false for NaN
        }
        __syncthreads();
        if (!s_ok) break;                        // uniform: read after the barrier
    }
    if (tid < 3) out[tid] = s_ok ? (float)(rint(s_xi[tid] * 1000.0) / 1000.0) : pm[tid];
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
        // the window's pose measurement: the (corrected) match
        meas[3 * n + lane] = (p.slam_gn_iters > 0 ? p.slam_gn_pose : p.csm_pose)[3 * e + lane];
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
    int k = 2;
    if (p.slam_gn_iters > 0) {
        int block = ((p.b_max + 31) / 32) * 32;
        block = block < 64 ? 64 : (block > kCorrBlockMax ? kCorrBlockMax : block);
        // samples reach K*ds from an accepted iterate (inside the box of
        // n_xy + 1 cells around the match); taps one cell further, plus rounding
        const int R = (int)ceilf(((float)p.uq_K * p.uq_ds) / p.res) + p.csm_n_xy + 4;
        const size_t win = 2 * (size_t)(2 * R + 1) * (2 * R + 1);
        const bool staged = win <= kCorrWindowMax;
        slam_correct2d_kernel<<<p.E, block, staged ? win : 0, s>>>(p, R, staged);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[k++], s);
        if (e != cudaSuccess) return e;
    }
    // one half-warp per env, few per CTA: the fp64 window solves spread over every
    // SM (the fp64 rate of one SM is small)
    slam_window2d_kernel<<<(p.E + kWinEnvs - 1) / kWinEnvs, 16 * kWinEnvs, 0, s>>>(p);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[k], s);
    return e;
}

}  // namespace aslam
