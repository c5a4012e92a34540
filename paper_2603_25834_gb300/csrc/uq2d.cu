// uq2d.cu -- in-step pose uncertainty U_t of the 2-D step (Sec. III-D,
// Eq. 5-6) on sm_103a.
//
// The scan-match information of the soft expected-range model: each beam's
// range r_b = sum_k T_k p_k s_k + T_K * K*ds over K samples s_k = (k+1)*ds
// of the belief (bilinear natural log-odds on cell centres, clamp to edge;
// p_k = sigmoid(l_k), T_{k+1} = T_k (1 - p_k)), differentiated in forward
// mode w.r.t. the pose (x, y, th); A = sum_b J_b J_b^T / sigma_r^2 is the
// Gauss-Newton Hessian of the scan-to-map residuals.  It is fused with the
// previous pose covariance propagated by one step of odometry noise Q
// (the last block of a two-pose window with an odometry factor):
//   Sigma_t = ((Sigma_{t-1} + Q)^-1 + A)^-1,   U_t = det(Sigma_t)^(1/3) / scale.
//
// Accuracy (the model of soft_model.cuh): each beam's direction comes from
// the fp64 heading and beam angle as double-floats, each sample's bilinear
// fraction is one rounding of a number below 1, the sigmoid uses the
// correctly rounded exp and reciprocal, the transmittance is a double-float,
// and J J^T is summed in fp64; U then agrees with an fp64 evaluation to
// about 1e-5 relative.
//
// Runs between the sensing and the update kernels, so the map is the one
// built before this scan.  One CTA per env, one thread per beam.  Every
// sample lies within K*ds of the robot, so the CTA first copies the map
// window of half-side R = ceil(K*ds/res) + 2 cells around the robot's cell
// (clamped to the map) into shared memory and reads its bilinear taps
// there; lanes of a warp follow beams that fan out, and their taps would
// otherwise touch up to 32 cache lines per load.  The six
// sums of J J^T are reduced in a fixed order (deterministic); the 3x3
// algebra runs in fp64 on one thread.  An env that resets this step has an
// all-unknown map (cleared by the update kernel), hence A = 0.
#include <cmath>

#include "aslam_internal.cuh"
#include "env_common.cuh"
#include "soft_model.cuh"

namespace aslam {
namespace {

__device__ __forceinline__ double det3d(const double *M) {
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// 3x3 inverse through the adjugate, one reciprocal of the determinant.
__device__ __forceinline__ void inv3d(const double *M, double *R) {
    const double id = 1.0 / det3d(M);
    R[0] = (M[4] * M[8] - M[5] * M[7]) * id;
    R[1] = (M[2] * M[7] - M[1] * M[8]) * id;
    R[2] = (M[1] * M[5] - M[2] * M[4]) * id;
    R[3] = (M[5] * M[6] - M[3] * M[8]) * id;
    R[4] = (M[0] * M[8] - M[2] * M[6]) * id;
    R[5] = (M[2] * M[3] - M[0] * M[5]) * id;
    R[6] = (M[3] * M[7] - M[4] * M[6]) * id;
    R[7] = (M[1] * M[6] - M[0] * M[7]) * id;
    R[8] = (M[0] * M[4] - M[1] * M[3]) * id;
}

// Three CTAs per SM (at most 42 registers a thread) hide the latency of
// each beam's sample chain better than fewer, fatter CTAs.  When the beams
// fit twice into a CTA (split = 2) two threads share a beam (samples
// [0, K1) and [K1, K)), halving the chain that sets the time; with more
// beams, fatter CTAs would cost more waves than the halved chain saves
// (timed at 360 beams: 97 us one thread per beam, 121 us two).
constexpr int kUqBlockMax = 512;

__global__ void __launch_bounds__(kUqBlockMax, 3) uq2d_kernel(const Step2DParams p, int R, bool staged,
                                                              int split) {
    extern __shared__ __align__(16) short s_win[];
    __shared__ double red[6][32];
    __shared__ double s_uv[2];
    __shared__ DF s_cs[2];
    const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int W = p.W[e], H = p.H[e], B = p.B[e];
    const bool reset = p.done[e] != 0;
    // a thread's own terms of J J^T in fp32 (one beam per thread up to the
    // block size; each product is one rounding), the sums over beams in fp64
    float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (!reset) {
        const short *Lq = p.belief + p.map_off[e];
        // the pose at the start of this step (integrated by the sensing kernel)
        const EnvStart &st = reinterpret_cast<const EnvSense *>(p.env_sense)[e].start;
        const float x = st.x, y = st.y, th = st.th;
        MapView m{Lq, W, H, 0, 0, W};
        if (staged) {
            // every tap (clamped to the map) is within R cells of the robot's cell
            const int ri = q16_of(x, p.res) >> 16, rj = q16_of(y, p.res) >> 16;
            const int x0 = min(max(ri - R, 0), W - 1), x1 = min(max(ri + R, 0), W - 1);
            const int y0 = min(max(rj - R, 0), H - 1), y1 = min(max(rj + R, 0), H - 1);
            const int ww = x1 - x0 + 1, wh = y1 - y0 + 1;
            for (int q = tid; q < ww * wh; q += nt) {
                const int jj = q / ww, ii = q - jj * ww;
                s_win[q] = __ldg(Lq + (long long)(y0 + jj) * W + x0 + ii);
            }
            m = MapView{s_win, W, H, x0, y0, ww};
        }
        if (tid == 0) {
            // the bilinear frame's origin u0 = x/res - 1/2 (and v0) and the
            // heading's cos / sin, in fp64
            s_uv[0] = (double)x / (double)p.res - 0.5;
            s_uv[1] = (double)y / (double)p.res - 0.5;
            double sd, cd;
            sincos((double)th, &sd, &cd);
            s_cs[0] = df_of(cd);
            s_cs[1] = df_of(sd);
        }
        __syncthreads();
        const double u0 = s_uv[0], v0 = s_uv[1];
        const DF ct = s_cs[0], st_ = s_cs[1];
        const DF dsr = df_of((double)p.uq_ds / (double)p.res);
        const float inv_res = 1.0f / p.res, scale = p.logodds_scale;
        const float r_far = (float)p.uq_K * p.uq_ds;
        // The sweep is linear in (T, dT): the second half runs from T = 1,
        // dT = 0 and also sums A = sum_k T'_k p_k s_k; with the first half's
        // (T, dT) at the split, the beam's totals are
        //   dr = dr_1 + dT_1 A + T_1 dr'_2,   dT = dT_1 Q + T_1 dT'_2,
        // Q the second half's product of q.
        const int h = split == 2 ? (tid & 1) : 0;
        const int K1 = split == 2 ? (p.uq_K + 1) >> 1 : p.uq_K;
        const int k0 = h ? K1 : 0, k1 = h ? p.uq_K : K1;
        for (int b0 = 0; b0 < B; b0 += nt / split) {
            const int b = b0 + tid / split;
            const bool live = b < B;
            float4 bd = make_float4(1.f, 0.f, 0.f, 0.f);
            if (live) bd = p.beam_df[p.ray_off[e] + b];
            const SoftRay ry = soft_ray(u0, v0, ct, st_, DF{bd.x, bd.y}, DF{bd.z, bd.w}, dsr);
            const float cp = ry.cp, sp = ry.sp;
            DF Td = {1.f, 0.f};
            float A = 0.f;
            float dT0 = 0.f, dT1 = 0.f, dT2 = 0.f, dr0 = 0.f, dr1 = 0.f, dr2 = 0.f;
            Tap t;
            for (int k = k0; live && k < k1; ++k) {
                const float sk = (float)(k + 1) * p.uq_ds;
                int i0, j0;
                float ax, ay;
                sample_coord(ry.u0, ry.du, k + 1, i0, ax);
                sample_coord(ry.v0, ry.dv, k + 1, j0, ay);
                bilinear_q(m, inv_res, scale, i0, j0, ax, ay, t);
                float pr, q;
                sigmoid_pq_accurate(t.l, pr, q);
                const float T = Td.hi;
                const float dpl = pr * q;
                const float d0 = dpl * t.gx, d1 = dpl * t.gy;
                const float d2 = dpl * (t.gx * (-sk * sp) + t.gy * (sk * cp));
                dr0 += (dT0 * pr + T * d0) * sk;
                dr1 += (dT1 * pr + T * d1) * sk;
                dr2 += (dT2 * pr + T * d2) * sk;
                A += T * pr * sk;
                dT0 = dT0 * q - T * d0;
                dT1 = dT1 * q - T * d1;
                dT2 = dT2 * q - T * d2;
                Td = trans_mul_q(Td, q);
            }
            const float T = Td.hi;
            // the second half's sums to its first half (the lane below); one
            // thread per beam combines with an empty second half
            float Q2 = 1.f, A2 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f;
            if (split == 2) {                      // uniform over the CTA
                Q2 = __shfl_down_sync(0xffffffffu, T, 1);
                A2 = __shfl_down_sync(0xffffffffu, A, 1);
                e0 = __shfl_down_sync(0xffffffffu, dT0, 1);
                e1 = __shfl_down_sync(0xffffffffu, dT1, 1);
                e2 = __shfl_down_sync(0xffffffffu, dT2, 1);
                f0 = __shfl_down_sync(0xffffffffu, dr0, 1);
                f1 = __shfl_down_sync(0xffffffffu, dr1, 1);
                f2 = __shfl_down_sync(0xffffffffu, dr2, 1);
            }
            if (h == 0 && live) {
                const float g0 = dr0 + dT0 * A2 + T * f0, g1 = dr1 + dT1 * A2 + T * f1;
                const float g2 = dr2 + dT2 * A2 + T * f2;
                const float u0 = dT0 * Q2 + T * e0, u1 = dT1 * Q2 + T * e1, u2 = dT2 * Q2 + T * e2;
                const float J0 = g0 + u0 * r_far, J1 = g1 + u1 * r_far, J2 = g2 + u2 * r_far;
                a[0] += J0 * J0;
                a[1] += J0 * J1;
                a[2] += J0 * J2;
                a[3] += J1 * J1;
                a[4] += J1 * J2;
                a[5] += J2 * J2;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        double v = (double)a[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double A[6];
        for (int q = 0; q < 6; ++q) {
            double v = 0.0;
            for (int w = 0; w < nw; ++w) v += red[q][w];
            A[q] = v * p.uq_inv_s2;
        }
        double *S = p.pose_cov + 6 * (long long)e;
        double Sp[6];
        if (reset) {
            Sp[0] = p.uq_prior[0];
            Sp[1] = Sp[2] = Sp[4] = 0.0;
            Sp[3] = p.uq_prior[1];
            Sp[5] = p.uq_prior[2];
        } else {
            for (int q = 0; q < 6; ++q) Sp[q] = S[q];
        }
        const double P[9] = {Sp[0] + p.uq_q[0], Sp[1], Sp[2], Sp[1], Sp[3] + p.uq_q[1], Sp[4],
                             Sp[2], Sp[4], Sp[5] + p.uq_q[2]};
        double Pi[9], Sn[9];
        inv3d(P, Pi);
        const double Info[9] = {Pi[0] + A[0], Pi[1] + A[1], Pi[2] + A[2],
                                Pi[3] + A[1], Pi[4] + A[3], Pi[5] + A[4],
                                Pi[6] + A[2], Pi[7] + A[4], Pi[8] + A[5]};
        inv3d(Info, Sn);
        S[0] = Sn[0];
        S[1] = 0.5 * (Sn[1] + Sn[3]);
        S[2] = 0.5 * (Sn[2] + Sn[6]);
        S[3] = Sn[4];
        S[4] = 0.5 * (Sn[5] + Sn[7]);
        S[5] = Sn[8];
        p.u_scan[e] = (float)(cbrt(det3d(Sn)) / p.uq_scale);
    }
}

constexpr size_t kUqWindowMax = 48 * 1024;     // shared bytes for the staged map window

}  // namespace

cudaError_t launch_uq2d(const Step2DParams &p, cudaStream_t s) {
    // two threads per beam when that still fits one CTA
    const int split = 2 * p.b_max <= kUqBlockMax ? 2 : 1;
    int block = ((split * p.b_max + 31) / 32) * 32;
    block = block < 64 ? 64 : (block > kUqBlockMax ? kUqBlockMax : block);
    // samples reach K*ds from the robot; taps one cell further, plus rounding
    const int R = (int)ceilf(((float)p.uq_K * p.uq_ds) / p.res) + 2;
    const size_t win = 2 * (size_t)(2 * R + 1) * (2 * R + 1);
    const bool staged = win <= kUqWindowMax;
    uq2d_kernel<<<p.E, block, staged ? win : 0, s>>>(p, R, staged, split);
    return cudaGetLastError();
}

}  // namespace aslam
