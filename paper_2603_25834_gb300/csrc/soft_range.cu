// soft_range.cu -- differentiable soft expected-range raycaster and batched
// scan-to-map Gauss-Newton (Sec. III-D, Eq. 5-6) on sm_103a.
//
// Soft range of beam b from pose (x, y, th): K samples s_k = (k+1)*ds along
// phi = th + beta_b; l_k = bilinear log-odds on cell centres (clamp to edge);
// p_k = sigmoid(l_k); T_0 = 1, T_{k+1} = T_k (1 - p_k);
// r = sum_k T_k p_k s_k + T_K * K*ds.
//
// Kernels (one CTA per environment, threads loop over beams):
//   soft_fwd      r                                        (one sweep)
//   soft_bwd      adjoint of sum(g*r) w.r.t. pose and map: a forward sweep
//                 recomputes T_k into shared memory, a reverse sweep runs
//                 R_k = p_k s_k + (1-p_k) R_{k+1} and dr/dp_k = T_k (s_k - R_{k+1})
//   soft_jac      r and dr/d(x,y,th) by forward-mode tangents (one sweep)
//   gn            `iters` damped Gauss-Newton steps per env, then the damped
//                 normal matrix at the final pose, its inverse scaled by the
//                 range variance (the pose covariance block, Eq. 6) and
//                 U = det(Sigma)^(1/3) (D-optimality, Table I "D-opt")
#include <math.h>

#include <algorithm>

#include <string>

#include "aslam_internal.cuh"
#include "soft_model.cuh"

namespace aslam {
namespace {

struct SoftParams {
    int E, W, H, B, K;
    float res, inv_res, ds, r_far, mu, sigma2;
    int full_turn;         // beam b at 2 pi b / B; else at -fov/2 + b fov / (B - 1)
    double fov, dsr;       // field of view; ds / res
    const float *L;        // [E, H, W]
    const float *pose;     // [E, 3]
};

// Angle of beam b, in fp64 (the definition of the beam layout).
__device__ __forceinline__ double soft_beam_angle(const SoftParams &p, int b) {
    const double two_pi = 2.0 * 3.14159265358979323846;
    if (p.full_turn) return (two_pi * (double)b) / (double)p.B;
    if (p.B == 1) return 0.0;
    return -0.5 * p.fov + ((double)b * p.fov) / (double)(p.B - 1);
}

// cos/sin of every beam's angle as double-floats, once per CTA.
__device__ __forceinline__ void stage_beams(const SoftParams &p, DF *s_cb, DF *s_sb) {
    for (int b = threadIdx.x; b < p.B; b += blockDim.x) {
        double sb, cb;
        sincos(soft_beam_angle(p, b), &sb, &cb);
        s_cb[b] = df_of(cb);
        s_sb[b] = df_of(sb);
    }
}

// The pose's part of every beam's geometry, in fp64 by one thread: the
// bilinear-frame origin u0 = x/res - 1/2, v0 = y/res - 1/2 and cos/sin of
// the heading.
struct SoftPose {
    double u0, v0;
    DF ct, st;
};

__device__ __forceinline__ SoftPose soft_pose(const SoftParams &p, float x, float y, float th) {
    SoftPose q;
    q.u0 = (double)x / (double)p.res - 0.5;
    q.v0 = (double)y / (double)p.res - 0.5;
    double s, c;
    sincos((double)th, &s, &c);
    q.ct = df_of(c);
    q.st = df_of(s);
    return q;
}

__device__ __forceinline__ SoftRay ray_of(const SoftParams &p, const SoftPose &q, DF cb, DF sb) {
    return soft_ray(q.u0, q.v0, q.ct, q.st, cb, sb, df_of(p.dsr));
}

struct Sample {
    float l, gx, gy;       // log-odds and its gradient (per metre)
    int idx[4];
    float w[4];
};

// Bilinear log-odds of sample k of a ray: lower-left tap (i0, j0) with
// fractions (ax, ay), taps clamped to the map.
__device__ __forceinline__ void soft_sample(const SoftParams &p, const float *L, const SoftRay &ry,
                                            int k, Sample &s) {
    int i0, j0;
    float ax, ay;
    sample_coord(ry.u0, ry.du, k + 1, i0, ax);
    sample_coord(ry.v0, ry.dv, k + 1, j0, ay);
    const int ia = min(max(i0, 0), p.W - 1), ib = min(max(i0 + 1, 0), p.W - 1);
    const int ja = min(max(j0, 0), p.H - 1), jb = min(max(j0 + 1, 0), p.H - 1);
    s.idx[0] = ja * p.W + ia;
    s.idx[1] = ja * p.W + ib;
    s.idx[2] = jb * p.W + ia;
    s.idx[3] = jb * p.W + ib;
    const float l00 = __ldg(L + s.idx[0]), l10 = __ldg(L + s.idx[1]);
    const float l01 = __ldg(L + s.idx[2]), l11 = __ldg(L + s.idx[3]);
    s.w[0] = (1.f - ax) * (1.f - ay);
    s.w[1] = ax * (1.f - ay);
    s.w[2] = (1.f - ax) * ay;
    s.w[3] = ax * ay;
    s.l = s.w[0] * l00 + s.w[1] * l10 + s.w[2] * l01 + s.w[3] * l11;
    s.gx = ((1.f - ay) * (l10 - l00) + ay * (l11 - l01)) * p.inv_res;
    s.gy = ((1.f - ax) * (l01 - l00) + ax * (l11 - l10)) * p.inv_res;
}

// Kahan step: (r, c) <- r + y with the running compensation c.
__device__ __forceinline__ void kahan_add(float &r, float &c, float y) {
    const float yc = __fsub_rn(y, c);
    const float t = __fadd_rn(r, yc);
    c = __fsub_rn(__fsub_rn(t, r), yc);
    r = t;
}

// Transmittance times one more factor q, as a double-float.
__device__ __forceinline__ DF trans_mul(DF T, float q) {
    const float p = __fmul_rn(T.hi, q);
    const float l = __fmaf_rn(T.lo, q, __fmaf_rn(T.hi, q, -p));
    const float h = __fadd_rn(p, l);
    return {h, __fsub_rn(l, __fsub_rn(h, p))};
}

// Forward-mode soft range: value and d/d(x, y, th).
__device__ __forceinline__ float soft_range_tangent(const SoftParams &p, const float *L,
                                                   const SoftRay &ry, float J[3]) {
    DF T = {1.f, 0.f};
    float r = 0.f, rc = 0.f;
    float dT0 = 0.f, dT1 = 0.f, dT2 = 0.f, dr0 = 0.f, dr1 = 0.f, dr2 = 0.f;
    Sample sm;
    for (int k = 0; k < p.K; ++k) {
        const float s = (float)(k + 1) * p.ds;
        soft_sample(p, L, ry, k, sm);
        float pr, q;
        sigmoid_pq_accurate(sm.l, pr, q);
        const float dpl = pr * q;
        const float d0 = dpl * sm.gx, d1 = dpl * sm.gy;
        const float d2 = dpl * (sm.gx * (-s * ry.sp) + sm.gy * (s * ry.cp));
        kahan_add(r, rc, __fmul_rn(__fmul_rn(T.hi, pr), s));
        dr0 += (dT0 * pr + T.hi * d0) * s;
        dr1 += (dT1 * pr + T.hi * d1) * s;
        dr2 += (dT2 * pr + T.hi * d2) * s;
        dT0 = dT0 * q - T.hi * d0;
        dT1 = dT1 * q - T.hi * d1;
        dT2 = dT2 * q - T.hi * d2;
        T = trans_mul(T, q);
    }
    kahan_add(r, rc, __fmaf_rn(T.hi, p.r_far, T.lo * p.r_far));
    J[0] = dr0 + dT0 * p.r_far;
    J[1] = dr1 + dT1 * p.r_far;
    J[2] = dr2 + dT2 * p.r_far;
    return r;
}

__global__ void soft_fwd_kernel(const SoftParams p, float *ranges) {
    __shared__ DF s_cb[ASLAM_MAX_BEAMS], s_sb[ASLAM_MAX_BEAMS];
    __shared__ SoftPose s_q;
    const int e = blockIdx.x;
    const float *L = p.L + (long long)e * p.W * p.H;
    stage_beams(p, s_cb, s_sb);
    if (threadIdx.x == 0) s_q = soft_pose(p, p.pose[3 * e], p.pose[3 * e + 1], p.pose[3 * e + 2]);
    __syncthreads();
    for (int b = threadIdx.x; b < p.B; b += blockDim.x) {
        const SoftRay ry = ray_of(p, s_q, s_cb[b], s_sb[b]);
        DF T = {1.f, 0.f};
        float r = 0.f, rc = 0.f;
        Sample sm;
        for (int k = 0; k < p.K; ++k) {
            const float s = (float)(k + 1) * p.ds;
            soft_sample(p, L, ry, k, sm);
            float pr, q;
            sigmoid_pq_accurate(sm.l, pr, q);
            kahan_add(r, rc, __fmul_rn(__fmul_rn(T.hi, pr), s));
            T = trans_mul(T, q);
        }
        kahan_add(r, rc, __fmaf_rn(T.hi, p.r_far, T.lo * p.r_far));
        ranges[(long long)e * p.B + b] = r;
    }
}

__global__ void soft_jac_kernel(const SoftParams p, float *ranges, float *jac) {
    __shared__ DF s_cb[ASLAM_MAX_BEAMS], s_sb[ASLAM_MAX_BEAMS];
    __shared__ SoftPose s_q;
    const int e = blockIdx.x;
    const float *L = p.L + (long long)e * p.W * p.H;
    stage_beams(p, s_cb, s_sb);
    if (threadIdx.x == 0) s_q = soft_pose(p, p.pose[3 * e], p.pose[3 * e + 1], p.pose[3 * e + 2]);
    __syncthreads();
    for (int b = threadIdx.x; b < p.B; b += blockDim.x) {
        float J[3];
        const float r = soft_range_tangent(p, L, ray_of(p, s_q, s_cb[b], s_sb[b]), J);
        const long long o = (long long)e * p.B + b;
        if (ranges) ranges[o] = r;
        jac[3 * o] = J[0];
        jac[3 * o + 1] = J[1];
        jac[3 * o + 2] = J[2];
    }
}

template <int N>
__device__ __forceinline__ void block_sum(float (&v)[N], float (*red)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        float a = v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[q][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            float a = 0.f;
            for (int w = 0; w < nw; ++w) a += red[q][w];
            v[q] = a;
        }
    }
    __syncthreads();
}

template <int N>
__device__ __forceinline__ void block_sum_d(double (&v)[N], double (*red)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        double a = v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[q][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            double a = 0.0;
            for (int w = 0; w < nw; ++w) a += red[q][w];
            v[q] = a;
        }
    }
    __syncthreads();
}

// Adjoint: one CTA per env; shared memory holds T_k for every thread's beam.
__global__ void soft_bwd_kernel(const SoftParams p, const float *grad_r, float *grad_pose,
                                float *grad_L) {
    extern __shared__ float s_T[];            // [K][blockDim]
    __shared__ float red[3][32];
    __shared__ DF s_cb[ASLAM_MAX_BEAMS], s_sb[ASLAM_MAX_BEAMS];
    __shared__ SoftPose s_q;
    const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const float *L = p.L + (long long)e * p.W * p.H;
    float *gL = grad_L ? grad_L + (long long)e * p.W * p.H : nullptr;
    stage_beams(p, s_cb, s_sb);
    if (tid == 0) s_q = soft_pose(p, p.pose[3 * e], p.pose[3 * e + 1], p.pose[3 * e + 2]);
    __syncthreads();
    float acc[3] = {0.f, 0.f, 0.f};
    for (int b0 = 0; b0 < p.B; b0 += nt) {
        const int b = b0 + tid;
        if (b < p.B) {
            const float g = grad_r[(long long)e * p.B + b];
            const SoftRay ry = ray_of(p, s_q, s_cb[b], s_sb[b]);
            Sample sm;
            // forward sweep: transmittance before each sample
            DF T = {1.f, 0.f};
            for (int k = 0; k < p.K; ++k) {
                s_T[k * nt + tid] = T.hi;
                soft_sample(p, L, ry, k, sm);
                float pr, q;
                sigmoid_pq_accurate(sm.l, pr, q);
                T = trans_mul(T, q);
            }
            // reverse sweep
            float R = p.r_far;
            for (int k = p.K - 1; k >= 0; --k) {
                const float s = (float)(k + 1) * p.ds;
                soft_sample(p, L, ry, k, sm);
                float pr, q;
                sigmoid_pq_accurate(sm.l, pr, q);
                const float dl = g * s_T[k * nt + tid] * (s - R) * pr * q;
                if (gL) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (sm.w[c] != 0.f) atomicAdd(gL + sm.idx[c], dl * sm.w[c]);
                }
                acc[0] += dl * sm.gx;
                acc[1] += dl * sm.gy;
                acc[2] += dl * (sm.gx * (-s * ry.sp) + sm.gy * (s * ry.cp));
                R = pr * s + q * R;
            }
        }
    }
    block_sum<3>(acc, red);
    if (tid == 0) {
        grad_pose[3 * e] = acc[0];
        grad_pose[3 * e + 1] = acc[1];
        grad_pose[3 * e + 2] = acc[2];
    }
}

__device__ __forceinline__ double det3(const double *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// One thread per beam (the normal equations summed in fp64); two CTAs per SM.
__global__ void __launch_bounds__(512, 2) gn_kernel(const SoftParams p, const float *z, int iters,
                                                    float *pose_out, float *cov, float *u_out) {
    __shared__ double red[9][32];
    __shared__ float s_pose[3];
    __shared__ DF s_cb[ASLAM_MAX_BEAMS], s_sb[ASLAM_MAX_BEAMS];
    __shared__ SoftPose s_q;
    const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const float *L = p.L + (long long)e * p.W * p.H;
    stage_beams(p, s_cb, s_sb);
    if (tid < 3) s_pose[tid] = p.pose[3 * e + tid];
    __syncthreads();
    for (int it = 0; it <= iters; ++it) {
        if (tid == 0) s_q = soft_pose(p, s_pose[0], s_pose[1], s_pose[2]);
        __syncthreads();
        // normal equations: A (xx, xy, xt, yy, yt, tt) and g = J^T e
        double v[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int b = tid; b < p.B; b += nt) {
            float J[3];
            const float r = soft_range_tangent(p, L, ray_of(p, s_q, s_cb[b], s_sb[b]), J);
            const double res = (double)r - (double)z[(long long)e * p.B + b];
            const double J0 = J[0], J1 = J[1], J2 = J[2];
            v[0] += J0 * J0;
            v[1] += J0 * J1;
            v[2] += J0 * J2;
            v[3] += J1 * J1;
            v[4] += J1 * J2;
            v[5] += J2 * J2;
            v[6] += J0 * res;
            v[7] += J1 * res;
            v[8] += J2 * res;
        }
        block_sum_d<9>(v, red);
        if (tid == 0) {
            double A[9] = {v[0] + (double)p.mu, v[1], v[2], v[1], v[3] + (double)p.mu, v[4],
                           v[2], v[4], v[5] + (double)p.mu};
            const double det = det3(A);
            const double idet = 1.0 / det;
            if (it < iters) {
                double d[3];
                for (int col = 0; col < 3; ++col) {
                    double M[9];
                    for (int q = 0; q < 9; ++q) M[q] = A[q];
                    M[col] = -v[6];
                    M[3 + col] = -v[7];
                    M[6 + col] = -v[8];
                    d[col] = det3(M) * idet;
                }
                s_pose[0] = (float)((double)s_pose[0] + d[0]);
                s_pose[1] = (float)((double)s_pose[1] + d[1]);
                s_pose[2] = (float)((double)s_pose[2] + d[2]);
            } else {
                pose_out[3 * e] = s_pose[0];
                pose_out[3 * e + 1] = s_pose[1];
                pose_out[3 * e + 2] = s_pose[2];
                // Sigma = sigma^2 A^{-1} (adjugate / det), U = det(Sigma)^(1/3)
                double Ai[9];
                Ai[0] = (A[4] * A[8] - A[5] * A[7]) * idet;
                Ai[1] = (A[2] * A[7] - A[1] * A[8]) * idet;
                Ai[2] = (A[1] * A[5] - A[2] * A[4]) * idet;
                Ai[3] = (A[5] * A[6] - A[3] * A[8]) * idet;
                Ai[4] = (A[0] * A[8] - A[2] * A[6]) * idet;
                Ai[5] = (A[2] * A[3] - A[0] * A[5]) * idet;
                Ai[6] = (A[3] * A[7] - A[4] * A[6]) * idet;
                Ai[7] = (A[1] * A[6] - A[0] * A[7]) * idet;
                Ai[8] = (A[0] * A[4] - A[1] * A[3]) * idet;
                if (cov)
                    for (int q = 0; q < 9; ++q) cov[9 * e + q] = (float)(p.sigma2 * Ai[q]);
                if (u_out) {
                    const double s2 = (double)p.sigma2;
                    u_out[e] = (float)cbrt(s2 * s2 * s2 / det);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace aslam

using namespace aslam;

namespace {

aslam_status soft_fail(aslam_status s, const char *m) {
    set_thread_error(m);
    return s;
}

aslam_status make_params(const aslam_soft_config *c, const float *L, const float *pose,
                         SoftParams *p) {
    if (!c || c->struct_size != sizeof(aslam_soft_config))
        return soft_fail(ASLAM_ERR_INVALID_ARG, "bad aslam_soft_config");
    if (c->n_envs < 1 || c->map_w < 1 || c->map_h < 1 || c->n_beams < 1 ||
        c->n_beams > ASLAM_MAX_BEAMS || c->n_samples < 1 || c->n_samples > ASLAM_SOFT_MAX_SAMPLES)
        return soft_fail(ASLAM_ERR_INVALID_ARG, "soft config sizes out of range");
    if (!(c->res_m > 0.f) || !(c->sample_step_m > 0.f) || !(c->gn_damping >= 0.f) ||
        !(c->range_sigma_m > 0.f))
        return soft_fail(ASLAM_ERR_INVALID_ARG, "soft config scales out of range");
    if (!L || !pose) return soft_fail(ASLAM_ERR_INVALID_ARG, "NULL map or pose");
    const double two_pi = 2.0 * 3.14159265358979323846;
    const double fov = (double)c->fov_rad;
    const bool full_turn = fov <= 0.0 || fov >= two_pi - 1e-9;
    p->E = c->n_envs;
    p->W = c->map_w;
    p->H = c->map_h;
    p->B = c->n_beams;
    p->K = c->n_samples;
    p->res = c->res_m;
    p->inv_res = 1.0f / c->res_m;
    p->ds = c->sample_step_m;
    p->r_far = (float)c->n_samples * c->sample_step_m;
    p->full_turn = full_turn ? 1 : 0;
    p->fov = fov;
    p->dsr = (double)c->sample_step_m / (double)c->res_m;
    p->mu = c->gn_damping;
    p->sigma2 = c->range_sigma_m * c->range_sigma_m;
    p->L = L;
    p->pose = pose;
    return ASLAM_OK;
}

int soft_block(int B) {
    int t = (B + 31) / 32 * 32;
    return t < 64 ? 64 : (t > 512 ? 512 : t);
}

aslam_status launch_ok(const char *where) {
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        std::string m = std::string(where) + ": " + cudaGetErrorString(ce);
        return soft_fail(ASLAM_ERR_CUDA, m.c_str());
    }
    return ASLAM_OK;
}

}  // namespace

extern "C" {

aslam_status aslam_soft_config_init(aslam_soft_config *c) {
    if (!c) return ASLAM_ERR_INVALID_ARG;
    c->struct_size = sizeof(aslam_soft_config);
    c->n_envs = 1;
    c->map_w = 256;
    c->map_h = 256;
    c->n_beams = 360;
    c->n_samples = 64;
    c->res_m = 0.05f;
    c->sample_step_m = 0.05f;
    c->fov_rad = 0.f;
    c->gn_damping = 1e-6f;
    c->range_sigma_m = 0.01f;
    return ASLAM_OK;
}

aslam_status aslam_soft_range_fwd(const aslam_soft_config *c, const float *d_logodds,
                                  const float *d_pose, float *d_ranges, void *stream) {
    SoftParams p;
    aslam_status st = make_params(c, d_logodds, d_pose, &p);
    if (st != ASLAM_OK) return st;
    if (!d_ranges) return soft_fail(ASLAM_ERR_INVALID_ARG, "NULL ranges");
    soft_fwd_kernel<<<p.E, soft_block(p.B), 0, (cudaStream_t)stream>>>(p, d_ranges);
    return launch_ok("soft_range_fwd");
}

aslam_status aslam_soft_range_jac(const aslam_soft_config *c, const float *d_logodds,
                                  const float *d_pose, float *d_ranges, float *d_jac,
                                  void *stream) {
    SoftParams p;
    aslam_status st = make_params(c, d_logodds, d_pose, &p);
    if (st != ASLAM_OK) return st;
    if (!d_jac) return soft_fail(ASLAM_ERR_INVALID_ARG, "NULL jacobian");
    soft_jac_kernel<<<p.E, soft_block(p.B), 0, (cudaStream_t)stream>>>(p, d_ranges, d_jac);
    return launch_ok("soft_range_jac");
}

aslam_status aslam_soft_range_bwd(const aslam_soft_config *c, const float *d_logodds,
                                  const float *d_pose, const float *d_grad_ranges,
                                  float *d_grad_pose, float *d_grad_logodds, void *stream) {
    SoftParams p;
    aslam_status st = make_params(c, d_logodds, d_pose, &p);
    if (st != ASLAM_OK) return st;
    if (!d_grad_ranges || !d_grad_pose) return soft_fail(ASLAM_ERR_INVALID_ARG, "NULL gradient");
    // as many beams per CTA as keep three CTAs' transmittances (4 K bytes a
    // thread) within about 72 KB each, at most 256 and no more than the beams
    int block = (int)((72 * 1024) / (4 * (size_t)p.K)) & ~31;
    block = std::min(std::max(block, 32), std::min(256, (p.B + 31) / 32 * 32));
    const size_t smem = sizeof(float) * (size_t)p.K * block;
    {
        // the static reduction buffer counts against the same per-block limit
        cudaError_t ce = cudaFuncSetAttribute(soft_bwd_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ce != cudaSuccess) return soft_fail(ASLAM_ERR_CUDA, "soft_range_bwd: shared memory");
    }
    soft_bwd_kernel<<<p.E, block, smem, (cudaStream_t)stream>>>(p, d_grad_ranges, d_grad_pose,
                                                                d_grad_logodds);
    return launch_ok("soft_range_bwd");
}

aslam_status aslam_gn_correct(const aslam_soft_config *c, const float *d_logodds,
                              const float *d_pose_in, const float *d_z, int32_t iters,
                              float *d_pose_out, float *d_cov, float *d_u, void *stream) {
    SoftParams p;
    aslam_status st = make_params(c, d_logodds, d_pose_in, &p);
    if (st != ASLAM_OK) return st;
    if (!d_z || !d_pose_out || iters < 0 || iters > 100)
        return soft_fail(ASLAM_ERR_INVALID_ARG, "bad GN arguments");
    gn_kernel<<<p.E, soft_block(p.B), 0, (cudaStream_t)stream>>>(p, d_z, iters, d_pose_out,
                                                                 d_cov, d_u);
    return launch_ok("gn_correct");
}

}  // extern "C"
