// aslam_internal.cuh -- private definitions of libaslam (device helpers,
// kernel parameter blocks, launcher declarations).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aslam.h"

namespace aslam {

// ---------------------------------------------------------------------------
// Deterministic fp32 elementary functions.  Every operation is an explicit
// round-to-nearest intrinsic so no FMA contraction can change a bit; the
// values feed integer state (robot cell, ray direction, range endpoint), so
// they must be reproducible by any IEEE-754 implementation that performs
// the same operations in the same order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// Global reductions without a returned value (relaxed, device scope, the
// ordering of atomicAdd / atomicOr): the issuing warp never waits for the
// L2, even when the counter's sector has to come from DRAM.  A later
// barrier of the CTA orders them before its own loads of the counters.
__device__ __forceinline__ void red_add(unsigned *a, unsigned v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_or(unsigned *a, unsigned v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Maclaurin series of sin and cos truncated after x^9 / x^10: on
// |r| <= pi/4 the first omitted term is below 2^-26 relative.
__device__ __forceinline__ void poly_sincos(float r, float &s, float &c) {
    const float s3 = (float)(-1.0 / 6.0), s5 = (float)(1.0 / 120.0),
                s7 = (float)(-1.0 / 5040.0), s9 = (float)(1.0 / 362880.0);
    const float c2 = (float)(-1.0 / 2.0), c4 = (float)(1.0 / 24.0),
                c6 = (float)(-1.0 / 720.0), c8 = (float)(1.0 / 40320.0),
                c10 = (float)(-1.0 / 3628800.0);
    float r2 = fmul(r, r);
    float ps = fadd(s7, fmul(r2, s9));
    ps = fadd(s5, fmul(r2, ps));
    ps = fadd(s3, fmul(r2, ps));
    s = fadd(r, fmul(fmul(r, r2), ps));
    float pc = fadd(c8, fmul(r2, c10));
    pc = fadd(c6, fmul(r2, pc));
    pc = fadd(c4, fmul(r2, pc));
    pc = fadd(c2, fmul(r2, pc));
    c = fadd(1.0f, fmul(r2, pc));
}

// sin/cos of an fp32 angle: the quadrant k = rint(x * 2/pi) and remainder
// x - k*pi/2 are formed in fp64 (exact enough for |x| << 2^20), the series
// runs in fp32 on the remainder.
__device__ __forceinline__ void det_sincos(float x, float &s, float &c) {
    double k = rint(__dmul_rn((double)x, 0.63661977236758134308));
    double rem = __dsub_rn((double)x, __dmul_rn(k, 1.57079632679489661923));
    float ps, pc;
    poly_sincos(__double2float_rn(rem), ps, pc);
    switch (((int)k) & 3) {
        case 0: s = ps; c = pc; break;
        case 1: s = pc; c = -ps; break;
        case 2: s = -ps; c = -pc; break;
        default: s = -pc; c = ps; break;
    }
}

// cos(2*pi*u), u in [0, 1): the quarter-turn index is taken on u itself,
// where the subtraction is exact.
__device__ __forceinline__ float det_cos2pi(float u) {
    const float two_pi = (float)(2.0 * 3.14159265358979323846);
    float q = rintf(fmul(u, 4.0f));
    float a = fmul(fsub(u, fmul(q, 0.25f)), two_pi);
    float ps, pc;
    poly_sincos(a, ps, pc);
    switch (((int)q) & 3) {
        case 0: return pc;
        case 1: return -ps;
        case 2: return -pc;
        default: return ps;
    }
}

// ln(u) for a positive normal float: split u = m * 2^e with m in
// [sqrt(1/2), sqrt(2)); ln m = 2*atanh(s), s = (m-1)/(m+1), by the odd
// series s + s^3/3 + ... + s^11/11; ln 2 in two parts (16 + 24 bits).
__device__ __forceinline__ float det_log(float u) {
    unsigned bits = __float_as_uint(u);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    unsigned mb = (bits & 0x7fffffu) | 0x3f800000u;
    float m = __uint_as_float(mb);
    if (mb > 0x3fb504f3u) { m = fmul(m, 0.5f); e += 1; }
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = (float)(0.69314718055994530942 - 0.693145751953125);
    float s = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
    float s2 = fmul(s, s);
    float p = fadd((float)(1.0 / 9.0), fmul(s2, (float)(1.0 / 11.0)));
    p = fadd((float)(1.0 / 7.0), fmul(s2, p));
    p = fadd((float)(1.0 / 5.0), fmul(s2, p));
    p = fadd((float)(1.0 / 3.0), fmul(s2, p));
    float ts = fadd(s, s);
    float lnm = fadd(ts, fmul(ts, fmul(s2, p)));
    float fe = (float)e;
    return fadd(fadd(fmul(fe, ln2_lo), lnm), fmul(fe, ln2_hi));
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// N(0,1) for (key, env, global step, beam): Box-Muller on u1 in (0, 1]
// (never 0) and u2 in [0, 1), each from the top 24 bits of one word.
__device__ __forceinline__ float det_gauss(uint2 key, unsigned env, unsigned step, unsigned beam) {
    uint4 r = philox4x32_10(make_uint4(beam, env, step, 0u), key);
    float u1 = fmul(__uint2float_rn((r.x >> 8) + 1u), 1.0f / 16777216.0f);
    float u2 = fmul(__uint2float_rn(r.y >> 8), 1.0f / 16777216.0f);
    float rad = __fsqrt_rn(fmul(-2.0f, det_log(u1)));
    return fmul(rad, det_cos2pi(u2));
}

// Measured range of a returned beam (Sec. IV-A sensor): Gaussian noise, then
// rounding to 1/dec_scale m (half to even on the scaled value) when
// dec_scale > 0, then the clip to [r_min, r_max].  One IEEE fp32 operation
// at a time.
__device__ __forceinline__ float measured_range(float z_true, float g, float sigma, float r_min,
                                                float r_max, float dec_scale) {
    float z = fadd(z_true, fmul(sigma, g));
    if (dec_scale > 0.0f) z = fdiv(rintf(fmul(z, dec_scale)), dec_scale);
    return fminf(fmaxf(z, r_min), r_max);
}

// Fixed-point helpers: metres -> Q16 cells, and the Q16 crossing count.
__device__ __forceinline__ int q16_of(float v_m, float res) {
    return __float2int_rn(fmul(fdiv(v_m, res), 65536.0f));
}

// Number of grid-line crossings along one axis whose ray parameter is <= T
// (T in Q16 cells); crossing m sits at (n0 + m*2^16) * 2^14 / ad cells.
__device__ __forceinline__ int crossings_le(long long n0, long long ad, long long T) {
    if (ad == 0) return 0;
    long long lhs = T * ad - (n0 << 30);
    if (lhs < 0) return 0;
    return (int)(lhs >> 46) + 1;
}

// ---------------------------------------------------------------------------
// Kernel parameter block of the 2-D step (passed by value).
// ---------------------------------------------------------------------------
struct Step2DParams {
    int E, b_max, n_spawn, flags, reward_mode;
    int hit_q, miss_q, clamp_q, t_episode, Tmax;
    int window;                  // S: window side (cells) of the shared 8-bit counters
    int gt_words_max;            // shared words reserved for ground-truth bits
    int win_words_max;           // shared words reserved for 8-bit counters (4 cells/word)
    int near_words_max;          // shared words reserved for the 32-bit near block
    int dims, n_rings, Pz;       // 3-D: ring count and sensor height (Q16 voxels)
    float res, r_max, sigma, dt, v_max, w_max, d_crash, d_full, visit_cell;
    float lam_col, lam_explore, lam_abs, lam_delta, kappa, u_hi;   // fp32 copies (Eq. 7-17)
    uint2 key;
    int env_base;
    float r_min, dec_scale;      // sensor quantisation (dec_scale 0: no rounding)
    // in-step pose uncertainty (u_mode 1)
    int u_mode, uq_K;
    float uq_ds, logodds_scale;
    double uq_inv_s2, uq_q[3], uq_prior[3], uq_scale;
    double *pose_cov;            // [E, 6]
    float *u_scan;               // [E]
    // SLAM backbone in the step (u_mode 2)
    int slam_L, slam_iters, csm_n_xy, csm_n_th, csm_sep, slam_weighted;
    float csm_dth, slam_meas_info[3], slam_prior_info[3];
    double slam_wo[3];           // odometry information 1 / uq_odo_sigma^2
    size_t csm_map_bytes;                             // staged evidence map (0: read global)
    int csm_ws;                                       // its row stride, bytes
    float *win_x, *win_odo, *win_meas, *win_minfo;   // [E, L, 3]
    int *win_n;                                       // [E]
    float *slam_pred, *slam_odo;                      // [E, 3]
    float *csm_pose, *csm_match;                      // [E, 3]
    long long *csm_scores;                            // [E, 3]
    float *slam_upd_w;           // [E] this step's scan weight (u_mode 2)
    int slam_gn_iters;           // scan-to-map Gauss-Newton steps on the match (0: none)
    float *slam_gn_pose;         // [E, 3] the corrected match, the window's measurement
    const float *upd_w;          // per-env update weight, or null (unweighted)
    // per-env static description
    const int *W, *H, *B, *Vw, *Vh, *R8, *Dd;
    int *order;                  // work order of the update queue (2-D: costliest first each step)
    const float2 *elev_cs;       // 3-D: (cos, sin) of each ring's elevation
    const long long *map_off, *gtb_off, *ray_off, *visit_off;
    const float2 *beam_cs;
    const float4 *beam_df;       // in-step U: per ray (cos, sin) of its angle as double-floats (hi, lo, hi, lo)
    const long long *lut;        // [2*clamp_q + 1], entropy of L in 2^-40 nats
    const unsigned *gt_bits;
    // mutable state
    float *x, *y, *th, *u_prev;
    int *t, *g, *ep, *done;
    long long *Hq;
    short *belief;
    int *visit;
    const float *spawn;
    // per-step results
    float *z, *z_true;
    unsigned char *hit;
    unsigned *dbg_counts;
    long long *ray_cells, *gt_cells;
    float *terms, *reward;
    unsigned *far_cnt;           // [sum cells] (hits << 16 | misses) outside the window
    unsigned *far_bits;          // [sum cells / 256] touched 8-cell chunks outside the window
    int *ray_code;               // [sum B] sensing result per beam: Ku | hit << 30, -1: no cells
    void *env_sense;             // [E] EnvSense: what the sensing kernel hands to the update kernel
    int chunk;                   // cells per update-walk chunk
    int lut_words;               // shared words of the entropy half table
    int geo_words;               // shared words of the per-beam directions, walk codes and h0
    int list_words;              // shared words of the chunk map / touched-chunk list
    const int2 *bundles;         // [n_bundles] (env, first beam) of each sensing CTA
    int n_bundles, sense_block;
    // this launch
    const float *actions, *u_in;
    float *out_reward, *out_obs;
    unsigned *queue, *err;
};

constexpr int kTerms = ASLAM_N_TERMS;
constexpr double kLutScale = 1099511627776.0;   // 2^40

// Error bit of the sticky device word (a failed ASLAM_FLAG_CHECKS check or a
// singular fixed-lag window).  No kernel waits on another, so there is no
// timeout bit.
constexpr unsigned kErrChecks = 1u;

// Records the calling thread's last error message (aslam_last_error(NULL)).
void set_thread_error(const char *msg);

// 10^d as the fp32 scale of the sensor's range rounding (0: no rounding).
float range_scale(int d);

// Launchers (defined next to their kernels).
// `ev` (optional) receives an event record before the first kernel and
// after each kernel of the step: 4 events for 2-D, 2 for 3-D.
constexpr int kStep2DKernels = 2, kStep3DKernels = 1;   // 2-D: +1 with u_mode 1, +4 with u_mode 2 (+5 with its correction)
cudaError_t launch_step2d(const Step2DParams &p, int grid, int block, size_t smem,
                          cudaStream_t s, const cudaEvent_t *ev = nullptr);
cudaError_t step2d_set_smem(size_t smem);
size_t update2d_static_smem();                   // static shared bytes of the update kernel
size_t step3d_static_smem();                     // ... of the voxel step kernel
size_t env_sense_bytes();
int sense_block(int gt_words_max);
cudaError_t launch_uq2d(const Step2DParams &p, cudaStream_t s);
cudaError_t launch_slam2d(const Step2DParams &p, cudaStream_t s, const cudaEvent_t *ev);
int flgn_max_window();
cudaError_t launch_flgn(int E, int L, int iters, const float *wo, float u_scale, float *x,
                        const float *odo, const float *meas, const float *meas_info,
                        const float *prior, const float *prior_info, float *cov, float *u,
                        int *status, cudaStream_t s);
int csm_max_n();
// shared bytes of the bordered evidence maps of E envs for a search of
// +-n cells, and their row stride in bytes (*ws)
size_t csm_map_layout(const int *W, const int *H, int E, int n, int *ws);
cudaError_t csm_set_smem(size_t bytes);
cudaError_t launch_csm2d(const Step2DParams &p, int n_xy, int n_th, int sep, float dth,
                         size_t map_bytes, int ws, const float *pose_pred, const float *ranges,
                         float *pose_out, float *match, long long *scores, bool reset_empty,
                         cudaStream_t s);
cudaError_t launch_bridge_u(const float *u_old, const float *u_new, float alpha, int E,
                            float *u_out, float *obs, int row, int col, cudaStream_t s);
cudaError_t launch_step3d(const Step2DParams &p, int grid, int block, size_t smem,
                          cudaStream_t s, const cudaEvent_t *ev = nullptr);
cudaError_t step3d_set_smem(size_t smem);
cudaError_t step3d_occupancy(int block, size_t smem, int *ctas_per_sm);
cudaError_t step2d_occupancy(int block, size_t smem, int *ctas_per_sm);
cudaError_t launch_pack_gt(const uint8_t *gt, const long long *src_off, const int *W,
                           const int *H, const int *D, const long long *dst_words, unsigned *bits,
                           int E, cudaStream_t s);
cudaError_t launch_init_state(const Step2DParams &p, cudaStream_t s);
cudaError_t launch_gather_obs(const Step2DParams &p, float *obs, cudaStream_t s);
cudaError_t launch_gather_reward(const Step2DParams &p, float *out, cudaStream_t s);
cudaError_t launch_mark_done(int *done, const uint8_t *mask, int E, cudaStream_t s);
cudaError_t launch_detmath(const float *x, const float *u, int n, float *s, float *c,
                           float *l, float *c2, uint2 key, float *g, cudaStream_t st);

}  // namespace aslam
