// env_common.cuh -- per-environment parts shared by the 2-D and 3-D step
// kernels: episode reset + action integration at the start of a step, and
// the reward / termination / bookkeeping at its end (run by one thread).
#pragma once

#include "aslam_internal.cuh"

namespace aslam {

struct EnvStart {
    float x, y, th, u_prev;
    int t, gstep, reset, ep;
    long long Hq;
};

// Handed from the 2-D sensing kernel to the kernels after it, one per env:
// the integrated start of the step, the robot's Q16 cell position, heading
// and collision cell, and the sums and minima the sensing CTAs reduce into
// (reset to 0 / r_max by the update kernel once it has read them).
struct EnvSense {
    EnvStart start;
    int Px, Py, col_cell, gt_cells;
    float c, s, dmin_meas, dmin_true;
    int upd_cells;               // cells of this step's belief walks (update cost)
};

// Reset a done env to its next spawn pose, then integrate the action with
// the Euler unicycle (pre-step heading, heading wrapped to [-pi, pi)).
// Reads only: the 2-D step evaluates it in every sensing CTA of the env and
// commits it (commit_start) in the update kernel.
__device__ __forceinline__ EnvStart integrate_env(const Step2DParams &p, int e, long long ncell) {
    // every load that does not depend on the reset flag is issued first
    const int done = p.done[e], ep = p.ep[e], t0 = p.t[e], g = p.g[e];
    const float x0 = p.x[e], y0 = p.y[e], th0 = p.th[e], up0 = p.u_prev[e];
    const long long Hq0 = p.Hq[e];
    const float a_v = p.actions[2 * e], a_w = p.actions[2 * e + 1];   // 4-byte aligned input
    // ASLAM_FLAG_CHECKS: a non-finite action is a caller error.  The clamps
    // below still give it a defined value (fmaxf / fminf return the non-NaN
    // operand: NaN -> 0 and -w_max; +-Inf -> the bounds), so the step goes on.
    if ((p.flags & ASLAM_FLAG_CHECKS) && !(isfinite(a_v) && isfinite(a_w)))
        atomicOr(p.err, kErrChecks);
    EnvStart s;
    s.reset = done != 0;
    s.ep = ep;
    if (s.reset) {
        s.ep += 1;
        const float *sp = p.spawn + ((long long)e * p.n_spawn + (s.ep % p.n_spawn)) * 3;
        s.x = sp[0];
        s.y = sp[1];
        s.th = sp[2];
        s.t = 0;
        s.u_prev = 0.0f;
        s.Hq = ncell * p.lut[p.clamp_q];
    } else {
        s.x = x0;
        s.y = y0;
        s.th = th0;
        s.t = t0;
        s.u_prev = up0;
        s.Hq = Hq0;
    }
    s.t += 1;
    const float pi_f = (float)3.14159265358979323846;
    const float two_pi_f = (float)(2.0 * 3.14159265358979323846);
    const float v = fminf(fmaxf(a_v, 0.0f), p.v_max);
    const float w = fminf(fmaxf(a_w, -p.w_max), p.w_max);
    float s0, c0;
    det_sincos(s.th, s0, c0);
    s.x = fadd(s.x, fmul(fmul(v, c0), p.dt));
    s.y = fadd(s.y, fmul(fmul(v, s0), p.dt));
    float th = fadd(s.th, fmul(w, p.dt));
    if (th >= pi_f) th = fsub(th, two_pi_f);
    if (th < -pi_f) th = fadd(th, two_pi_f);
    s.th = th;
    s.gstep = g;
    return s;
}

// Writes an integrated start into the env state: pose, step, episode.
__device__ __forceinline__ void commit_start(const Step2DParams &p, int e, const EnvStart &s) {
    if (s.reset) p.ep[e] = s.ep;
    p.x[e] = s.x;
    p.y[e] = s.y;
    p.th[e] = s.th;
    p.t[e] = s.t;
}

// integrate_env + commit_start, for a step that runs in one kernel.
__device__ __forceinline__ EnvStart begin_env(const Step2DParams &p, int e, long long ncell) {
    const EnvStart s = integrate_env(p, e, ncell);
    commit_start(p, e, s);
    return s;
}

// Reductions of one env's step.
struct EnvTotals {
    long long dHq, ray_cells, gt_cells;
    float dmin_meas, dmin_true;
};

// Entropy gain, visit grid (Eq. 8-9), reward terms (Eq. 7-17), termination
// and the per-env outputs.  One thread, in fp32: every term is a product or
// quotient of a few fp32 inputs (a few ulp each), and the fp64 pipe of
// sm_103a is slow enough that fp64 here would lengthen the step.  commit:
// also write the start of the step (integrate_env) into the env state.
__device__ __forceinline__ void finish_env(const Step2DParams &p, int e, int W, int H,
                                           const EnvStart &s, int col_cell, const EnvTotals &r,
                                           bool commit) {
    if (commit) commit_start(p, e, s);
    const long long Hq = s.Hq + r.dHq;
    p.Hq[e] = Hq;
    constexpr float kInvLut = 1.0f / 1099511627776.0f;   // 2^-40, exact
    // H_{t-1} - H_t (nats): one correctly rounded conversion, an exact scaling
    const float dH = fmul(__ll2float_rn(-r.dHq), kInvLut);
    const int col = col_cell || (r.dmin_true < p.d_crash);
    const int Vw = p.Vw[e], Vh = p.Vh[e];
    const float vx0 = fmul(-0.5f, fmul((float)W, p.res));
    const float vy0 = fmul(-0.5f, fmul((float)H, p.res));
    int vi = (int)floorf(fdiv(fsub(s.x, vx0), p.visit_cell));
    int vj = (int)floorf(fdiv(fsub(s.y, vy0), p.visit_cell));
    vi = min(max(vi, 0), Vw - 1);
    vj = min(max(vj, 0), Vh - 1);
    int *vc = p.visit + p.visit_off[e] + (long long)vj * Vw + vi;
    const int last = *vc;
    float dcells = 1.0f;
    if (last >= 0)
        dcells = fminf(fmaxf(fdiv(fmul(0.5f, (float)(s.t - last)), (float)p.t_episode), 0.0f), 1.0f);
    *vc = s.t;
    const float Up = s.u_prev;
    const float U = p.u_in ? p.u_in[e] : 0.0f;
    // ASLAM_FLAG_CHECKS: a non-finite U_t (a caller input, or the in-step
    // estimate of a degenerate window) makes the reward non-finite
    if ((p.flags & ASLAM_FLAG_CHECKS) && !isfinite(U)) atomicOr(p.err, kErrChecks);
    const float dU = fsub(Up, U);                  // exact sign
    float cg = fminf(fmaxf(fdiv(fsub(p.u_hi, Up), p.u_hi), 0.0f), 1.0f);
    cg = fmul(cg, cg);
    const float iota = fminf(fmaxf(fdiv(fmaxf(dU, 0.0f), p.kappa), 0.0f), 1.0f);
    const float I = fadd(cg, fmul(fsub(1.0f, cg), iota));
    const float r_explore = fmul(fmul(p.lam_explore, dcells), I);
    const float eU = expf(Up);
    const float r_abs = fmul(fmul(p.lam_abs, eU), Up);
    const float r_delta = fmul(fmul(p.lam_delta, eU), dU);
    const float alpha = fminf(fmaxf(fdiv(fsub(r.dmin_meas, p.d_crash), fsub(p.d_full, p.d_crash)),
                                    0.0f), 1.0f);
    const float r_explore_s = fmul(r_explore, alpha);
    const float r_delta_s = dU > 0.0f ? fmul(r_delta, alpha) : r_delta;
    const float R = col ? -p.lam_col : fadd(fsub(r_explore_s, r_abs), r_delta_s);
    float *tm = p.terms + (long long)e * kTerms;
    tm[0] = dH;
    tm[1] = dcells;
    tm[2] = I;
    tm[3] = alpha;
    tm[4] = r_explore_s;
    tm[5] = r_abs;
    tm[6] = r_delta_s;
    tm[7] = R;
    tm[8] = (float)col;
    tm[9] = r.dmin_meas;
    tm[10] = r.dmin_true;
    tm[11] = fmul(__ll2float_rn(Hq), kInvLut);
    const float rew = p.reward_mode == ASLAM_REWARD_COMPOSITE ? R : dH;
    p.reward[e] = rew;
    if (p.out_reward) p.out_reward[e] = rew;
    p.done[e] = (col || s.t >= p.t_episode) ? 1 : 0;
    p.u_prev[e] = U;
    p.g[e] = s.gstep + 1;
    p.ray_cells[e] = r.ray_cells;
    p.gt_cells[e] = r.gt_cells;
    if (p.out_obs) {
        float *o = p.out_obs + (long long)e * (p.b_max + 2);
        o[p.b_max] = s.th;
        o[p.b_max + 1] = (float)U;
    }
}

}  // namespace aslam
