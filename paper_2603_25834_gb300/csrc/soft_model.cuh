// soft_model.cuh -- the soft expected-range model of one beam (Sec. III-D scan
// residuals, the range model the scan-to-map Gauss-Newton differentiates),
// evaluated in fp32 to within about 1e-5 of the range:
//
//   samples s_k = (k+1)*ds, k < K, at q_k = (x, y) + s_k (cos phi, sin phi);
//   l_k = bilinear log-odds at q_k on cell centres (clamp to edge);
//   p_k = sigmoid(l_k);  T_0 = 1, T_{k+1} = T_k (1 - p_k);
//   r = sum_k T_k p_k s_k + T_K K ds.
//
// Where fp32 loses the accuracy:
//   * the bilinear fraction of q_k: formed as x/res + s_k cos(phi)/res in
//     fp32 it carries one ulp of the map coordinate (7.6e-6 cells at 128
//     cells), and a log-odds step of 6 per cell turns that into 5e-5 in l.
//     Here the origin u0 = x/res - 1/2 and the per-sample step ds cos(phi)/res
//     are rounded once from fp64 to Q32.32 fixed point; a sample's position
//     is the exact integer u0 + m du, so its fraction is one rounding of a
//     number below 1 (and the origin and step add 2^-27 cells at most);
//   * the direction: phi = th + beta rounded to fp32 moves a sample at
//     3.2 m by ~3e-7 m; cos/sin of th (fp64, once per env) and of beta
//     (fp64, once per beam) are rotated in fp64;
//   * the sigmoid: exp and the reciprocal are the correctly rounded library
//     forms (a few ulp), not the approximate intrinsics;
//   * the sums: the range is summed with Kahan's compensation and the
//     transmittance product is carried as a double-float, so 64 samples add
//     no more than a few ulp.
// The forward-mode tangents (d/dx, d/dy, d/dth) reuse the same samples in
// plain fp32.
#pragma once

#include "aslam_internal.cuh"

namespace aslam {

// A double-float: the unevaluated sum hi + lo of two fp32 numbers.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_of(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// (a.hi + a.lo) (b.hi + b.lo) to about 2^-44 relative: TwoProd of the high
// parts with one FMA, the cross terms added to its error.
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    const float l = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    const float s = __fadd_rn(p, l);
    return {s, __fsub_rn(l, __fsub_rn(s, p))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    const float l = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s.hi, l);
    return {h, __fsub_rn(l, __fsub_rn(h, s.hi))};
}

__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }

// The geometry of one beam in the bilinear frame (u = x/res - 1/2, the
// coordinate whose integer part is the lower-left tap's column), in Q32.32
// fixed point: sample m sits at u0 + m du exactly (integer arithmetic), so
// its fraction is one rounding of a number below 1.  The origin and the
// step are rounded once from fp64 (2^-33 cells each; 64 steps add 2^-27
// cells).
struct SoftRay {
    long long u0, v0;     // origin, Q32.32 cells
    long long du, dv;     // per-sample steps ds cos(phi)/res, ds sin(phi)/res, Q32.32
    float cp, sp;         // cos(phi), sin(phi) in fp32 (the th tangent)
};

// (ct, st) = cos/sin of the heading and (cb, sb) = cos/sin of the beam's
// angle, each a double-float of its fp64 value; dsr = ds/res.  The
// direction is rotated in fp64.
__device__ __forceinline__ SoftRay soft_ray(double u0, double v0, DF ct, DF st, DF cb, DF sb,
                                            DF dsr) {
    const double c = (double)ct.hi + (double)ct.lo, s = (double)st.hi + (double)st.lo;
    const double cbd = (double)cb.hi + (double)cb.lo, sbd = (double)sb.hi + (double)sb.lo;
    const double cphi = c * cbd - s * sbd, sphi = s * cbd + c * sbd;
    const double d = (double)dsr.hi + (double)dsr.lo;
    const double q32 = 4294967296.0;
    SoftRay r;
    r.u0 = __double2ll_rn(u0 * q32);
    r.v0 = __double2ll_rn(v0 * q32);
    r.du = __double2ll_rn(d * cphi * q32);
    r.dv = __double2ll_rn(d * sphi * q32);
    r.cp = __double2float_rn(cphi);
    r.sp = __double2float_rn(sphi);
    return r;
}

// Cell and fraction of the m-th sample along one axis: the Q32.32 position
// u0 + m d, its integer part (floor) and its fraction in [0, 1).
__device__ __forceinline__ void sample_coord(long long u0, long long d, int m, int &cell,
                                             float &frac) {
    const long long u = u0 + (long long)m * d;
    cell = (int)(u >> 32);
    frac = __fmul_rn(__uint2float_rn((unsigned)u), 2.3283064365386963e-10f);   // 2^-32
    if (frac >= 1.0f) {                  // a fraction that rounds up to 1
        frac = 0.0f;
        cell += 1;
    }
}

// p = sigmoid(l) and q = 1 - p, each without cancellation, from the
// correctly rounded exp and reciprocal.
__device__ __forceinline__ void sigmoid_pq_accurate(float l, float &pr, float &q) {
    const float e = expf(-fabsf(l));
    const float inv = __frcp_rn(__fadd_rn(1.0f, e));
    if (l >= 0.f) {
        pr = inv;
        q = __fmul_rn(e, inv);
    } else {
        pr = __fmul_rn(e, inv);
        q = inv;
    }
}

// ---------------------------------------------------------------------------
// The model on an int16 log-odds belief (the in-step forms): the map as a
// kernel reads it, bilinear taps, and one beam's range with its pose tangents.
// ---------------------------------------------------------------------------
struct Tap {
    float l, gx, gy;       // log-odds (nats) and its gradient per metre
};

// The map as the kernel reads it: the whole env grid in global memory, or
// the window [x0, x0+ww) x [y0, y0+wh) of it staged in shared memory.
struct MapView {
    const short *L;
    int W, H, x0, y0, ww;
};

// Bilinear log-odds (nats) and gradient (per metre) at the sample whose
// lower-left tap is (i0, j0) with fractions (ax, ay); taps clamped to the map.
__device__ __forceinline__ void bilinear_q(const MapView &m, float inv_res, float scale, int i0,
                                           int j0, float ax, float ay, Tap &t) {
    const int ia = min(max(i0, 0), m.W - 1) - m.x0, ib = min(max(i0 + 1, 0), m.W - 1) - m.x0;
    const int ja = min(max(j0, 0), m.H - 1) - m.y0, jb = min(max(j0 + 1, 0), m.H - 1) - m.y0;
    const float l00 = (float)m.L[ja * m.ww + ia] * scale;
    const float l10 = (float)m.L[ja * m.ww + ib] * scale;
    const float l01 = (float)m.L[jb * m.ww + ia] * scale;
    const float l11 = (float)m.L[jb * m.ww + ib] * scale;
    t.l = (1.f - ax) * (1.f - ay) * l00 + ax * (1.f - ay) * l10 + (1.f - ax) * ay * l01 +
          ax * ay * l11;
    t.gx = ((1.f - ay) * (l10 - l00) + ay * (l11 - l01)) * inv_res;
    t.gy = ((1.f - ax) * (l01 - l00) + ax * (l11 - l10)) * inv_res;
}

// The double-float transmittance times one more factor q.
__device__ __forceinline__ DF trans_mul_q(DF T, float q) {
    const float p = __fmul_rn(T.hi, q);
    const float l = __fmaf_rn(T.lo, q, __fmaf_rn(T.hi, q, -p));
    const float h = __fadd_rn(p, l);
    return {h, __fsub_rn(l, __fsub_rn(h, p))};
}

// Kahan step: (r, c) <- r + y with the running compensation c.
__device__ __forceinline__ void kahan_step(float &r, float &c, float y) {
    const float yc = __fsub_rn(y, c);
    const float t = __fadd_rn(r, yc);
    c = __fsub_rn(__fsub_rn(t, r), yc);
    r = t;
}

// Soft range of one beam on the belief view, and (J != nullptr) its
// derivatives d r / d(x, y, th) by forward-mode tangents.  K samples of ds
// metres; the range is summed with Kahan's compensation and the
// transmittance carried as a double-float.
__device__ __forceinline__ float soft_range_q(const MapView &m, float inv_res, float scale,
                                             const SoftRay &ry, int K, float ds, float r_far,
                                             float *J) {
    DF T = {1.f, 0.f};
    float r = 0.f, rc = 0.f;
    float dT0 = 0.f, dT1 = 0.f, dT2 = 0.f, dr0 = 0.f, dr1 = 0.f, dr2 = 0.f;
    Tap t;
    for (int k = 0; k < K; ++k) {
        const float sk = (float)(k + 1) * ds;
        int i0, j0;
        float ax, ay;
        sample_coord(ry.u0, ry.du, k + 1, i0, ax);
        sample_coord(ry.v0, ry.dv, k + 1, j0, ay);
        bilinear_q(m, inv_res, scale, i0, j0, ax, ay, t);
        float pr, q;
        sigmoid_pq_accurate(t.l, pr, q);
        kahan_step(r, rc, __fmul_rn(__fmul_rn(T.hi, pr), sk));
        if (J) {
            const float dpl = pr * q;
            const float d0 = dpl * t.gx, d1 = dpl * t.gy;
            const float d2 = dpl * (t.gx * (-sk * ry.sp) + t.gy * (sk * ry.cp));
            dr0 += (dT0 * pr + T.hi * d0) * sk;
            dr1 += (dT1 * pr + T.hi * d1) * sk;
            dr2 += (dT2 * pr + T.hi * d2) * sk;
            dT0 = dT0 * q - T.hi * d0;
            dT1 = dT1 * q - T.hi * d1;
            dT2 = dT2 * q - T.hi * d2;
        }
        T = trans_mul_q(T, q);
    }
    kahan_step(r, rc, __fmaf_rn(T.hi, r_far, T.lo * r_far));
    if (J) {
        J[0] = dr0 + dT0 * r_far;
        J[1] = dr1 + dT1 * r_far;
        J[2] = dr2 + dT2 * r_far;
    }
    return r;
}

}  // namespace aslam
