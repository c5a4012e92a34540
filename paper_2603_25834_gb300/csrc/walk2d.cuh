// walk2d.cuh -- device helpers of the 2-D step kernels: the exact
// fixed-point beam geometry (Q16 origin, Q30 direction, the walk's in-map
// length), the walk code handed from sensing to
// the update, ground-truth bit tests, L2 prefetch, programmatic dependent
// launch, and the per-cell log-odds apply with its entropy change.
#pragma once

#include "aslam_internal.cuh"

namespace aslam {

// Walk code of a beam (sensing -> update): the index of the last cell of its
// belief walk, whether that cell takes a hit, and whether the beam returned
// at all (its range is a measurement, not r_max); -1: the walk has no cells.
constexpr int kCodeCells = 0x1fffffff;
constexpr int kCodeRet = 1 << 29;
constexpr int kCodeHit = 1 << 30;

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start once every CTA of the kernel before it has called
// pdl_trigger (so all of those CTAs already hold their resources); it runs
// its independent prologue, then pdl_wait blocks until that kernel has
// finished and its writes are visible.  Without the launch attribute both
// are no-ops.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ unsigned gt_bit(const unsigned *bits, int k) {
    return (bits[k >> 5] >> (k & 31)) & 1u;
}

// L2 prefetch of a byte range (bulk-copy engine, nothing to wait for).
__device__ __forceinline__ void prefetch_l2(const void *ptr, unsigned bytes) {
    bytes &= ~15u;
    if (bytes == 0u) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

// Fixed-point beam geometry shared by both kernels.
struct Beam {
    int sx, sy;
    long long adx, ady, nx0, ny0;
};

// Q30 direction of a beam: its angle in the robot frame rotated by the
// heading (c, s), in fp32, one rounding per operation.
__device__ __forceinline__ int2 beam_dir(const Step2DParams &p, long long ray, float c, float s) {
    const float2 cs = p.beam_cs[ray];
    const float dx = fsub(fmul(c, cs.x), fmul(s, cs.y));
    const float dy = fadd(fmul(s, cs.x), fmul(c, cs.y));
    return make_int2(__float2int_rn(fmul(dx, 1073741824.0f)), __float2int_rn(fmul(dy, 1073741824.0f)));
}

__device__ __forceinline__ Beam beam_setup(const Step2DParams &p, long long ray, int Px, int Py,
                                           int i0, int j0, float c, float s) {
    const int2 D = beam_dir(p, ray, c, s);
    const int Dx = D.x, Dy = D.y;
    Beam b;
    b.sx = (Dx > 0) - (Dx < 0);
    b.sy = (Dy > 0) - (Dy < 0);
    b.adx = Dx < 0 ? -(long long)Dx : (long long)Dx;
    b.ady = Dy < 0 ? -(long long)Dy : (long long)Dy;
    // Q16 distance from the origin to the first grid line along each axis
    b.nx0 = Dx > 0 ? ((long long)(i0 + 1) << 16) - Px
                   : (Dx < 0 ? (long long)Px - ((long long)i0 << 16) : 65536);
    b.ny0 = Dy > 0 ? ((long long)(j0 + 1) << 16) - Py
                   : (Dy < 0 ? (long long)Py - ((long long)j0 << 16) : 65536);
    return b;
}

// The traversal steps along x while e = nx*ady - ny*adx < 0 (nx, ny: Q16
// distances to the next x and y grid lines), adding ady << 16 or
// subtracting adx << 16 per step.  The low 16 bits of e never change and
// lie in [0, 2^16), so e < 0 exactly when floor(e / 2^16) < 0, and the walk
// can carry h = floor(e / 2^16) with steps +ady / -adx.  |e| <= 2^46 at the
// start (nx, ny <= 2^16, adx, ady <= 2^30) and each step moves a negative h
// up by at most 2^30 or a non-negative h down by at most 2^30, so h stays in
// [-2^30, 2^30]: a 32-bit integer.
__device__ __forceinline__ int dda_hi(long long e) { return (int)(e >> 16); }

// A 64-bit integer as an approximate float, from its 32-bit halves (exact
// 32-bit conversions only).
__device__ __forceinline__ float approx_f32(long long v) {
    return fmaf(__int2float_rn((int)(v >> 32)), 4294967296.0f, __uint2float_rn((unsigned)v));
}

// floor(D / (ad * 2^16)) for 0 <= D < 2^60, 0 < ad <= 2^30, when the quotient
// is at most a map side (8192): a float estimate (relative error ~2^-22, so
// off by at most one) corrected by exact 64-bit comparisons.
__device__ __forceinline__ long long floor_div_q16(long long D, long long ad) {
    const long long dv = ad << 16;
    const float qf = __fdividef(approx_f32(D), approx_f32(dv));
    long long q = qf < 1.0e9f ? (long long)__float2int_rd(qf) : 1000000000LL;
    q = q < 0 ? 0 : q;
    for (int t = 0; t < 8 && q * dv > D; ++t) --q;
    for (int t = 0; t < 8 && (q + 1) * dv <= D; ++t) ++q;
    return q;
}

// Number of cells of the beam's walk that lie in the W x H map (the walk
// leaves at the first crossing past the last column or row in its way).
__device__ __forceinline__ int cells_in_map(const Beam &b, int i0, int j0, int W, int H) {
    const int rx = b.sx > 0 ? W - 1 - i0 : i0;       // x-crossings that stay inside
    const int ry = b.sy > 0 ? H - 1 - j0 : j0;
    if (b.adx == 0) return b.ady == 0 ? 0x7fffffff : ry + 1;
    if (b.ady == 0) return rx + 1;
    const long long NX = b.nx0 + ((long long)rx << 16);    // the crossing that leaves along x
    const long long NY = b.ny0 + ((long long)ry << 16);    // ... along y
    if (NX * b.ady < NY * b.adx) {
        // leaves along x: y-crossings before it (ties go Y first, so <=)
        const long long D = NX * b.ady - b.ny0 * b.adx;
        const long long cy = D < 0 ? 0 : floor_div_q16(D, b.adx) + 1;
        return rx + (int)cy + 1;
    }
    // leaves along y: x-crossings strictly before it
    const long long D = NY * b.adx - b.nx0 * b.ady;
    const long long cx = D <= 0 ? 0 : floor_div_q16(D - 1, b.ady) + 1;
    return ry + (int)cx + 1;
}

// Entropy of log-odds L in 2^-40 nats from the half table h(|L|) (h is even).
__device__ __forceinline__ long long h_of(const long long *s_lut, int L) { return s_lut[abs(L)]; }

// Applies (h, m) to one cell's log-odds, scaled by the env's update weight
// wgt when wgt >= 0 (rint of the fp32 product); returns the entropy change
// (2^-40 nats).  kWeighted = false: the caller knows wgt < 0.
template <bool kWeighted = true>
__device__ __forceinline__ long long apply_cell(const Step2DParams &p, const long long *s_lut,
                                                short &L, unsigned h, unsigned m, float wgt) {
    const int l0 = L;
    int d = (int)h * p.hit_q + (int)m * p.miss_q;
    if (kWeighted && wgt >= 0.0f) d = (int)rintf(fmul(wgt, (float)d));
    int l1 = l0 + d;
    l1 = min(max(l1, -p.clamp_q), p.clamp_q);
    L = (short)l1;
    return h_of(s_lut, l1) - h_of(s_lut, l0);
}

// Applies the 8-bit counters of 8 consecutive cells (two words).
// kGeneric = false: unweighted scan, no debug counts (the common case).
template <bool kGeneric = true>
__device__ __forceinline__ long long apply8(const Step2DParams &p, const long long *s_lut,
                                            uint2 cw, int4 &lv, unsigned *dbg, float wgt) {
    short *L = reinterpret_cast<short *>(&lv);
    long long dh = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const unsigned c8 = ((q < 4 ? cw.x : cw.y) >> ((q & 3) << 3)) & 0xffu;
        if (c8) dh += apply_cell<kGeneric>(p, s_lut, L[q], c8 >> 4, c8 & 0xfu, wgt);
        if (kGeneric && dbg) dbg[q] = ((c8 >> 4) << 16) | (c8 & 0xfu);
    }
    return dh;
}

// Applies 32-bit (hits << 16 | misses) counters of 8 consecutive cells.
__device__ __forceinline__ long long apply8_wide(const Step2DParams &p, const long long *s_lut,
                                                 const uint4 &c0, const uint4 &c1, int4 &lv,
                                                 unsigned *dbg, float wgt) {
    short *L = reinterpret_cast<short *>(&lv);
    const unsigned c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    long long dh = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (c[q]) dh += apply_cell(p, s_lut, L[q], c[q] >> 16, c[q] & 0xffffu, wgt);
        if (dbg) dbg[q] = c[q];
    }
    return dh;
}

}  // namespace aslam
