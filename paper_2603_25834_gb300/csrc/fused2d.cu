// fused2d.cu -- the batched 2-D environment step in one persistent kernel
// (the plain and the batched uneven forms; U_t supplied by the caller).
//
// Persistent CTAs take environments from a queue.  For one env a CTA:
//   * integrates the action (Euler unicycle, Sec. III-C Eq. 4 / Sec. IV-A)
//     and stages the env's ground truth (one bit per cell) in shared memory;
//   * walks every beam once over the ground truth with the exact fixed-point
//     traversal (Amanatides-Woo order, exact comparisons, ties Y first) to
//     its first occupied cell (Sec. IV-A LiDAR), and counts a miss for every
//     cell it leaves on the way (Sec. III-D log-odds grid): the cells before
//     the hit are exactly the cells before the measured endpoint unless the
//     range noise moves the endpoint across a cell boundary.  The noise is
//     drawn when the walk stops, and the counts are then corrected at the
//     endpoint: usually one atomic (the hit cell, or the previous cell's miss
//     turned into a hit); an endpoint farther away re-walks the short span
//     between the two;
//   * applies every touched cell once, L' = clamp(L + h*HIT + m*MISS), with
//     the entropy change from a fixed-point table;
//   * and, on its control warp while the next env walks, computes the reward
//     (Eq. 7-17), the visit grid (Eq. 8-9), termination and the observation.
// One walk per beam replaces the separate sensing walk and update re-walk of
// the two-kernel step (sense2d + update2d), which the in-step U_t modes still
// use: they need the ranges before the map is updated.
//
// Counters as in the update kernel (8-bit (hits:4 | misses:4) fields that
// cannot carry at Chebyshev distance >= R8 from the robot, a 32-bit block
// inside it, an S x S shared window and global counters beyond it for maps
// larger than the window).  A correction only removes a count the same beam
// added before (or turns its own miss into a hit with one add), so a field
// never drops below the other beams' counts and never borrows.
//
// Work order: costliest env first, by the previous step's cells (an env's
// cost changes little from one step to the next).  Each finished env adds
// itself to a 256-class histogram of its cells; the last CTA to leave turns
// the histogram into the next step's order (counting sort) and re-arms the
// queue.  The first step uses the host's static order.
#include "aslam_internal.cuh"
#include "env_common.cuh"
#include "walk2d.cuh"

namespace aslam {
namespace {

struct FusedEnv {
    int e, W, H, B, reset, partial, R8, NB, words;
    int Px, Py, ri, rj, in0, col_cell;
    int wx0, wy0, SW, SH;
    float c, s;
    long long map_off, ray_off, gtb_off;
    EnvStart start;
};

// Count increments of one beam at one cell: a miss, a hit, its own miss
// turned into a hit, and its own miss removed.  8-bit fields (hits:4 |
// misses:4) and 32-bit ones (hits << 16 | misses); the negative ones are
// two's-complement adds that never borrow (the beam's own count is there).
enum { kMiss = 0, kHit = 1, kHitForMiss = 2, kUnmiss = 3 };
__device__ __forceinline__ unsigned d8_of(int kind) {
    return kind == kMiss ? 0x01u : kind == kHit ? 0x10u : kind == kHitForMiss ? 0x0fu : 0xffffffffu;
}
__device__ __forceinline__ unsigned d32_of(int kind) {
    return kind == kMiss ? 1u : kind == kHit ? 0x10000u : kind == kHitForMiss ? 0xffffu : 0xffffffffu;
}

// Adds one increment of `kind` to cell (i, j) (flat k).  kNear: the cell may
// lie in the 32-bit block around the robot.  kChecks: a cell outside the
// env's grid records kErrChecks and is skipped.
template <bool kPartial, bool kNear, bool kChecks>
__device__ __forceinline__ void count(const Step2DParams &p, const FusedEnv &sh, int i, int j, int k,
                                      int kind, unsigned *s_win, unsigned *s_near) {
    if (kChecks && ((unsigned)i >= (unsigned)sh.W || (unsigned)j >= (unsigned)sh.H ||
                    k != j * sh.W + i)) {
        atomicOr(p.err, kErrChecks);
        return;
    }
    if (kNear) {
        const int ni = i - sh.ri + sh.R8 - 1, nj = j - sh.rj + sh.R8 - 1;
        if ((unsigned)ni < (unsigned)sh.NB && (unsigned)nj < (unsigned)sh.NB) {
            atomicAdd(&s_near[nj * sh.NB + ni], d32_of(kind));
            return;
        }
    }
    if (!kPartial) {
        atomicAdd(&s_win[k >> 2], d8_of(kind) << ((k & 3) << 3));
        return;
    }
    const int wi = i - sh.wx0, wj = j - sh.wy0;
    if ((unsigned)wi < (unsigned)sh.SW && (unsigned)wj < (unsigned)sh.SH) {
        const int q = wj * sh.SW + wi;
        atomicAdd(&s_win[q >> 2], d8_of(kind) << ((q & 3) << 3));
        return;
    }
    red_add(&p.far_cnt[sh.map_off + k], d32_of(kind));
    red_or(&p.far_bits[(sh.map_off + k) >> 8], 1u << ((k >> 3) & 31));
}

// Adds `kind` to the cells of steps s0 .. s1 of a beam's walk (each checked
// against the near block): the rare endpoint corrections that span more than
// one cell.  The walk jumps to step s0 with the exact x-step count.
template <bool kPartial, bool kChecks>
__device__ __noinline__ void count_span(const Step2DParams &p, const FusedEnv &sh, const Beam &bm,
                                        int s0, int s1, int kind, unsigned *s_win,
                                        unsigned *s_near) {
    if (s0 > s1) return;
    const int kx = s0 ? x_steps_after(bm, s0) : 0, ky = s0 - kx;
    const int W = sh.W;
    int i = sh.ri + bm.sx * kx, j = sh.rj + bm.sy * ky;
    int k = j * W + i;
    int eh = dda_hi((bm.nx0 + ((long long)kx << 16)) * bm.ady - (bm.ny0 + ((long long)ky << 16)) * bm.adx);
    const int ady = (int)bm.ady, adx = (int)bm.adx, syW = bm.sy * W;
    for (int s = s0;; ++s) {
        count<kPartial, true, kChecks>(p, sh, i, j, k, kind, s_win, s_near);
        if (s == s1) break;
        if (eh < 0) {
            i += bm.sx;
            k += bm.sx;
            eh += ady;
        } else {
            j += bm.sy;
            k += syW;
            eh -= adx;
        }
    }
}

// Per-beam results a walking thread accumulates for its env.
struct BeamSums {
    int gc, uc;
    float dmin_m, dmin_t;
};

// Senses beam b of the env and counts its inverse-sensor update.
template <bool kPartial, bool kChecks>
__device__ __forceinline__ void sense_and_count(const Step2DParams &p, const FusedEnv &sh, int b,
                                                const unsigned *gt, unsigned *s_win,
                                                unsigned *s_near, bool debug, BeamSums &acc) {
    const long long ray = sh.ray_off + b;
    bool hit = false;
    float z_true = p.r_max, z = p.r_max;
    if (sh.in0) {
        const int W = sh.W;
        const Beam bm = beam_setup(p, ray, sh.Px, sh.Py, sh.ri, sh.rj, sh.c, sh.s);
        const int nm = cells_in_map(bm, sh.ri, sh.rj, W, sh.H);
        int k = sh.rj * W + sh.ri;
        int i = sh.ri, j = sh.rj;                 // tracked when the window needs them
        int s = 0, kx = 0;
        bool lastx = false;
        if (gt_bit(gt, k)) {
            hit = true;                           // an obstacle in the robot's own cell
            z_true = 0.0f;
        } else {
            const int Ks = crossings_le(bm.nx0, bm.adx, p.Tmax) + crossings_le(bm.ny0, bm.ady, p.Tmax);
            const int nsteps = min(Ks, nm - 1);
            const int syW = bm.sy * W;
            int eh = dda_hi(bm.nx0 * bm.ady - bm.ny0 * bm.adx);
            const int ady = (int)bm.ady, nadx = -(int)bm.adx;
            // steps whose departing cell can lie in the near block: after s
            // steps the walk is >= s/2 cells (Chebyshev) from the robot
            const int nA = min(nsteps, 2 * sh.R8);
            for (; s < nA; ++s) {
                count<kPartial, true, kChecks>(p, sh, i, j, k, kMiss, s_win, s_near);
                lastx = eh < 0;
                k += lastx ? bm.sx : syW;
                i += lastx ? bm.sx : 0;
                j += lastx ? 0 : bm.sy;
                eh += lastx ? ady : nadx;
                kx += lastx;
                if (kChecks && (unsigned)k >= (unsigned)(W * sh.H)) {
                    atomicOr(p.err, kErrChecks);
                    break;
                }
                if (gt_bit(gt, k)) {
                    hit = true;
                    ++s;
                    break;
                }
            }
            if (!hit && !kChecks) {
                // four steps per iteration: their four bits loaded together and
                // tested with one branch; the block with the hit is walked again
                // one step at a time below
                for (; s + 4 <= nsteps; s += 4) {
                    const bool x1 = eh < 0;
                    const int k1 = k + (x1 ? bm.sx : syW);
                    const int e1 = eh + (x1 ? ady : nadx);
                    const bool x2 = e1 < 0;
                    const int k2 = k1 + (x2 ? bm.sx : syW);
                    const int e2 = e1 + (x2 ? ady : nadx);
                    const bool x3 = e2 < 0;
                    const int k3 = k2 + (x3 ? bm.sx : syW);
                    const int e3 = e2 + (x3 ? ady : nadx);
                    const bool x4 = e3 < 0;
                    const int k4 = k3 + (x4 ? bm.sx : syW);
                    if (gt_bit(gt, k1) | gt_bit(gt, k2) | gt_bit(gt, k3) | gt_bit(gt, k4)) break;
                    if (kPartial) {
                        const int i1 = i + (x1 ? bm.sx : 0), j1 = j + (x1 ? 0 : bm.sy);
                        const int i2 = i1 + (x2 ? bm.sx : 0), j2 = j1 + (x2 ? 0 : bm.sy);
                        const int i3 = i2 + (x3 ? bm.sx : 0), j3 = j2 + (x3 ? 0 : bm.sy);
                        count<true, false, false>(p, sh, i, j, k, kMiss, s_win, s_near);
                        count<true, false, false>(p, sh, i1, j1, k1, kMiss, s_win, s_near);
                        count<true, false, false>(p, sh, i2, j2, k2, kMiss, s_win, s_near);
                        count<true, false, false>(p, sh, i3, j3, k3, kMiss, s_win, s_near);
                        i = i3 + (x4 ? bm.sx : 0);
                        j = j3 + (x4 ? 0 : bm.sy);
                    } else {
                        count<false, false, false>(p, sh, i, j, k, kMiss, s_win, s_near);
                        count<false, false, false>(p, sh, i, j, k1, kMiss, s_win, s_near);
                        count<false, false, false>(p, sh, i, j, k2, kMiss, s_win, s_near);
                        count<false, false, false>(p, sh, i, j, k3, kMiss, s_win, s_near);
                    }
                    k = k4;
                    eh = e3 + (x4 ? ady : nadx);
                    kx += x1 + x2 + x3 + x4;
                    lastx = x4;
                }
            }
            if (!hit) {
                for (; s < nsteps; ++s) {
                    count<kPartial, false, kChecks>(p, sh, i, j, k, kMiss, s_win, s_near);
                    lastx = eh < 0;
                    k += lastx ? bm.sx : syW;
                    i += lastx ? bm.sx : 0;
                    j += lastx ? 0 : bm.sy;
                    eh += lastx ? ady : nadx;
                    kx += lastx;
                    if (kChecks && (unsigned)k >= (unsigned)(W * sh.H)) {
                        atomicOr(p.err, kErrChecks);
                        break;
                    }
                    if (gt_bit(gt, k)) {
                        hit = true;
                        ++s;
                        break;
                    }
                }
            }
            if (hit) {
                // entry parameter of the hit cell: the crossing that entered it
                const long long n = lastx ? bm.nx0 + ((long long)(kx - 1) << 16)
                                          : bm.ny0 + ((long long)(s - kx - 1) << 16);
                const long long ad = lastx ? bm.adx : bm.ady;
                z_true = fmul(fmul(fdiv(__int2float_rn((int)n), __int2float_rn((int)ad)), 16384.0f), p.res);
            }
        }
        // the walk stopped at cell s (the hit, or the last cell in range and
        // in the map); cells 0 .. s-1 hold a miss of this beam
        const int st = s;
        z = z_true;
        if (hit) {
            const float g = det_gauss(p.key, (unsigned)(p.env_base + sh.e), (unsigned)sh.start.gstep,
                                      (unsigned)b);
            z = measured_range(z_true, g, p.sigma, p.r_min, p.r_max, p.dec_scale);
        }
        const int Tz = hit ? q16_of(z, p.res) : p.Tmax;
        const int Ku = crossings_le(bm.nx0, bm.adx, Tz) + crossings_le(bm.ny0, bm.ady, Tz);
        const int el = min(Ku, nm - 1);           // last cell of the update walk
        const bool hit_end = hit && Ku < nm;
        // cell (i, j) of step st from its x-step count (the four-step loop
        // does not track them on a map without a window)
        i = sh.ri + bm.sx * kx;
        j = sh.rj + bm.sy * (st - kx);
        if (el == st) {
            count<kPartial, true, kChecks>(p, sh, i, j, k, hit_end ? kHit : kMiss, s_win, s_near);
        } else if (el == st - 1) {
            // the endpoint lies in the cell before the hit: its miss becomes the hit
            const int ip = lastx ? i - bm.sx : i, jp = lastx ? j : j - bm.sy;
            count<kPartial, true, kChecks>(p, sh, ip, jp, jp * W + ip, kHitForMiss, s_win, s_near);
        } else if (el < st) {
            count_span<kPartial, kChecks>(p, sh, bm, el, el, kHitForMiss, s_win, s_near);
            count_span<kPartial, kChecks>(p, sh, bm, el + 1, st - 1, kUnmiss, s_win, s_near);
        } else {
            count<kPartial, true, kChecks>(p, sh, i, j, k, kMiss, s_win, s_near);
            count_span<kPartial, kChecks>(p, sh, bm, st + 1, el - 1, kMiss, s_win, s_near);
            count_span<kPartial, kChecks>(p, sh, bm, el, el, hit_end ? kHit : kMiss, s_win, s_near);
        }
        acc.gc += st + 1;
        acc.uc += el + 1;
    }
    p.z[ray] = z;
    if (debug) {
        p.z_true[ray] = z_true;
        p.hit[ray] = hit ? 1 : 0;
    }
    if (p.out_obs) p.out_obs[(long long)sh.e * (p.b_max + 2) + b] = z;
    acc.dmin_m = fminf(acc.dmin_m, z);
    acc.dmin_t = fminf(acc.dmin_t, z_true);
}

// Cost class of an env for the next step's queue order: its update-walk
// cells, 256 classes of 2^cost_shift cells, costliest first.
__device__ __forceinline__ int cost_class(const Step2DParams &p, long long cells) {
    return 255 - (int)min(cells >> p.cost_shift, 255LL);
}

// Fills sh with the env of queue item `item` (sh.e = -1 past the last): its
// integrated start of the step (reset of a done env, Euler step of the
// action), the Q16 origin and heading of its beams, and the placement of the
// shared counter window; starts L2 prefetches of its belief and ground truth.
__device__ __forceinline__ void load_env(const Step2DParams &p, int item, FusedEnv &sh) {
    if (item >= p.E) {
        sh.e = -1;
        return;
    }
    const int e = p.order[item];
    const int W = p.W[e], H = p.H[e];
    const long long ncell = (long long)W * H;
    sh.words = (int)((((ncell + 31) >> 5) + 3) & ~3LL);
    sh.map_off = p.map_off[e];
    sh.gtb_off = p.gtb_off[e];
    prefetch_l2(p.belief + sh.map_off, (unsigned)min(2 * ncell, 1LL << 30));
    prefetch_l2(p.gt_bits + sh.gtb_off, 4u * (unsigned)sh.words);
    sh.e = e;
    sh.W = W;
    sh.H = H;
    sh.B = p.B[e];
    sh.R8 = p.R8[e];
    sh.NB = 2 * sh.R8 - 1;
    sh.ray_off = p.ray_off[e];
    const EnvStart st = integrate_env(p, e, ncell);
    sh.start = st;
    sh.reset = st.reset;
    sh.Px = q16_of(st.x, p.res);
    sh.Py = q16_of(st.y, p.res);
    det_sincos(st.th, sh.s, sh.c);
    sh.ri = sh.Px >> 16;
    sh.rj = sh.Py >> 16;
    sh.in0 = (unsigned)sh.ri < (unsigned)W && (unsigned)sh.rj < (unsigned)H;
    sh.col_cell = 1;                             // set from the staged ground truth
    const int S = p.window;
    sh.partial = ncell > (long long)S * S;
    if (sh.partial) {
        const int SW = min(S, W), SH = min(S, H);
        sh.SW = SW;
        sh.SH = SH;
        sh.wx0 = min(max(sh.ri - SW / 2, 0), W - SW) & ~7;
        sh.wy0 = min(max(sh.rj - SH / 2, 0), H - SH);
    } else {
        sh.SW = W;
        sh.SH = H;
        sh.wx0 = 0;
        sh.wy0 = 0;
    }
}

// Reward, termination, outputs and the next step's cost class of a finished
// env (one thread).
__device__ __forceinline__ void finish_fused(const Step2DParams &p, const FusedEnv &sh,
                                             long long dHq, long long ray_cells, long long gt_cells,
                                             float dmin_m, float dmin_t) {
    EnvTotals r;
    r.dHq = dHq;
    r.ray_cells = ray_cells;
    r.gt_cells = gt_cells;
    r.dmin_meas = dmin_m;
    r.dmin_true = dmin_t;
    finish_env(p, sh.e, sh.W, sh.H, sh.start, sh.col_cell, r, true);
    atomicAdd(&p.order_hist[cost_class(p, ray_cells)], 1u);
}

// Results of the env a CTA finished last (read by the control warp).
struct FusedTotals {
    long long dHq, rc, gc;
    float dmin_m, dmin_t;
};

template <bool kChecks>
__global__ void __launch_bounds__(1024, 1) fused2d_kernel(const Step2DParams p) {
    extern __shared__ __align__(16) unsigned smem[];
    long long *s_lut = reinterpret_cast<long long *>(smem);           // [clamp_q + 1]
    unsigned *s_gt = smem + p.lut_words;                              // [gt_words_max]
    unsigned *s_win = s_gt + p.gt_words_max;                          // [win_words_max]
    unsigned *s_near = s_win + p.win_words_max;                       // [near_words_max]
    __shared__ FusedEnv shb[2];
    __shared__ long long r_dh[32], r_rc[32], r_gc[32];
    __shared__ float r_dm[32], r_dt[32];
    __shared__ FusedTotals s_tot;
    __shared__ int s_tq[32 * 64];                // per-warp rings of touched chunks
    __shared__ unsigned s_hist[256];
    __shared__ int s_last;
    __shared__ unsigned s_bkt[32];                // beam-order classes
    __shared__ short s_perm[ASLAM_MAX_BEAMS];     // the env's beams, longest expected first

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const int nwalk = nt - 32;                       // threads of the walking warps
    const bool control = warp == nwarps - 1;
    const bool debug = (p.flags & ASLAM_FLAG_DEBUG) != 0;

    // entropy half table h(|L|), L = 0..clamp_q, shared by every env of the
    // CTA; all of a thread's loads are in flight before its first store
    {
        constexpr int kLutUnroll = 8;
        const long long *src = p.lut + p.clamp_q;
        for (int q0 = tid; q0 <= p.clamp_q; q0 += kLutUnroll * nt) {
            long long v[kLutUnroll];
#pragma unroll
            for (int u = 0; u < kLutUnroll; ++u)
                if (q0 + u * nt <= p.clamp_q) v[u] = __ldg(src + q0 + u * nt);
#pragma unroll
            for (int u = 0; u < kLutUnroll; ++u)
                if (q0 + u * nt <= p.clamp_q) s_lut[q0 + u * nt] = v[u];
        }
    }
    if (tid == 0) load_env(p, (int)atomicAdd(p.queue, 1u), shb[0]);
    __syncthreads();
    int it = 0;
    for (;; ++it) {
        const FusedEnv &sh = shb[it & 1];
        if (sh.e < 0) break;                         // uniform: read after a barrier

        // ---- reset, clear counters, stage the ground truth -----------------
        const int e = sh.e, W = sh.W, H = sh.H, B = sh.B;
        const long long ncell = (long long)W * H;
        const int nch = (int)((ncell + 7) >> 3);
        if (sh.reset) {
            int4 *bz = reinterpret_cast<int4 *>(p.belief + sh.map_off);
            for (int q = tid; q < nch; q += nt) bz[q] = make_int4(0, 0, 0, 0);
            const long long vo = p.visit_off[e], vn = p.visit_off[e + 1] - vo;
            for (long long q = tid; q < vn; q += nt) p.visit[vo + q] = -1;
        }
        {
            int words = sh.words;
            if (kChecks && words > p.gt_words_max) {
                if (tid == 0) atomicOr(p.err, kErrChecks);    // the grid exceeds the staged words
                words = 0;
            }
            const uint4 *src = reinterpret_cast<const uint4 *>(p.gt_bits + sh.gtb_off);
            uint4 *dst = reinterpret_cast<uint4 *>(s_gt);
            for (int q = tid; q < (words >> 2); q += nt) dst[q] = __ldg(&src[q]);
            const int cw = sh.partial ? (sh.SW * sh.SH + 3) >> 2 : (int)((ncell + 3) >> 2);
            uint4 *wz = reinterpret_cast<uint4 *>(s_win);
            for (int q = tid; q < (cw + 3) >> 2; q += nt) wz[q] = make_uint4(0, 0, 0, 0);
            for (int q = tid; q < sh.NB * sh.NB; q += nt) s_near[q] = 0u;
            if (debug)
                for (long long q = tid; q < ncell; q += nt) p.dbg_counts[sh.map_off + q] = 0u;
        }
        if (control) {
            // Beam order of the walk: longest expected walk first, by the
            // beam's range of the last step in 32 classes (a counting sort),
            // so that each warp walks beams of similar length.  Only the
            // schedule changes: every count is an integer sum.
            const float kscale = 32.0f / p.r_max;
            auto cls = [&](int b) {
                const float zp = p.z[sh.ray_off + b];
                return 31 - min(max((int)(zp * kscale), 0), 31);
            };
            s_bkt[lane] = 0u;
            __syncwarp();
            for (int b = lane; b < B; b += 32) atomicAdd(&s_bkt[cls(b)], 1u);
            __syncwarp();
            const unsigned c = s_bkt[lane];
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            s_bkt[lane] = incl - c;
            __syncwarp();
            for (int b = lane; b < B; b += 32) s_perm[atomicAdd(&s_bkt[cls(b)], 1u)] = (short)b;
        }
        __syncthreads();

        // ---- sense + count (control warp: finish n-1, load n+1) -------------
        BeamSums acc;
        acc.gc = 0;
        acc.uc = 0;
        acc.dmin_m = p.r_max;
        acc.dmin_t = p.r_max;
        if (control) {
            if (lane == 0) {
                FusedEnv &cur = shb[it & 1];
                cur.col_cell = !cur.in0 || gt_bit(s_gt, cur.rj * W + cur.ri);
                if (it > 0)
                    finish_fused(p, shb[(it - 1) & 1], s_tot.dHq, s_tot.rc, s_tot.gc, s_tot.dmin_m,
                                 s_tot.dmin_t);
                load_env(p, (int)atomicAdd(p.queue, 1u), shb[(it + 1) & 1]);
            }
        } else {
            for (int q = tid; q < B; q += nwalk) {
                const int b = s_perm[q];
                if (sh.partial)
                    sense_and_count<true, kChecks>(p, sh, b, s_gt, s_win, s_near, debug, acc);
                else
                    sense_and_count<false, kChecks>(p, sh, b, s_gt, s_win, s_near, debug, acc);
            }
        }
        __syncthreads();
        // ---- apply counters to the log-odds -------------------------------------
        long long dh = 0;
        short *Lenv = p.belief + sh.map_off;
        unsigned *dbg = debug ? p.dbg_counts + sh.map_off : nullptr;
        {
            // 8-cell chunks of the shared counters.  Each warp scans groups of
            // 32 chunks and queues the touched ones (ballot) in a ring of 64
            // in shared memory; whenever 32 are queued, every lane applies
            // one, so the sparse touched chunks are applied by full warps.
            const int SW = sh.SW, rch = (SW + 7) >> 3;
            const int nchunk = sh.partial ? sh.SH * rch : nch;
            const uint2 *cw2 = reinterpret_cast<const uint2 *>(s_win);
            int *ring = s_tq + 64 * warp;
            auto apply_chunk = [&](int q) {
                long long k;
                int sidx;
                if (sh.partial) {
                    const int jj = q / rch, cc = q - jj * rch;
                    k = (long long)(sh.wy0 + jj) * W + sh.wx0 + 8 * cc;
                    sidx = (jj * SW >> 3) + cc;
                } else {
                    k = 8LL * q;
                    sidx = q;
                }
                int4 lv = *reinterpret_cast<const int4 *>(Lenv + k);
                dh += apply8(p, s_lut, cw2[sidx], lv, dbg ? dbg + k : nullptr, -1.0f);
                *reinterpret_cast<int4 *>(Lenv + k) = lv;
            };
            int head = 0, nq = 0;                        // warp-uniform
            for (int base = 32 * warp; base < nchunk; base += nt) {
                const int q = base + lane;
                bool touched = false;
                if (q < nchunk) {
                    int sidx = q;
                    if (sh.partial) {
                        const int jj = q / rch;
                        sidx = (jj * SW >> 3) + q - jj * rch;
                    }
                    const uint2 c = cw2[sidx];
                    touched = (c.x | c.y) != 0u;
                }
                const unsigned m = __ballot_sync(0xffffffffu, touched);
                if (touched) ring[(head + nq + __popc(m & ((1u << lane) - 1u))) & 63] = q;
                nq += __popc(m);
                __syncwarp();
                if (nq >= 32) {
                    apply_chunk(ring[(head + lane) & 63]);
                    head = (head + 32) & 63;
                    nq -= 32;
                }
                __syncwarp();
            }
            if (lane < nq) apply_chunk(ring[(head + lane) & 63]);
        }
        if (sh.partial) {
            // chunks outside the window, found through the touched-chunk bitmap
            const long long nbw = (ncell + 255) >> 8;
            unsigned *bits = p.far_bits + (sh.map_off >> 8);
            for (long long w = tid; w < nbw; w += nt) {
                unsigned m = __ldcg(&bits[w]);
                if (!m) continue;
                bits[w] = 0u;
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    const long long k = w * 256 + bit * 8;
                    uint4 *cp = reinterpret_cast<uint4 *>(p.far_cnt + sh.map_off + k);
                    const uint4 c0 = __ldcg(cp), c1 = __ldcg(cp + 1);
                    cp[0] = make_uint4(0u, 0u, 0u, 0u);
                    cp[1] = make_uint4(0u, 0u, 0u, 0u);
                    int4 lv = *reinterpret_cast<const int4 *>(Lenv + k);
                    dh += apply8_wide(p, s_lut, c0, c1, lv, dbg ? dbg + k : nullptr, -1.0f);
                    *reinterpret_cast<int4 *>(Lenv + k) = lv;
                }
            }
        }
        __syncthreads();
        for (int q = tid; q < sh.NB * sh.NB; q += nt) {
            const int i = sh.ri + q % sh.NB - (sh.R8 - 1), j = sh.rj + q / sh.NB - (sh.R8 - 1);
            if ((unsigned)i < (unsigned)W && (unsigned)j < (unsigned)H) {
                const unsigned c = s_near[q];
                const long long k = (long long)j * W + i;
                if (c) dh += apply_cell(p, s_lut, Lenv[k], c >> 16, c & 0xffffu, -1.0f);
                if (dbg) dbg[k] = c;
            }
        }

        // ---- reductions (the finish runs on the control warp next round) -------
        long long rc = acc.uc, gc = acc.gc;
        float dm = acc.dmin_m, dt = acc.dmin_t;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            dh += __shfl_down_sync(0xffffffffu, dh, o);
            rc += __shfl_down_sync(0xffffffffu, rc, o);
            gc += __shfl_down_sync(0xffffffffu, gc, o);
            dm = fminf(dm, __shfl_down_sync(0xffffffffu, dm, o));
            dt = fminf(dt, __shfl_down_sync(0xffffffffu, dt, o));
        }
        if (lane == 0) {
            r_dh[warp] = dh;
            r_rc[warp] = rc;
            r_gc[warp] = gc;
            r_dm[warp] = dm;
            r_dt[warp] = dt;
        }
        if (p.out_obs) {
            float *o = p.out_obs + (long long)e * (p.b_max + 2);
            for (int b = B + tid; b < p.b_max; b += nt) o[b] = p.r_max;
        }
        __syncthreads();
        if (tid == 0) {
            FusedTotals t;
            t.dHq = 0;
            t.rc = 0;
            t.gc = 0;
            t.dmin_m = p.r_max;
            t.dmin_t = p.r_max;
            for (int w = 0; w < nwarps; ++w) {
                t.dHq += r_dh[w];
                t.rc += r_rc[w];
                t.gc += r_gc[w];
                t.dmin_m = fminf(t.dmin_m, r_dm[w]);
                t.dmin_t = fminf(t.dmin_t, r_dt[w]);
            }
            s_tot = t;
        }
        __syncthreads();                 // s_tot and shb[(it+1)&1] visible
    }
    // The CTA's last env; then the last CTA to leave orders the envs for the
    // next step by this step's costs (counting sort of the histogram the
    // finished envs filled) and re-arms the queue.  Thread 0's release ticket
    // publishes this CTA's writes; the CTA with the last ticket fences
    // (acquire) and its barrier extends that to all its threads.
    if (tid == 0) {
        if (it > 0)
            finish_fused(p, shb[(it - 1) & 1], s_tot.dHq, s_tot.rc, s_tot.gc, s_tot.dmin_m,
                         s_tot.dmin_t);
        unsigned old;
        asm volatile("atom.release.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(old) : "l"(p.queue + 1) : "memory");
        s_last = old == gridDim.x - 1;
        if (s_last) asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
    if (!s_last) return;
    for (int q = tid; q < 256; q += nt) s_hist[q] = __ldcg(&p.order_hist[q]);
    __syncthreads();
    if (tid < 32) {
        // exclusive scan of the 256 class counts, 8 per lane
        unsigned v[8], sum = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = s_hist[8 * tid + k];
            sum += v[k];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += t;
        }
        unsigned run = incl - sum;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s_hist[8 * tid + k] = run;
            run += v[k];
        }
        if (tid == 31) s_last = run == (unsigned)p.E;   // one entry per env
    }
    __syncthreads();
    if (s_last) {
        for (int q = tid; q < p.E; q += nt) {
            const long long c = __ldcg(&p.ray_cells[q]);
            const unsigned pos = atomicAdd(&s_hist[cost_class(p, c)], 1u);
            if (pos < (unsigned)p.E) p.order[pos] = q;
        }
    } else {
        for (int q = tid; q < p.E; q += nt) p.order[q] = q;       // not a valid histogram
    }
    for (int q = tid; q < 256; q += nt) p.order_hist[q] = 0u;
    if (tid == 0) {
        p.queue[0] = 0u;
        p.queue[1] = 0u;
    }
}

}  // namespace

size_t fused2d_static_smem() {
    cudaFuncAttributes a, b;
    if (cudaFuncGetAttributes(&a, fused2d_kernel<false>) != cudaSuccess ||
        cudaFuncGetAttributes(&b, fused2d_kernel<true>) != cudaSuccess)
        return (size_t)24576;
    return a.sharedSizeBytes > b.sharedSizeBytes ? a.sharedSizeBytes : b.sharedSizeBytes;
}

cudaError_t fused2d_set_smem(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(fused2d_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fused2d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    return e;
}

cudaError_t fused2d_occupancy(int block, size_t smem, int *ctas_per_sm) {
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fused2d_kernel<false>, block, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fused2d_kernel<true>, block, smem);
    *ctas_per_sm = a < b ? a : b;
    return e;
}

cudaError_t launch_fused2d(const Step2DParams &p, int grid, int block, size_t smem, cudaStream_t s,
                           const cudaEvent_t *ev) {
    cudaError_t e = ev ? cudaEventRecord(ev[0], s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (p.flags & ASLAM_FLAG_CHECKS)
        fused2d_kernel<true><<<grid, block, smem, s>>>(p);
    else
        fused2d_kernel<false><<<grid, block, smem, s>>>(p);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    return e;
}

}  // namespace aslam
