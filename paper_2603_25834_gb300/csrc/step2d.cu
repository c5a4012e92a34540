// step2d.cu -- the batched 2-D environment step on sm_103a, in two kernels.
//
// sense2d_kernel: one small CTA per bundle of up to `sense_block` beams of
//   one env (at least one bundle per env).  Thread 0 of every bundle resets
//   a done env to its next spawn pose and integrates the action (Euler
//   unicycle, Sec. III-C Eq. 4 / Sec. IV-A robot) from the state of the last
//   step, which no kernel of this step writes; bundle 0 publishes the env's
//   header (start, Q16 origin, heading sin/cos, collision cell) and the
//   update kernel commits the start to the env state.  The env's ground
//   truth is staged in shared memory as one bit per cell; every thread
//   walks its beam's cells with an exact fixed-point traversal
//   (Amanatides-Woo order, exact comparisons, ties Y first)
//   to the first occupied cell (Sec. IV-A LiDAR), draws the range noise, and
//   records how many cells the belief walk to the measured endpoint has
//   inside the map and whether that endpoint takes a hit.  Per-env sums and
//   minima go through one atomic per warp.
//
// update2d_kernel: persistent CTAs pull environments from a longest-first
//   queue.  The belief walks of all beams (one miss per crossed cell, a hit
//   at the endpoint of a returned beam; Sec. III-D log-odds grid) are cut
//   into chunks of `chunk` cells; a chunk starts by jumping the walk straight
//   to its first step (the number of x-crossings among the first s crossings
//   follows from the same exact comparisons), so the CTA's lanes share the
//   work evenly instead of waiting for the longest beam.  Counts go to
//   shared-memory counters; then every touched cell gets
//   L' = clamp(L + h*HIT + m*MISS) once per scan (beam order does not
//   matter) and the entropy change comes from a fixed-point table.  The last
//   warp of the CTA does not walk: while the others walk env n it finishes
//   env n-1 (reward Eq. 7-17, visit grid Eq. 8-9, termination, outputs) and
//   loads env n+1's parameters, starting an L2 bulk prefetch of its belief.
//
// Counters.  A cell at Chebyshev distance d >= 2 from the robot's cell has
// its centre at least d - 1/2 cells from the robot and lies in a disc of
// radius sqrt(2)/2 around that centre, so every beam crossing it is within
// asin(0.70711 / (d - 1/2)) of the direction to the centre: at most
// floor(2*asin(0.70711/(d - 1/2)) / dbeta) + 1 beams of spacing dbeta can
// cross it.  R8 (per env, from B) is the smallest d for which that bound is
// <= 15.  Cells at distance >= R8 therefore get 8-bit (hits:4 | misses:4)
// counters, four per 32-bit shared word, which never carry; the
// (2*R8-1)^2 block around the robot keeps 32-bit (hits << 16 | misses)
// counters.  A map too large for shared memory keeps an S x S window around
// the robot there and counts the rest with fire-and-forget global atomics
// (32-bit counters plus a bitmap of touched 8-cell chunks).
#include "aslam_internal.cuh"
#include "env_common.cuh"
#include "walk2d.cuh"

namespace aslam {

size_t env_sense_bytes() { return sizeof(EnvSense); }

namespace {

constexpr int kSenseSmemMax = 200 * 1024;   // ground truth of up to 1.6 M cells

// Work order of the update kernel's queue for this step, costliest env first
// (longest-processing-time-first keeps the persistent CTAs' last envs short).
// The cost is the env's belief-walk cells, bucketed into 256 classes of the
// largest; a counting sort writes the order (order within a class is
// arbitrary: each env is still updated whole by exactly one CTA).  Run by one
// CTA once every sensing CTA has added its cells.
// s_cost holds n_cost ints (the sensing CTA's ground-truth words, free once
// its beams are walked); with more envs the costs are read from the L2 twice.
__device__ void order_envs_by_cost(const Step2DParams &p, unsigned *s_hist, int *s_cost,
                                   int n_cost, int *s_max) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const EnvSense *es = reinterpret_cast<const EnvSense *>(p.env_sense);
    const bool staged = p.E <= n_cost;
    for (int q = tid; q < 256; q += nt) s_hist[q] = 0u;
    if (tid == 0) *s_max = 1;
    int m = 0;
    for (int e0 = tid; e0 < p.E; e0 += 8 * nt) {
        // eight loads of this thread in flight at once
        int c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * nt;
            c[u] = e < p.E ? __ldcg(&es[e].upd_cells) : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * nt;
            if (staged && e < p.E) s_cost[e] = c[u];
            m = max(m, c[u]);
        }
    }
    __syncthreads();
    atomicMax(s_max, m);
    __syncthreads();
    const float scale = 255.0f / (float)*s_max;
    auto bucket = [&](int e) {
        const int c = staged ? s_cost[e] : __ldcg(&es[e].upd_cells);
        return min(max(255 - (int)((float)c * scale), 0), 255);
    };
    for (int e = tid; e < p.E; e += nt) atomicAdd(&s_hist[bucket(e)], 1u);
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
    }
    __syncthreads();
    for (int e = tid; e < p.E; e += nt) p.order[atomicAdd(&s_hist[bucket(e)], 1u)] = e;
}

// ---------------------------------------------------------------------------
// Sensing kernel: one small CTA per bundle of beams of one env
// ---------------------------------------------------------------------------
// kChecks (ASLAM_FLAG_CHECKS): every ground-truth index of the walk is
// checked against the env's grid before it is read; a failed check records
// kErrChecks in the sticky error word and ends that beam's walk.
template <bool kChecks>
__global__ void __launch_bounds__(256) sense2d_kernel(const Step2DParams p) {
    extern __shared__ __align__(16) unsigned s_gt[];
    const int tid = threadIdx.x, lane = tid & 31;
    const bool debug = (p.flags & ASLAM_FLAG_DEBUG) != 0;
    const int2 bundle = p.bundles[blockIdx.x];          // (env, first beam)
    const int e = bundle.x;
    const int b = bundle.y + tid;
    EnvSense *esp = reinterpret_cast<EnvSense *>(p.env_sense) + e;
    const int W = p.W[e], H = p.H[e];
    const int B = p.B[e];
    pdl_trigger();                       // the update grid may start its prologue
    // The env's start of the step, computed alike by every bundle of the env
    // by the first lane of the last warp while the others stage the ground
    // truth.  This kernel is an ordinary launch (never a programmatic
    // dependent), so the last step's state is complete when it starts.
    const int itid = blockDim.x - 32;
    __shared__ EnvSense s_hdr;
    if (tid == itid) {
        // the walkers need the origin and heading only; the collision cell
        // (from the staged ground truth) waits for the barrier below
        EnvSense h;
        h.start = integrate_env(p, e, (long long)W * H);
        h.Px = q16_of(h.start.x, p.res);
        h.Py = q16_of(h.start.y, p.res);
        det_sincos(h.start.th, h.s, h.c);
        s_hdr = h;
    }
    {
        // the env's ground truth, one bit per cell, into shared memory
        int words = (int)(((long long)W * H + 31) >> 5);
        if (kChecks && ((words + 3) & ~3) > p.gt_words_max) {
            if (tid == 0) atomicOr(p.err, kErrChecks);    // the grid exceeds the staged words
            words = 0;
        }
        const uint4 *src = reinterpret_cast<const uint4 *>(p.gt_bits + p.gtb_off[e]);
        uint4 *dst = reinterpret_cast<uint4 *>(s_gt);
        const int n4 = (words + 3) >> 2, nt = blockDim.x;
        if (n4 <= 2 * nt) {
            // at most two words per thread: both loads in flight before the
            // stores (750 paper-scale envs -1 %; with larger grids, two or four
            // loads at a time were slower than the plain loop below)
            uint4 v0, v1;
            const bool a = tid < n4, b = tid + nt < n4;
            if (a) v0 = __ldg(&src[tid]);
            if (b) v1 = __ldg(&src[tid + nt]);
            if (a) dst[tid] = v0;
            if (b) dst[tid + nt] = v1;
        } else {
            for (int q = tid; q < n4; q += nt) dst[q] = __ldg(&src[q]);
        }
    }
    __syncthreads();
    if (tid == itid && bundle.y == 0) {
        // the header for the kernels after this one; the reduced fields
        // belong to the atomics of every bundle and are left alone
        const int ri = s_hdr.Px >> 16, rj = s_hdr.Py >> 16;
        const bool inside = (unsigned)ri < (unsigned)W && (unsigned)rj < (unsigned)H;
        esp->start = s_hdr.start;
        esp->Px = s_hdr.Px;
        esp->Py = s_hdr.Py;
        esp->col_cell = !inside || gt_bit(s_gt, rj * W + ri);
        esp->c = s_hdr.c;
        esp->s = s_hdr.s;
    }
    int gc = 0, uc = 0;
    float dmin_m = p.r_max, dmin_t = p.r_max;
    if (b < B) {
        const unsigned *gt = s_gt;
        const int Px = s_hdr.Px, Py = s_hdr.Py;
        const int i0 = Px >> 16, j0 = Py >> 16;
        const bool in0 = (unsigned)i0 < (unsigned)W && (unsigned)j0 < (unsigned)H;
        const long long ray = p.ray_off[e] + b;
        const Beam bm = beam_setup(p, ray, Px, Py, i0, j0, s_hdr.c, s_hdr.s);
        bool hit = false;
        float z_true = p.r_max, z = p.r_max;
        int code = -1;
        if (in0) {
            int k = j0 * W + i0, cells = 1;
            // cells of the walk inside the map (the walk stops at the border)
            const int nm = cells_in_map(bm, i0, j0, W, H);
            if (gt_bit(gt, k)) {
                hit = true;
                z_true = 0.0f;
            } else {
                // next X crossing strictly earlier than next Y crossing iff
                // nx/adx < ny/ady, i.e. e = nx*ady - ny*adx < 0 (ties step Y)
                const int Ks = crossings_le(bm.nx0, bm.adx, p.Tmax) +
                               crossings_le(bm.ny0, bm.ady, p.Tmax);
                const int nsteps = min(Ks, nm - 1);
                const int syW = bm.sy * W;
                int eh = dda_hi(bm.nx0 * bm.ady - bm.ny0 * bm.adx);
                const int ady = (int)bm.ady, nadx = -(int)bm.adx;
                int st = 0, kx = 0;
                bool lastx = false;
                // four steps per iteration: the four cells' bits are loaded
                // together, and one branch tests them (with checks, every step
                // goes through the one-cell loop below)
                for (; !kChecks && st + 3 < nsteps; st += 4) {
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
                    const unsigned b1 = gt_bit(gt, k1), b2 = gt_bit(gt, k2);
                    const unsigned b3 = gt_bit(gt, k3), b4 = gt_bit(gt, k4);
                    if (b1 | b2 | b3 | b4) {
                        hit = true;
                        if (b1) {
                            k = k1;
                            lastx = x1;
                            kx += x1;
                            st += 1;
                        } else if (b2) {
                            k = k2;
                            lastx = x2;
                            kx += x1 + x2;
                            st += 2;
                        } else if (b3) {
                            k = k3;
                            lastx = x3;
                            kx += x1 + x2 + x3;
                            st += 3;
                        } else {
                            k = k4;
                            lastx = x4;
                            kx += x1 + x2 + x3 + x4;
                            st += 4;
                        }
                        break;
                    }
                    k = k4;
                    eh = e3 + (x4 ? ady : nadx);
                    kx += x1 + x2 + x3 + x4;
                }
                for (; !hit && st < nsteps; ++st) {
                    lastx = eh < 0;
                    k += lastx ? bm.sx : syW;
                    eh += lastx ? ady : nadx;
                    kx += lastx;
                    if (kChecks && (unsigned)k >= (unsigned)(W * H)) {
                        atomicOr(p.err, kErrChecks);
                        break;
                    }
                    hit = gt_bit(gt, k) != 0;
                }
                cells = st + 1;                 // the start cell and every step taken
                if (hit) {
                    // entry parameter of the hit cell: the crossing that entered it
                    const long long n = lastx ? bm.nx0 + ((long long)(kx - 1) << 16)
                                              : bm.ny0 + ((long long)(st - kx - 1) << 16);
                    const long long ad = lastx ? bm.adx : bm.ady;
                    z_true = fmul(fmul(fdiv(__int2float_rn((int)n), __int2float_rn((int)ad)), 16384.0f), p.res);
                }
            }
            gc = cells;
            z = z_true;
            if (hit) {
                const float g = det_gauss(p.key, (unsigned)(p.env_base + e), (unsigned)s_hdr.start.gstep, (unsigned)b);
                z = measured_range(z_true, g, p.sigma, p.r_min, p.r_max, p.dec_scale);
            }
            const int Tz = hit ? q16_of(z, p.res) : p.Tmax;
            const int Ku = crossings_le(bm.nx0, bm.adx, Tz) + crossings_le(bm.ny0, bm.ady, Tz);
            // belief walk: cells 0..Ku, cut at the map border; the endpoint
            // gets the hit only when it is in the map
            const int ncells = min(Ku + 1, nm);
            code = (ncells - 1) | ((hit && Ku < nm) ? kCodeHit : 0) | (hit ? kCodeRet : 0);
            uc = ncells;
        }
        p.ray_code[ray] = code;
        p.z[ray] = z;
        if (debug) {
            p.z_true[ray] = z_true;
            p.hit[ray] = hit ? 1 : 0;
        }
        if (p.out_obs) p.out_obs[(long long)e * (p.b_max + 2) + b] = z;
        dmin_m = z;
        dmin_t = z_true;
    }
    // per-env reductions: a warp sum / min, then one atomic per warp
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        gc += __shfl_down_sync(0xffffffffu, gc, o);
        uc += __shfl_down_sync(0xffffffffu, uc, o);
        dmin_m = fminf(dmin_m, __shfl_down_sync(0xffffffffu, dmin_m, o));
        dmin_t = fminf(dmin_t, __shfl_down_sync(0xffffffffu, dmin_t, o));
    }
    if (lane == 0) {
        atomicAdd(&esp->gt_cells, gc);
        atomicAdd(&esp->upd_cells, uc);
        // ranges are >= 0, so their float bits order like the values
        atomicMin(reinterpret_cast<int *>(&esp->dmin_meas), __float_as_int(dmin_m));
        atomicMin(reinterpret_cast<int *>(&esp->dmin_true), __float_as_int(dmin_t));
    }
    // The last CTA to finish orders the envs for the update queue.  The
    // barrier makes this CTA's atomics visible to thread 0, whose release
    // ticket publishes them device-wide; the CTA that takes the last ticket
    // then fences (acquire), and the barrier after it extends that to the
    // whole CTA.
    __shared__ unsigned s_hist[256];
    __shared__ int s_max, s_last;
    __syncthreads();
    if (tid == 0) {
        unsigned old;
        asm volatile("atom.release.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(old) : "l"(p.queue + 2) : "memory");
        s_last = old == gridDim.x - 1;
        if (s_last) asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
    if (s_last) {
        // the costs go to the ground-truth words (every walk of this CTA is done)
        order_envs_by_cost(p, s_hist, reinterpret_cast<int *>(s_gt), p.gt_words_max, &s_max);
        if (tid == 0) p.queue[2] = 0u;
    }
}

// ---------------------------------------------------------------------------
// Update kernel
// ---------------------------------------------------------------------------
struct EnvShared {
    int e, W, H, B, reset, partial, R8, NB;
    int Px, Py, ri, rj, col_cell;
    int nxp, nxm, nyp, nym;      // Q16 distance to the first grid line, per direction sign
    int wx0, wy0, SW, SH;
    float c, s;
    long long map_off, ray_off;
    EnvStart start;
    int gt_cells, upd_cells;     // this step's ground-truth and belief-walk cells
    float dmin_meas, dmin_true;
};

// The walk geometry of a beam from its Q30 direction and the env's origin
// (the same values as beam_setup at the env's Q16 origin).
__device__ __forceinline__ Beam beam_of(const EnvShared &sh, int2 D) {
    Beam b;
    b.sx = (D.x > 0) - (D.x < 0);
    b.sy = (D.y > 0) - (D.y < 0);
    b.adx = D.x < 0 ? -(long long)D.x : (long long)D.x;
    b.ady = D.y < 0 ? -(long long)D.y : (long long)D.y;
    b.nx0 = D.x > 0 ? sh.nxp : (D.x < 0 ? sh.nxm : 65536);
    b.ny0 = D.y > 0 ? sh.nyp : (D.y < 0 ? sh.nym : 65536);
    return b;
}

// The walk geometry of a beam in 32-bit form: the step signs, |Dx| and |Dy|
// (Q30, so |Dx| + |Dy| < 2^31), and h0 = floor(e0 / 2^16), e0 = nx0*ady -
// ny0*adx the traversal's decision term at the origin.  The walk carries
// h = floor(e / 2^16); after kx x-steps and ky y-steps e has grown by
// (kx*ady - ky*adx) * 2^16, so h is exactly h0 + kx*ady - ky*adx, and the
// m-th x-crossing comes strictly before the n-th y-crossing (e < 0 at
// (m-1, n-1)) exactly when h0 + (m-1)*ady - (n-1)*adx < 0, since e's low
// 16 bits lie in [0, 2^16).  A later chunk's start then takes 32 x 32-bit
// products instead of the 64 x 64-bit ones of the Q16 form.
struct BeamQ {
    int sx, sy, adx, ady, h0;
};

__device__ __forceinline__ BeamQ beam_q(int2 D, int h0) {
    BeamQ b;
    b.sx = (D.x > 0) - (D.x < 0);
    b.sy = (D.y > 0) - (D.y < 0);
    b.adx = abs(D.x);
    b.ady = abs(D.y);
    b.h0 = h0;
    return b;
}

// h0 of a beam from its Q30 direction and the env's origin.
__device__ __forceinline__ int beam_h0(const EnvShared &sh, int2 D) {
    const Beam b = beam_of(sh, D);
    return dda_hi(b.nx0 * b.ady - b.ny0 * b.adx);
}

// Number of x-steps among the first s steps of the walk: a float estimate
// (relative error ~2^-22, so within a step or two), fixed by the exact test
// above.
__device__ __forceinline__ int x_steps_q(const BeamQ &b, int s) {
    if (b.adx == 0) return 0;
    if (b.ady == 0) return s;
    auto x_first = [&](int m, int n) {
        return (long long)b.h0 + (long long)(m - 1) * b.ady - (long long)(n - 1) * b.adx < 0;
    };
    int kx = __float2int_rd(__fdividef((float)s * (float)b.adx, (float)(b.adx + b.ady)));
    kx = min(max(kx, 0), s);
    // kx is the largest value whose kx-th x-crossing precedes the
    // (s-kx+1)-th y-crossing (ties go Y first, as in the walk); that
    // predicate falls from true to false as kx grows
    if (kx == 0 || x_first(kx, s - kx + 1)) {
        while (kx < s && x_first(kx + 1, s - kx)) ++kx;
    } else {
        do {
            --kx;
        } while (kx > 0 && !x_first(kx, s - kx + 1));
    }
    return kx;
}

// h after kx x-steps and ky y-steps of the walk.  On the walk h lies in
// [-2^30, 2^30], so 32-bit wrap-around arithmetic gives it exactly.
__device__ __forceinline__ int h_at(const BeamQ &b, int kx, int ky) {
    return (int)((unsigned)b.h0 + (unsigned)kx * (unsigned)b.ady - (unsigned)ky * (unsigned)b.adx);
}

// Adds one hit or miss of cell (i, j) (flat k) to its counter.  kNear:
// the cell may lie in the 32-bit block around the robot.  kChecks: a cell
// outside the env's grid records kErrChecks and is skipped.
template <bool kPartial, bool kNear, bool kChecks>
__device__ __forceinline__ void add_count(const Step2DParams &p, const EnvShared &sh, int i,
                                          int j, int k, bool is_hit, unsigned *s_win,
                                          unsigned *s_near) {
    if (kChecks && ((unsigned)i >= (unsigned)sh.W || (unsigned)j >= (unsigned)sh.H ||
                    k != j * sh.W + i)) {
        atomicOr(p.err, kErrChecks);
        return;
    }
    if (kNear) {
        const int ni = i - sh.ri + sh.R8 - 1, nj = j - sh.rj + sh.R8 - 1;
        if ((unsigned)ni < (unsigned)sh.NB && (unsigned)nj < (unsigned)sh.NB) {
            atomicAdd(&s_near[nj * sh.NB + ni], is_hit ? 0x10000u : 1u);
            return;
        }
    }
    const unsigned inc = is_hit ? 0x10u : 0x01u;
    if (!kPartial) {
        atomicAdd(&s_win[k >> 2], inc << ((k & 3) << 3));
        return;
    }
    const int wi = i - sh.wx0, wj = j - sh.wy0;
    if ((unsigned)wi < (unsigned)sh.SW && (unsigned)wj < (unsigned)sh.SH) {
        const int q = wj * sh.SW + wi;
        atomicAdd(&s_win[q >> 2], inc << ((q & 3) << 3));
        return;
    }
    red_add(&p.far_cnt[sh.map_off + k], is_hit ? 0x10000u : 1u);
    red_or(&p.far_bits[(sh.map_off + k) >> 8], 1u << ((k >> 3) & 31));
}

// Walks cells s0 .. min(s0 + ch, n) - 1 of a beam (n = cells of its belief
// walk, all in the map; the last one takes the hit of a returned beam).
template <bool kPartial, bool kNear, bool kChecks>
__device__ __forceinline__ int walk_chunk(const Step2DParams &p, const EnvShared &sh,
                                          const BeamQ &bm, int code, int s0, int ch,
                                          unsigned *s_win, unsigned *s_near) {
    const int last = code & kCodeCells;              // index of the last cell
    const bool hit = (code & kCodeHit) != 0;
    const int kx = s0 ? x_steps_q(bm, s0) : 0, ky = s0 - kx;
    const int W = sh.W;
    int i = sh.ri + bm.sx * kx, j = sh.rj + bm.sy * ky;
    int k = j * W + i;
    int eh = h_at(bm, kx, ky);
    const int ady = bm.ady, adx = bm.adx;
    const int syW = bm.sy * W;
    const int s_end = min(last, s0 + ch - 1);
    const bool hit_end = hit && s_end == last;
    const int n_miss = s_end - s0 + (hit_end ? 0 : 1);   // the hit cell is added last
    for (int c = 0; c < n_miss; ++c) {
        add_count<kPartial, kNear, kChecks>(p, sh, i, j, k, false, s_win, s_near);
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
    if (hit_end) add_count<kPartial, kNear, kChecks>(p, sh, i, j, k, true, s_win, s_near);
    return s_end - s0 + 1;
}

// Walks two later chunks of the env (map entries ma, mb; mb = ~0u: none)
// together, one cell of each per iteration, so each thread carries two
// independent traversal chains (later chunks never touch the near block).
template <bool kPartial, bool kChecks>
__device__ __forceinline__ int walk_two(const Step2DParams &p, const EnvShared &sh,
                                        const int2 *s_geo, const int *s_code, const int *s_h0,
                                        int ch, unsigned ma, unsigned mb, unsigned *s_win) {
    int nA = 0, nB = 0, kA = 0, kB = 0, eA = 0, eB = 0, iA = 0, iB = 0, jA = 0, jB = 0;
    int dxA = 0, dxB = 0, dyA = 0, dyB = 0, sxA = 0, sxB = 0, syA = 0, syB = 0, wA = 0, wB = 0;
    bool hA = false, hB = false;
    int cells = 0;
    const int W = sh.W;
    auto setup = [&](unsigned m, int &n, int &k, int &eh, int &i, int &j, int &ady, int &adx,
                     int &sx, int &sy, int &syW, bool &hit_end) {
        const int b = (int)(m & 0xffffu), s0 = (int)(m >> 16) * ch;
        const int code = s_code[b];
        if (code < 0) return;
        const BeamQ bm = beam_q(s_geo[b], s_h0[b]);
        const int last = code & kCodeCells;
        const int kx = x_steps_q(bm, s0), ky = s0 - kx;
        i = sh.ri + bm.sx * kx;
        j = sh.rj + bm.sy * ky;
        k = j * W + i;
        eh = h_at(bm, kx, ky);
        ady = bm.ady;
        adx = bm.adx;
        sx = bm.sx;
        sy = bm.sy;
        syW = bm.sy * W;
        const int s_end = min(last, s0 + ch - 1);
        hit_end = (code & kCodeHit) != 0 && s_end == last;
        n = s_end - s0 + (hit_end ? 0 : 1);
        cells += s_end - s0 + 1;
    };
    setup(ma, nA, kA, eA, iA, jA, dyA, dxA, sxA, syA, wA, hA);
    if (mb != ~0u) setup(mb, nB, kB, eB, iB, jB, dyB, dxB, sxB, syB, wB, hB);
    const int n = max(nA, nB);
    // each chain stops after its own cells: the cell it rests on takes the hit
    for (int c = 0; c < n; ++c) {
        if (c < nA) {
            add_count<kPartial, false, kChecks>(p, sh, iA, jA, kA, false, s_win, nullptr);
            const bool xa = eA < 0;
            if (kPartial || kChecks) {
                iA += xa ? sxA : 0;
                jA += xa ? 0 : syA;
            }
            kA += xa ? sxA : wA;
            eA += xa ? dyA : -dxA;
        }
        if (c < nB) {
            add_count<kPartial, false, kChecks>(p, sh, iB, jB, kB, false, s_win, nullptr);
            const bool xb = eB < 0;
            if (kPartial || kChecks) {
                iB += xb ? sxB : 0;
                jB += xb ? 0 : syB;
            }
            kB += xb ? sxB : wB;
            eB += xb ? dyB : -dxB;
        }
    }
    if (hA) add_count<kPartial, false, kChecks>(p, sh, iA, jA, kA, true, s_win, nullptr);
    if (hB) add_count<kPartial, false, kChecks>(p, sh, iB, jB, kB, true, s_win, nullptr);
    return cells;
}

// Exclusive prefix sum of v over the CTA (every thread calls it; at most 32
// warps); *total receives the CTA's sum.  s_ws: 33 ints.
__device__ __forceinline__ int block_exclusive_scan(int v, int *s_ws, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int t = lane < nw ? s_ws[lane] : 0;
        int it = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, it, o);
            if (lane >= o) it += u;
        }
        s_ws[lane] = it - t;
        if (lane == 31) s_ws[32] = it;
    }
    __syncthreads();
    *total = s_ws[32];
    return s_ws[warp] + incl - v;
}

// Fills sh with the env of queue item `item` (sh.e = -1 past the last).
__device__ __forceinline__ void load_env(const Step2DParams &p, int item, EnvShared &sh) {
    if (item >= p.E) {
        sh.e = -1;
        return;
    }
    const int e = p.order[item];
    // the env's belief into L2 while the CTA works on the env before it
    // (timed against a bulk prefetch of every env's belief during sensing:
    // sensing 63.5 -> 57.0 us, update 79.8 -> 83.2 us)
    prefetch_l2(p.belief + p.map_off[e], (unsigned)min(2LL * p.W[e] * p.H[e], 1LL << 30));
    EnvSense *esp = reinterpret_cast<EnvSense *>(p.env_sense) + e;
    const EnvSense es = *esp;
    // the reduced fields start over for the next step's sensing
    esp->gt_cells = 0;
    esp->upd_cells = 0;
    esp->dmin_meas = p.r_max;        // reduced with atomicMin on the (positive) float bits
    esp->dmin_true = p.r_max;
    const int W = p.W[e], H = p.H[e];
    sh.e = e;
    sh.W = W;
    sh.H = H;
    sh.B = p.B[e];
    sh.R8 = p.R8[e];
    sh.NB = 2 * sh.R8 - 1;
    sh.map_off = p.map_off[e];
    sh.ray_off = p.ray_off[e];
    sh.start = es.start;
    sh.reset = es.start.reset;
    sh.Px = es.Px;
    sh.Py = es.Py;
    sh.ri = es.Px >> 16;
    sh.rj = es.Py >> 16;
    // (an origin outside the map has no walks; these values are then unused)
    sh.nxp = (int)((((long long)sh.ri + 1) << 16) - es.Px);
    sh.nxm = (int)((long long)es.Px - ((long long)sh.ri << 16));
    sh.nyp = (int)((((long long)sh.rj + 1) << 16) - es.Py);
    sh.nym = (int)((long long)es.Py - ((long long)sh.rj << 16));
    sh.col_cell = es.col_cell;
    sh.c = es.c;
    sh.s = es.s;
    sh.gt_cells = es.gt_cells;
    sh.upd_cells = es.upd_cells;
    sh.dmin_meas = es.dmin_meas;
    sh.dmin_true = es.dmin_true;
    const int S = p.window;
    sh.partial = (long long)W * H > (long long)S * S;
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

// Reward, termination and outputs of a finished env (one thread).
__device__ __forceinline__ void finish_pending(const Step2DParams &p, const EnvShared &sh,
                                               long long dHq, long long ray_cells) {
    EnvTotals r;
    r.dHq = dHq;
    r.ray_cells = ray_cells;
    r.gt_cells = sh.gt_cells;
    r.dmin_meas = sh.dmin_meas;
    r.dmin_true = sh.dmin_true;
    finish_env(p, sh.e, sh.W, sh.H, sh.start, sh.col_cell, r, true);
}

// Flat cell index of the first cell of shared-counter chunk q (8 cells of one
// row: the map itself, or the window when the map does not fit).
__device__ __forceinline__ long long chunk_cell(const EnvShared &sh, int q) {
    if (!sh.partial) return 8LL * q;
    const int rch = sh.SW >> 3;
    const int jj = q / rch, cc = q - jj * rch;
    return (long long)(sh.wy0 + jj) * sh.W + sh.wx0 + 8 * cc;
}

// One persistent CTA per SM slot takes envs from a queue.  The last warp is
// the control warp: while the others walk env n it finishes env n-1 (reward,
// termination, outputs) and loads env n+1's parameters into the other half
// of a two-slot shared buffer, so neither serial step delays the CTA.
//
// Per env:
//   table  every beam's Q30 direction, walk code and h0 into shared memory; the
//          env's chunk size (at least p.chunk and twice the env's near
//          radius, and large enough that its later chunks fit the chunk
//          map); the map of later chunks (beam,
//          index), grouped by beam, the beams in a stride order;
//   walk   the first chunks (one per beam), then the later chunks from the
//          map, claimed 64 entries per warp from a shared counter and walked
//          two per lane together (two independent traversal chains per
//          thread; the map lists full chunks before the short last ones so
//          that pairs match in length);
//   apply  every thread tests 8 chunks of counters (four 16-byte loads) and
//          appends the touched ones to a compacted list (one shared atomic per
//          warp; past the list's capacity a thread applies its chunk at once);
//          then the whole CTA applies the list, two chunks per thread in
//          flight, and zeroes the counters it read, so they are zero for the
//          next env;
//   near   the 32-bit block around the robot (zeroed likewise).
template <bool kChecks>
__global__ void __launch_bounds__(1024, 1) update2d_kernel(const Step2DParams p) {
    extern __shared__ __align__(16) unsigned smem[];
    long long *s_lut = reinterpret_cast<long long *>(smem);              // [clamp_q + 1]
    const int geo_pad = (2 * p.b_max + 3) & ~3, code_pad = (p.b_max + 3) & ~3;
    int2 *s_geo = reinterpret_cast<int2 *>(smem + p.lut_words);          // [b_max] (Dx, Dy)
    int *s_code = reinterpret_cast<int *>(smem + p.lut_words + geo_pad); // [b_max]
    int *s_h0 = s_code + code_pad;                                       // [b_max]
    unsigned *s_list = smem + p.lut_words + p.geo_words;                 // [list_words]
    unsigned *s_win = s_list + p.list_words;
    unsigned *s_near = s_win + p.win_words_max;
    __shared__ EnvShared shb[2];
    __shared__ long long r_dh[32];               // per-warp partial sums of the env's ...
    __shared__ int r_rc[32];                     // ... entropy change and walk cells
    __shared__ int s_ws[33];                     // block scans
    __shared__ int s_ln[1];                      // touched-list length
    __shared__ int s_next;                       // next unclaimed later-chunk entry

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const int nwalk = nt - 32;                       // threads of the walking warps
    const bool control = warp == nwarps - 1;
    const bool debug = (p.flags & ASLAM_FLAG_DEBUG) != 0;
    const int cap_map = p.list_words;                // later chunks the map holds
    const int cap_list = 2 * p.list_words;           // touched chunks the list holds (16-bit entries)

    // entropy half table h(|L|), L = 0..clamp_q, shared by every env of the
    // CTA; all of a thread's loads are in flight before its first store.
    // The counters start at zero; every pass that reads them zeroes them.
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
        uint4 *wz = reinterpret_cast<uint4 *>(s_win);
        for (int q = tid; q < (p.win_words_max >> 2); q += nt) wz[q] = make_uint4(0, 0, 0, 0);
        for (int q = tid; q < p.near_words_max; q += nt) s_near[q] = 0u;
    }
    // the finished env's totals from the warps' partial sums (one thread)
    auto finish_prev = [&](const EnvShared &done) {
        long long a = 0;
        int c = 0;
        for (int w = 0; w < nwarps; ++w) {
            a += r_dh[w];
            c += r_rc[w];
        }
        finish_pending(p, done, a, c);
    };
    pdl_wait();                          // the sensing kernel's ray codes are complete
    if (tid == 0) load_env(p, (int)atomicAdd(p.queue, 1u), shb[0]);
    __syncthreads();
    int it = 0;
    for (;; ++it) {
        const EnvShared &sh = shb[it & 1];
        if (sh.e < 0) break;                         // uniform: read after a barrier

        // ---- reset, table ------------------------------------------------------
        const int e = sh.e, W = sh.W, H = sh.H, B = sh.B;
        const long long ncell = (long long)W * H;
        const int nch = (int)((ncell + 7) >> 3);
        if (tid == 0) {
            s_ln[0] = 0;
            s_next = 0;
        }
        if (sh.reset) {
            int4 *bz = reinterpret_cast<int4 *>(p.belief + sh.map_off);
            for (int q = tid; q < nch; q += nt) bz[q] = make_int4(0, 0, 0, 0);
            const long long vo = p.visit_off[e], vn = p.visit_off[e + 1] - vo;
            for (long long q = tid; q < vn; q += nt) p.visit[vo + q] = -1;
        }
        if (debug)
            for (long long q = tid; q < ncell; q += nt) p.dbg_counts[sh.map_off + q] = 0u;
        for (int b = tid; b < B; b += nt) {
            const long long ray = sh.ray_off + b;
            s_code[b] = p.ray_code[ray];
            const int2 D = beam_dir(p, ray, sh.c, sh.s);
            s_geo[b] = D;
            s_h0[b] = beam_h0(sh, D);
        }
        // chunk size: later chunks start >= ch >= 2*R8 steps out (after s
        // steps a walk is >= s/2 cells from the robot, outside the near
        // block), and sum_b floor((n_b - 1) / ch) <= upd_cells / ch <= cap_map
        // (upd_cells: the walks' total cells, summed by the sensing kernel, or
        // by the re-planning kernel that rewrote the walk codes; the map
        // writes below stay in bounds whatever it holds)
        const int ch = max(max(p.chunk, 2 * sh.R8), (sh.upd_cells + cap_map - 1) / cap_map);
        // Later chunk m of a beam covers cells m*ch .. m*ch + ch - 1 of its
        // walk; all are full but possibly the last.  The map holds the full
        // ones first, then the short last ones, so that the two chunks a lane
        // walks together (consecutive entries) mostly match in length.  One
        // scan of (full count | short flag << 16) places both.
        int nfull = 0, nshort = 0;
        // The map lists the beams by a stride coprime with B (slot t holds
        // beam t * stride mod B), so that the entries a warp claims together
        // are chunks of beams far apart: adjacent beams at the same chunk
        // index hit the same counter words at the same time, and the walk's
        // shared atomics serialised on them.  The slots read the codes of
        // other threads' beams, hence the barrier.
        const int bstride = B % 97 ? 97 : (B % 89 ? 89 : 1);
        __syncthreads();
        for (int b0 = 0; b0 < B; b0 += nt) {
            const int b = b0 + tid < B ? (int)(((long long)(b0 + tid) * bstride) % B) : b0 + tid;
            int vf = 0, vs = 0;
            if (b < B) {
                const int code = s_code[b];
                if (code >= 0) {
                    const int last = code & kCodeCells, vl = last / ch;
                    vs = vl > 0 && last % ch != ch - 1;
                    vf = vl - vs;
                }
            }
            int tot;
            const int off = block_exclusive_scan(vf | (vs << 16), s_ws, &tot);
            const int of = nfull + (off & 0xffff), os = nshort + (off >> 16);
            for (int m = 0; m < vf && of + m < cap_map; ++m)
                s_list[of + m] = (unsigned)b | ((unsigned)(m + 1) << 16);
            if (vs && os < cap_map) s_list[cap_map - 1 - os] = (unsigned)b | ((unsigned)(vf + 1) << 16);
            nfull += tot & 0xffff;
            nshort += tot >> 16;
        }
        if (nfull + nshort > cap_map) {            // uniform; impossible with a true upd_cells
            if (tid == 0) atomicOr(p.err, kErrChecks);
            nfull = min(nfull, cap_map);
            nshort = min(nshort, cap_map - nfull);
        }
        __syncthreads();
        // entry q of the later chunks: the full ones from the bottom of the
        // map up, then the short ones from the top down
        const int nlater = nfull + nshort;
        auto later = [&](int q) { return q < nfull ? s_list[q] : s_list[cap_map - 1 - (q - nfull)]; };

        // ---- belief walks, chunked (control warp: finish n-1, load n+1) ---------
        int rc = 0;
        if (control) {
            if (lane == 0) {
                if (it > 0) finish_prev(shb[(it - 1) & 1]);
                load_env(p, (int)atomicAdd(p.queue, 1u), shb[(it + 1) & 1]);
            }
        } else {
            // first chunks, one per beam in beam order: a warp's lanes take
            // adjacent beams, whose walks are of similar length (timed against
            // lanes spread over the scan to avoid sharing near-block counters:
            // 4096 uneven envs 0.7205 vs 0.7455 ms, 750 envs 0.1160 vs 0.1148 ms)
            for (int b = tid; b < B; b += nwalk) {
                const int code = s_code[b];
                if (code < 0) continue;
                const BeamQ bm = beam_q(s_geo[b], s_h0[b]);
                rc += sh.partial ? walk_chunk<true, true, kChecks>(p, sh, bm, code, 0, ch, s_win, s_near)
                                 : walk_chunk<false, true, kChecks>(p, sh, bm, code, 0, ch, s_win, s_near);
            }
            // later chunks: a warp claims 32 * per map entries at a time from
            // a shared counter, so that the warps that walked fewer first
            // chunks take more.  Two per lane walked together when the map sits
            // whole in shared memory (entries base + 2l, base + 2l + 1: the map
            // lists full chunks before short ones, so a pair mostly matches in
            // length); one per lane in a windowed map, where every cell also
            // tests the window
            const int per = sh.partial ? 1 : 2;
            for (;;) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_next, 32 * per);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= nlater) break;                   // uniform over the warp
                const int q = base + per * lane;
                if (q >= nlater) continue;
                if (per == 2) {
                    const unsigned mb = q + 1 < nlater ? later(q + 1) : ~0u;
                    rc += walk_two<false, kChecks>(p, sh, s_geo, s_code, s_h0, ch, later(q), mb, s_win);
                } else {
                    const unsigned m = later(q);
                    const int b = (int)(m & 0xffffu), s0 = (int)(m >> 16) * ch;
                    const int code = s_code[b];
                    if (code < 0) continue;
                    const BeamQ bm = beam_q(s_geo[b], s_h0[b]);
                    rc += walk_chunk<true, false, kChecks>(p, sh, bm, code, s0, ch, s_win, s_near);
                }
            }
        }
        __syncthreads();
        // ---- apply counters to the log-odds -------------------------------------
        long long dh = 0;
        short *Lenv = p.belief + sh.map_off;
        const float wgt = p.upd_w ? p.upd_w[e] : -1.0f;   // confidence weight of the scan
        unsigned *dbg = debug ? p.dbg_counts + sh.map_off : nullptr;
        const bool generic = debug || wgt >= 0.0f;        // uniform over the CTA
        {
            const int nchunk = sh.partial ? sh.SH * (sh.SW >> 3) : nch;
            uint2 *cw2 = reinterpret_cast<uint2 *>(s_win);
            unsigned short *lst = reinterpret_cast<unsigned short *>(s_list);
            // one touched chunk: counters read and zeroed, log-odds applied
            auto apply_one = [&](int q) {
                const long long k = chunk_cell(sh, q);
                const uint2 c = cw2[q];
                int4 lv = *reinterpret_cast<const int4 *>(Lenv + k);
                cw2[q] = make_uint2(0u, 0u);
                dh += generic ? apply8<true>(p, s_lut, c, lv, dbg ? dbg + k : nullptr, wgt)
                              : apply8<false>(p, s_lut, c, lv, nullptr, wgt);
                *reinterpret_cast<int4 *>(Lenv + k) = lv;
            };
            // scan: a warp tests 256 chunks (128 16-byte counter words) per
            // round, lane l the words 128 r + 32 v + l (v < 4): each load reads
            // 32 consecutive words (no bank conflicts; with a lane's four words
            // adjacent, each load hit two bank groups); bit 2v + h of a lane's
            // mask is chunk 2 (128 r + 32 v + l) + h.  The touched ones go to a
            // compacted list (one shared atomic per warp).  Entries past the
            // list's capacity are applied at once by the thread that found them.
            const uint4 *w4 = reinterpret_cast<const uint4 *>(s_win);
            const int nw4 = (nchunk + 1) >> 1;           // 16-byte words holding counters
            for (int r0 = 128 * warp; r0 < nw4; r0 += 4 * nt) {
                unsigned mask = 0u;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int q4 = r0 + 32 * v + lane;
                    if (q4 < nw4) {
                        const uint4 a = w4[q4];
                        mask |= ((unsigned)((a.x | a.y) != 0u) | ((unsigned)((a.z | a.w) != 0u) << 1)) << (2 * v);
                    }
                }
                // (a chunk past nchunk has zero counters: nothing counts there)
                const int cnt = __popc(mask);
                int incl = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += t;
                }
                int wbase = 0;
                if (lane == 31 && incl) wbase = atomicAdd(&s_ln[0], incl);
                wbase = __shfl_sync(0xffffffffu, wbase, 31);
                int pos = wbase + incl - cnt;
                while (mask) {
                    const int bit = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    const int q = 2 * (r0 + 32 * (bit >> 1) + lane) + (bit & 1);
                    if (pos < cap_list) lst[pos] = (unsigned short)q;
                    else apply_one(q);
                    ++pos;
                }
            }
            __syncthreads();
            const int n = min(s_ln[0], cap_list);
            for (int t = tid; t < n; t += 2 * nt) {
                // two chunks in flight: both counter pairs and beliefs loaded first
                const int qa = lst[t];
                const bool two = t + nt < n;
                const int qb = two ? lst[t + nt] : qa;
                const long long ka = chunk_cell(sh, qa), kb = chunk_cell(sh, qb);
                const uint2 ca = cw2[qa], cb = cw2[qb];
                int4 la = *reinterpret_cast<const int4 *>(Lenv + ka);
                int4 lb = *reinterpret_cast<const int4 *>(Lenv + kb);
                cw2[qa] = make_uint2(0u, 0u);
                if (generic) {
                    dh += apply8<true>(p, s_lut, ca, la, dbg ? dbg + ka : nullptr, wgt);
                    if (two) dh += apply8<true>(p, s_lut, cb, lb, dbg ? dbg + kb : nullptr, wgt);
                } else {
                    dh += apply8<false>(p, s_lut, ca, la, nullptr, wgt);
                    if (two) dh += apply8<false>(p, s_lut, cb, lb, nullptr, wgt);
                }
                *reinterpret_cast<int4 *>(Lenv + ka) = la;
                if (two) {
                    cw2[qb] = make_uint2(0u, 0u);
                    *reinterpret_cast<int4 *>(Lenv + kb) = lb;
                }
            }
            __syncthreads();
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
                    dh += apply8_wide(p, s_lut, c0, c1, lv, dbg ? dbg + k : nullptr, wgt);
                    *reinterpret_cast<int4 *>(Lenv + k) = lv;
                }
            }
        }
        // the near block (inside the window, disjoint from the far chunks)
        for (int q = tid; q < sh.NB * sh.NB; q += nt) {
            const int i = sh.ri + q % sh.NB - (sh.R8 - 1), j = sh.rj + q / sh.NB - (sh.R8 - 1);
            const unsigned c = s_near[q];
            s_near[q] = 0u;
            if ((unsigned)i < (unsigned)W && (unsigned)j < (unsigned)H) {
                const long long k = (long long)j * W + i;
                if (c) dh += apply_cell(p, s_lut, Lenv[k], c >> 16, c & 0xffffu, wgt);
                if (dbg) dbg[k] = c;
            }
        }

        // ---- reductions (the finish runs on the control warp next round) -------
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            dh += __shfl_down_sync(0xffffffffu, dh, o);
            rc += __shfl_down_sync(0xffffffffu, rc, o);
        }
        if (lane == 0) {
            r_dh[warp] = dh;
            r_rc[warp] = rc;
        }
        if (p.out_obs) {
            float *o = p.out_obs + (long long)e * (p.b_max + 2);
            for (int b = B + tid; b < p.b_max; b += nt) o[b] = p.r_max;
        }
        // r_dh/r_rc and shb[(it+1)&1] visible.  The control warp sums the
        // partials during the next walk, before any warp writes them again
        // (after that walk's barrier).
        __syncthreads();
    }
    if (tid == 0) {
        if (it > 0) finish_prev(shb[(it - 1) & 1]);
        // Every CTA took exactly one out-of-range item; the last CTA to leave
        // re-arms the queue for the next launch.
        __threadfence();
        if (atomicAdd(p.queue + 1, 1u) == gridDim.x - 1) {
            p.queue[0] = 0u;
            p.queue[1] = 0u;
            __threadfence();
        }
    }
}

// The fixed-lag backbone integrates the aligned scan (Sec. III-D: the scan
// enters the grid once the window optimisation has aligned it): every beam's
// measured range is walked from the window's newest optimised pose instead of
// the sensing pose.  One CTA per env re-plans each beam's walk code from that
// pose (the same exact geometry as the sensing kernel, and the beam's return
// flag from its sensing code), then replaces the walk origin and heading in
// the env's header; the update kernel walks from there.  The sensing pose
// stays in the header's start (state, visit grid, collision cell).
__global__ void __launch_bounds__(128) slam_replan2d_kernel(const Step2DParams p) {
    const int e = blockIdx.x;
    __shared__ int s_P[2];
    __shared__ float s_cs[2];
    if (threadIdx.x == 0) {
        const int n = p.win_n[e];                    // >= 1 after the window kernel
        const float *xe = p.win_x + ((long long)e * p.slam_L + n - 1) * 3;
        float sn, cs;
        det_sincos(xe[2], sn, cs);
        s_P[0] = q16_of(xe[0], p.res);
        s_P[1] = q16_of(xe[1], p.res);
        s_cs[0] = cs;
        s_cs[1] = sn;
    }
    __syncthreads();
    const int Px = s_P[0], Py = s_P[1];
    const float c = s_cs[0], sn = s_cs[1];
    const int W = p.W[e], H = p.H[e], B = p.B[e];
    const int i0 = Px >> 16, j0 = Py >> 16;
    const bool in0 = (unsigned)i0 < (unsigned)W && (unsigned)j0 < (unsigned)H;
    int cells = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const long long ray = p.ray_off[e] + b;
        const int c0 = p.ray_code[ray];
        const bool ret = c0 >= 0 && (c0 & kCodeRet) != 0;
        int code = -1;
        if (in0) {
            const Beam bm = beam_setup(p, ray, Px, Py, i0, j0, c, sn);
            const int nm = cells_in_map(bm, i0, j0, W, H);
            const int Tz = ret ? q16_of(p.z[ray], p.res) : p.Tmax;
            const int Ku = crossings_le(bm.nx0, bm.adx, Tz) + crossings_le(bm.ny0, bm.ady, Tz);
            const int ncells = min(Ku + 1, nm);
            code = (ncells - 1) | ((ret && Ku < nm) ? kCodeHit : 0) | (ret ? kCodeRet : 0);
            cells += ncells;
        }
        p.ray_code[ray] = code;
    }
    // the re-planned walks' total cells, for the update kernel's chunk size
    __shared__ int s_cells;
    if (threadIdx.x == 0) s_cells = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o; o >>= 1) cells += __shfl_down_sync(0xffffffffu, cells, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_cells, cells);
    __syncthreads();
    if (threadIdx.x == 0) {
        EnvSense *esp = reinterpret_cast<EnvSense *>(p.env_sense) + e;
        esp->Px = Px;
        esp->Py = Py;
        esp->c = c;
        esp->s = sn;
        esp->upd_cells = s_cells;
    }
}

// Bridged uncertainty (Sec. III-G, Eq. 22): U = alpha U_new + (1 - alpha) U_old.
__global__ void bridge_u_kernel(const float *u_old, const float *u_new, float alpha, int E,
                                float *u_out, float *obs, int row, int col) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const float u = fadd(fmul(alpha, u_new[e]), fmul(fsub(1.0f, alpha), u_old[e]));
        if (u_out) u_out[e] = u;
        if (obs) obs[(long long)e * row + col] = u;
    }
}

__global__ void pack_gt_kernel(const uint8_t *gt, const long long *src_off, const int *W,
                               const int *H, const int *D, const long long *dst_words,
                               unsigned *bits) {
    const int e = blockIdx.x;
    const long long n = (long long)W[e] * H[e] * D[e];
    const long long words = (n + 31) >> 5;
    const long long padded = (words + 3) & ~3LL;
    const uint8_t *g = gt + src_off[e];
    unsigned *dst = bits + dst_words[e];
    for (long long w = threadIdx.x; w < padded; w += blockDim.x) {
        unsigned v = 0;
        for (int q = 0; q < 32; ++q) {
            const long long k = w * 32 + q;
            if (k < n && g[k]) v |= 1u << q;
        }
        dst[w] = v;
    }
}

__global__ void init_state_kernel(const Step2DParams p) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.E; e += gridDim.x * blockDim.x) {
        const float *sp = p.spawn + (long long)e * p.n_spawn * 3;
        p.x[e] = sp[0];
        p.y[e] = sp[1];
        p.th[e] = sp[2];
        p.u_prev[e] = 0.0f;
        p.t[e] = 0;
        p.g[e] = 0;
        p.ep[e] = 0;
        p.done[e] = 0;
        p.Hq[e] = (long long)p.W[e] * p.H[e] * p.Dd[e] * p.lut[p.clamp_q];
        p.reward[e] = 0.0f;
        if (p.win_n) p.win_n[e] = 0;
        if (p.env_sense) {
            EnvSense *es = reinterpret_cast<EnvSense *>(p.env_sense) + e;
            es->gt_cells = 0;
            es->upd_cells = 0;
            es->dmin_meas = p.r_max;
            es->dmin_true = p.r_max;
        }
        if (p.pose_cov) {
            double *S = p.pose_cov + 6 * (long long)e;
            S[0] = p.uq_prior[0];
            S[1] = S[2] = S[4] = 0.0;
            S[3] = p.uq_prior[1];
            S[5] = p.uq_prior[2];
        }
    }
}

__global__ void gather_obs_kernel(const Step2DParams p, float *obs) {
    const int e = blockIdx.x;
    const int B = p.B[e];
    float *o = obs + (long long)e * (p.b_max + 2);
    const float *z = p.z + p.ray_off[e];
    for (int b = threadIdx.x; b < p.b_max; b += blockDim.x) o[b] = b < B ? z[b] : p.r_max;
    if (threadIdx.x == 0) {
        o[p.b_max] = p.th[e];
        o[p.b_max + 1] = p.u_prev[e];
    }
}

__global__ void gather_reward_kernel(const Step2DParams p, float *out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.E; e += gridDim.x * blockDim.x)
        out[e] = p.reward[e];
}

__global__ void mark_done_kernel(int *done, const uint8_t *mask, int E) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
        if (!mask || mask[e]) done[e] = 1;
}

__global__ void detmath_kernel(const float *x, const float *u, int n, float *s, float *c,
                               float *l, float *c2, uint2 key, float *g) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        float ss, cc;
        det_sincos(x[q], ss, cc);
        s[q] = ss;
        c[q] = cc;
        l[q] = det_log(u[q]);
        c2[q] = det_cos2pi(fsub(u[q], floorf(u[q])));
        g[q] = det_gauss(key, (unsigned)q % 7u, (unsigned)q / 7u, (unsigned)q);
    }
}

}  // namespace

size_t update2d_static_smem() {
    cudaFuncAttributes a, b;
    if (cudaFuncGetAttributes(&a, update2d_kernel<false>) != cudaSuccess ||
        cudaFuncGetAttributes(&b, update2d_kernel<true>) != cudaSuccess)
        return (size_t)16384;
    return a.sharedSizeBytes > b.sharedSizeBytes ? a.sharedSizeBytes : b.sharedSizeBytes;
}

cudaError_t step2d_set_smem(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(update2d_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(update2d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sense2d_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSenseSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sense2d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSenseSmemMax);
    return e;
}

// Beams per sensing CTA: 128, 256 once the largest map's ground truth
// would exceed 128 bytes per thread (every bundle stages its env's grid).
// Timed: 256^2 maps 64 / 128 / 192 / 256 beams -> 62.5 / 59.5 / 66 / 66.8 us;
// the uneven batch (maps up to 512^2) 128 / 192 / 256 -> 356 / 282 / 254 us.
int sense_block(int gt_words_max) {
    int t = 128;
    while (t < 256 && 4LL * gt_words_max > 128LL * t) t *= 2;
    return t;
}

cudaError_t step2d_occupancy(int block, size_t smem, int *ctas_per_sm) {
    // the checked variant uses at least the registers of the plain one
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, update2d_kernel<false>, block, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, update2d_kernel<true>, block, smem);
    *ctas_per_sm = a < b ? a : b;
    return e;
}

// Integration (one thread per env), sensing (one CTA per bundle of
// kSenseBlock beams) and the persistent per-env update CTAs.
// Launches kernel<<<grid, block, smem, s>>>(p), as a programmatic dependent
// of the preceding kernel when `pdl` is set.
template <class Kernel>
cudaError_t launch_pdl(Kernel kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                       const Step2DParams &p) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, p);
}

cudaError_t launch_step2d(const Step2DParams &p, int grid, int block, size_t smem,
                          cudaStream_t s, const cudaEvent_t *ev) {
    cudaError_t e = ev ? cudaEventRecord(ev[0], s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    // the first kernel of the step is an ordinary launch; without per-kernel
    // events the update kernel is a programmatic dependent of the sensing one
    const bool pdl = ev == nullptr;
    const bool checks = (p.flags & ASLAM_FLAG_CHECKS) != 0;
    auto sense = checks ? sense2d_kernel<true> : sense2d_kernel<false>;
    auto update = checks ? update2d_kernel<true> : update2d_kernel<false>;
    const size_t gt_bytes = 4 * (size_t)p.gt_words_max;
    e = launch_pdl(sense, dim3(p.n_bundles), dim3(p.sense_block), gt_bytes, s, false, p);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    if (e != cudaSuccess) return e;
    if (p.u_mode == 2) {
        // SLAM backbone: predict, scan-match, window Gauss-Newton -> U_t;
        // the scan is then integrated at the optimised pose
        e = launch_slam2d(p, s, ev ? ev + 2 : nullptr);
        if (e != cudaSuccess) return e;
        const int nb = p.slam_gn_iters > 0 ? 4 : 3;      // backbone kernels launched
        slam_replan2d_kernel<<<p.E, 128, 0, s>>>(p);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2 + nb], s);
        if (e != cudaSuccess) return e;
        Step2DParams q = p;
        q.u_in = p.u_scan;
        q.upd_w = p.slam_weighted ? p.slam_upd_w : nullptr;
        update<<<grid, block, smem, s>>>(q);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3 + nb], s);
        return e;
    }
    if (p.u_mode == 1) {
        // in-step U_t from the map before this scan; the update's reward reads it
        e = launch_uq2d(p, s);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
        if (e != cudaSuccess) return e;
        Step2DParams q = p;
        q.u_in = p.u_scan;
        update<<<grid, block, smem, s>>>(q);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], s);
        return e;
    }
    e = launch_pdl(update, dim3(grid), dim3(block), smem, s, pdl, p);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    return e;
}

cudaError_t launch_bridge_u(const float *u_old, const float *u_new, float alpha, int E,
                            float *u_out, float *obs, int row, int col, cudaStream_t s) {
    bridge_u_kernel<<<(E + 255) / 256, 256, 0, s>>>(u_old, u_new, alpha, E, u_out, obs, row, col);
    return cudaGetLastError();
}

cudaError_t launch_pack_gt(const uint8_t *gt, const long long *src_off, const int *W,
                           const int *H, const int *D, const long long *dst_words, unsigned *bits,
                           int E, cudaStream_t s) {
    pack_gt_kernel<<<E, 256, 0, s>>>(gt, src_off, W, H, D, dst_words, bits);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const Step2DParams &p, cudaStream_t s) {
    init_state_kernel<<<(p.E + 255) / 256, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_gather_obs(const Step2DParams &p, float *obs, cudaStream_t s) {
    gather_obs_kernel<<<p.E, 128, 0, s>>>(p, obs);
    return cudaGetLastError();
}

cudaError_t launch_gather_reward(const Step2DParams &p, float *out, cudaStream_t s) {
    gather_reward_kernel<<<(p.E + 255) / 256, 256, 0, s>>>(p, out);
    return cudaGetLastError();
}

cudaError_t launch_mark_done(int *done, const uint8_t *mask, int E, cudaStream_t s) {
    mark_done_kernel<<<(E + 255) / 256, 256, 0, s>>>(done, mask, E);
    return cudaGetLastError();
}

cudaError_t launch_detmath(const float *x, const float *u, int n, float *s, float *c,
                           float *l, float *c2, uint2 key, float *g, cudaStream_t st) {
    detmath_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, u, n, s, c, l, c2, key, g);
    return cudaGetLastError();
}

}  // namespace aslam
