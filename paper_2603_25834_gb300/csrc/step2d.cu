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
constexpr int kOrderSmem = 1024;  // envs whose costs are kept in shared memory

__device__ void order_envs_by_cost(const Step2DParams &p, unsigned *s_hist, int *s_cost,
                                   int *s_max) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const EnvSense *es = reinterpret_cast<const EnvSense *>(p.env_sense);
    const bool staged = p.E <= kOrderSmem;
    for (int q = tid; q < 256; q += nt) s_hist[q] = 0u;
    if (tid == 0) *s_max = 1;
    int m = 0;
    if (staged && p.E <= 8 * nt) {
        // every load of this thread in flight at once
        int c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + u * nt;
            c[u] = e < p.E ? __ldcg(&es[e].upd_cells) : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + u * nt;
            if (e < p.E) s_cost[e] = c[u];
            m = max(m, c[u]);
        }
    } else {
        for (int e = tid; e < p.E; e += nt) {
            const int c = __ldcg(&es[e].upd_cells);
            if (staged) s_cost[e] = c;
            m = max(m, c);
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
        for (int q = tid; q < (words + 3) >> 2; q += blockDim.x) dst[q] = __ldg(&src[q]);
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
    __shared__ int s_cost[kOrderSmem];
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
        order_envs_by_cost(p, s_hist, s_cost, &s_max);
        if (tid == 0) p.queue[2] = 0u;
    }
}

// ---------------------------------------------------------------------------
// Update kernel
// ---------------------------------------------------------------------------
struct EnvShared {
    int e, W, H, B, reset, partial, R8, NB;
    int Px, Py, ri, rj, col_cell;
    int wx0, wy0, SW, SH;
    float c, s;
    long long map_off, ray_off;
    EnvStart start;
    int gt_cells;
    float dmin_meas, dmin_true;
};

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

// Walks cells s0 .. min(s0 + chunk, n) - 1 of beam b, where n = cells of its
// belief walk (all in the map; the last one takes the hit of a returned beam).
template <bool kPartial, bool kNear, bool kChecks>
__device__ __forceinline__ int walk_chunk(const Step2DParams &p, const EnvShared &sh, int b,
                                          int code, int s0, unsigned *s_win, unsigned *s_near) {
    const Beam bm = beam_setup(p, sh.ray_off + b, sh.Px, sh.Py, sh.ri, sh.rj, sh.c, sh.s);
    const int last = code & kCodeCells;              // index of the last cell
    const bool hit = (code & kCodeHit) != 0;
    const int kx = s0 ? x_steps_after(bm, s0) : 0, ky = s0 - kx;
    const int W = sh.W;
    int i = sh.ri + bm.sx * kx, j = sh.rj + bm.sy * ky;
    int k = j * W + i;
    int eh = dda_hi((bm.nx0 + ((long long)kx << 16)) * bm.ady - (bm.ny0 + ((long long)ky << 16)) * bm.adx);
    const int ady = (int)bm.ady, adx = (int)bm.adx;
    const int syW = bm.sy * W;
    const int s_end = min(last, s0 + p.chunk - 1);
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
    sh.col_cell = es.col_cell;
    sh.c = es.c;
    sh.s = es.s;
    sh.gt_cells = es.gt_cells;
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

// One persistent CTA per SM slot takes envs from a queue.  The last warp is
// the control warp: while the others walk env n it finishes env n-1 (reward,
// termination, outputs) and loads env n+1's parameters into the other half
// of a two-slot shared buffer, so neither serial step delays the CTA.
template <bool kChecks>
__global__ void __launch_bounds__(1024, 1) update2d_kernel(const Step2DParams p) {
    extern __shared__ __align__(16) unsigned smem[];
    long long *s_lut = reinterpret_cast<long long *>(smem);           // [clamp_q + 1]
    int *s_pref = reinterpret_cast<int *>(smem + p.lut_words);       // [b_max + 1]
    int *s_beam = s_pref + ((p.b_max + 1 + 3) & ~3);                  // [b_max]
    unsigned *s_win = smem + p.lut_words + 2 * ((p.b_max + 1 + 3) & ~3);
    unsigned *s_near = s_win + p.win_words_max;
    __shared__ EnvShared shb[2];
    __shared__ long long r_dh[32];
    __shared__ int r_rc[32];
    __shared__ long long s_dHq;
    __shared__ int s_rc;
    __shared__ int s_wsum[130];                  // chunk table: warp sums, offsets, totals
    __shared__ int s_tq[32 * 64];                // per-warp rings of touched chunks

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
    pdl_wait();                          // the sensing kernel's ray codes are complete
    if (tid == 0) load_env(p, (int)atomicAdd(p.queue, 1u), shb[0]);
    __syncthreads();
    int it = 0;
    for (;; ++it) {
        const EnvShared &sh = shb[it & 1];
        if (sh.e < 0) break;                         // uniform: read after a barrier

        // ---- reset, clear counters, chunk table --------------------------------
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
            const int cw = sh.partial ? (sh.SW * sh.SH + 3) >> 2 : (int)((ncell + 3) >> 2);
            uint4 *wz = reinterpret_cast<uint4 *>(s_win);
            for (int q = tid; q < (cw + 3) >> 2; q += nt) wz[q] = make_uint4(0, 0, 0, 0);
            for (int q = tid; q < sh.NB * sh.NB; q += nt) s_near[q] = 0u;
            if (debug)
                for (long long q = tid; q < ncell; q += nt) p.dbg_counts[sh.map_off + q] = 0u;
        }
        // Chunk table, one pass over the beams by all warps.  Chunks 0 ..
        // n0-1 are the first chunks of the n0 beams with cells (beam ids in
        // s_beam); the rest, in beam order, are the later chunks (s_pref:
        // running count of later chunks per beam).  Each warp scans 32 beams
        // with shuffles, warp 0 scans the warp sums; n0 and nlater are the
        // running totals (uniform).
        int n0 = 0, nlater = 0;
        if (tid == 0) s_pref[0] = 0;
        for (int b0 = 0; b0 < B; b0 += nt) {
            const int b = b0 + tid;
            const int code = b < B ? p.ray_code[sh.ray_off + b] : -1;
            int vl = code < 0 ? 0 : (code & kCodeCells) / p.chunk;    // later chunks
            int vf = code < 0 ? 0 : 1;                                  // a first chunk
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int tl = __shfl_up_sync(0xffffffffu, vl, o);
                const int tf = __shfl_up_sync(0xffffffffu, vf, o);
                if (lane >= o) {
                    vl += tl;
                    vf += tf;
                }
            }
            if (lane == 31) {
                s_wsum[warp] = vl;
                s_wsum[32 + warp] = vf;
            }
            __syncthreads();
            if (warp == 0) {
                const int tl = lane < nwarps ? s_wsum[lane] : 0;
                const int tf = lane < nwarps ? s_wsum[32 + lane] : 0;
                int il = tl, jf = tf;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int ul = __shfl_up_sync(0xffffffffu, il, o);
                    const int uf = __shfl_up_sync(0xffffffffu, jf, o);
                    if (lane >= o) {
                        il += ul;
                        jf += uf;
                    }
                }
                s_wsum[64 + lane] = il - tl;             // exclusive warp offsets
                s_wsum[96 + lane] = jf - tf;
                if (lane == 31) {
                    s_wsum[128] = il;                    // this round's totals
                    s_wsum[129] = jf;
                }
            }
            __syncthreads();
            if (b < B) {
                s_pref[b + 1] = nlater + s_wsum[64 + warp] + vl;
                if (code >= 0) s_beam[n0 + s_wsum[96 + warp] + vf - 1] = b;
            }
            nlater += s_wsum[128];
            n0 += s_wsum[129];
        }
        __syncthreads();

        // ---- belief walks, chunked (control warp: finish n-1, load n+1) ---------
        int rc = 0;
        if (control) {
            if (lane == 0) {
                if (it > 0) finish_pending(p, shb[(it - 1) & 1], s_dHq, s_rc);
                load_env(p, (int)atomicAdd(p.queue, 1u), shb[(it + 1) & 1]);
            }
        } else {
            const int total = n0 + nlater;
            for (int q = tid; q < total; q += nwalk) {
                if (q < n0) {
                    // first chunk of a beam: may touch the 32-bit block near the robot
                    const int b = s_beam[q];
                    const int code = p.ray_code[sh.ray_off + b];
                    rc += sh.partial ? walk_chunk<true, true, kChecks>(p, sh, b, code, 0, s_win, s_near)
                                     : walk_chunk<false, true, kChecks>(p, sh, b, code, 0, s_win, s_near);
                } else {
                    // later chunks start >= chunk >= 2*R8 steps out: after s steps a walk
                    // is >= s/2 cells (Chebyshev) from the robot, outside the near block
                    const int qq = q - n0;
                    int lo = 0, hi = B - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_pref[mid] <= qq) lo = mid;
                        else hi = mid - 1;
                    }
                    const int b = lo;
                    const int code = p.ray_code[sh.ray_off + b];
                    const int s0 = (qq - s_pref[b] + 1) * p.chunk;
                    rc += sh.partial ? walk_chunk<true, false, kChecks>(p, sh, b, code, s0, s_win, s_near)
                                     : walk_chunk<false, false, kChecks>(p, sh, b, code, s0, s_win, s_near);
                }
            }
        }
        __syncthreads();
        // ---- apply counters to the log-odds -------------------------------------
        long long dh = 0;
        short *Lenv = p.belief + sh.map_off;
        const float wgt = p.upd_w ? p.upd_w[e] : -1.0f;   // confidence weight of the scan
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
                dh += apply8(p, s_lut, cw2[sidx], lv, dbg ? dbg + k : nullptr, wgt);
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
                    dh += apply8_wide(p, s_lut, c0, c1, lv, dbg ? dbg + k : nullptr, wgt);
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
        __syncthreads();
        if (tid == 0) {
            long long a = 0;
            int c = 0;
            for (int w = 0; w < nwarps; ++w) {
                a += r_dh[w];
                c += r_rc[w];
            }
            s_dHq = a;
            s_rc = c;
        }
        __syncthreads();                 // s_dHq/s_rc and shb[(it+1)&1] visible
    }
    if (tid == 0) {
        if (it > 0) finish_pending(p, shb[(it - 1) & 1], s_dHq, s_rc);
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
        }
        p.ray_code[ray] = code;
    }
    if (threadIdx.x == 0) {
        EnvSense *esp = reinterpret_cast<EnvSense *>(p.env_sense) + e;
        esp->Px = Px;
        esp->Py = Py;
        esp->c = c;
        esp->s = sn;
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
        slam_replan2d_kernel<<<p.E, 128, 0, s>>>(p);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[5], s);
        if (e != cudaSuccess) return e;
        Step2DParams q = p;
        q.u_in = p.u_scan;
        q.upd_w = p.slam_weighted ? p.slam_upd_w : nullptr;
        update<<<grid, block, smem, s>>>(q);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[6], s);
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
