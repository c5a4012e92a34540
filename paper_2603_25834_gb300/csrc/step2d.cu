// step2d.cu -- the batched 2-D environment step on sm_103a.
//
// One persistent CTA takes one environment at a time from a cost-ordered
// work queue and runs the whole step for it:
//   A. thread 0: reset if the env was done, action integration (Euler
//      unicycle, Sec. III-C Eq. 4 / Sec. IV-A robot), ray origin in Q16;
//   B. all threads: stage the env's ground-truth grid (1 bit per cell) in
//      shared memory and clear the shared hit/miss counters;
//   C. one thread per beam: exact fixed-point grid traversal (Amanatides-Woo
//      order with exact 64-bit comparisons) of the ground truth until the
//      first occupied cell (Sec. IV-A LiDAR), Gaussian range noise, then a
//      second traversal of the belief grid to the measured endpoint that
//      adds one miss to every crossed cell and a hit to the endpoint of a
//      returned beam (Sec. III-D log-odds grid);
//   D. all threads: per cell, L' = clamp(L + h*HIT + m*MISS) (one clamp per
//      scan, so the result does not depend on beam order) and the change of
//      the cell's entropy from a fixed-point table;
//   E. thread 0: segmented reductions -> entropy gain, Eq. 7-17 reward,
//      visit grid (Eq. 8-9), termination; all threads: observation (Eq. 3).
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

namespace aslam {
namespace {

struct EnvShared {
    int e, W, H, B, reset, partial, R8, NB;
    int Px, Py, ri, rj, col_cell;
    int wx0, wy0, SW, SH;
    float c, s;
    long long map_off, gtb_off, ray_off;
    EnvStart start;
};

__device__ __forceinline__ unsigned gt_bit(const unsigned *bits, int k) {
    return (bits[k >> 5] >> (k & 31)) & 1u;
}

// L2 prefetch of a byte range (bulk-copy engine, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void *ptr, unsigned bytes) {
    bytes &= ~15u;
    if (bytes == 0u) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

// Grab the next queue item; for an in-range item prefetch what its step reads.
__device__ __forceinline__ int grab_item(const Step2DParams &p) {
    const int item = (int)atomicAdd(p.queue, 1u);
    if (item < p.E) {
        const int e = p.order[item];
        const long long n = (long long)p.W[e] * p.H[e];
        prefetch_l2(p.gt_bits + p.gtb_off[e], (unsigned)(((n + 127) >> 7) << 4));
        prefetch_l2(p.belief + p.map_off[e], (unsigned)min(2 * n, (long long)(1 << 30)));
    }
    return item;
}

__device__ __forceinline__ void env_prologue(const Step2DParams &p, int e, EnvShared &sh) {
    const int W = p.W[e], H = p.H[e];
    sh.e = e;
    sh.W = W;
    sh.H = H;
    sh.B = p.B[e];
    sh.R8 = p.R8[e];
    sh.NB = 2 * sh.R8 - 1;
    sh.map_off = p.map_off[e];
    sh.gtb_off = p.gtb_off[e];
    sh.ray_off = p.ray_off[e];
    const EnvStart st = begin_env(p, e, (long long)W * H);
    sh.start = st;
    sh.reset = st.reset;
    const float x = st.x, y = st.y, th = st.th;
    int Px = q16_of(x, p.res), Py = q16_of(y, p.res);
    sh.Px = Px;
    sh.Py = Py;
    int ri = Px >> 16, rj = Py >> 16;
    sh.ri = ri;
    sh.rj = rj;
    int inside = (unsigned)ri < (unsigned)W && (unsigned)rj < (unsigned)H;
    sh.col_cell = !inside || gt_bit(p.gt_bits + sh.gtb_off, rj * W + ri);
    float s1, c1;
    det_sincos(th, s1, c1);
    sh.c = c1;
    sh.s = s1;
    const int S = p.window;
    int partial = (long long)W * H > (long long)S * S;
    sh.partial = partial;
    if (partial) {
        int SW = min(S, W), SH = min(S, H);
        sh.SW = SW;
        sh.SH = SH;
        sh.wx0 = min(max(ri - SW / 2, 0), W - SW) & ~7;
        sh.wy0 = min(max(rj - SH / 2, 0), H - SH);
    } else {
        sh.SW = W;
        sh.SH = H;
        sh.wx0 = 0;
        sh.wy0 = 0;
    }
}

// Adds (or, with sign < 0, removes) one hit or miss of cell (i, j) (flat k).
template <bool kPartial>
__device__ __forceinline__ void add_count(const Step2DParams &p, const EnvShared &sh, int i,
                                          int j, int k, bool is_hit, unsigned *s_win,
                                          unsigned *s_near) {
    const int ni = i - sh.ri + sh.R8 - 1, nj = j - sh.rj + sh.R8 - 1;
    if ((unsigned)ni < (unsigned)sh.NB && (unsigned)nj < (unsigned)sh.NB) {
        atomicAdd(&s_near[nj * sh.NB + ni], is_hit ? 0x10000u : 1u);
        return;
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
    atomicAdd(&p.far_cnt[sh.map_off + k], is_hit ? 0x10000u : 1u);
    atomicOr(&p.far_bits[(sh.map_off + k) >> 8], 1u << ((k >> 3) & 31));
}

// One beam: ground-truth traversal, noise, belief traversal with counting.
template <bool kPartial>
__device__ __forceinline__ void trace_beam(const Step2DParams &p, const EnvShared &sh, int b,
                                           const unsigned *s_gt, unsigned *s_win,
                                           unsigned *s_near, int &rc, int &gc, float &dmin_m,
                                           float &dmin_t) {
    const float2 cs = p.beam_cs[sh.ray_off + b];
    const float dx = fsub(fmul(sh.c, cs.x), fmul(sh.s, cs.y));
    const float dy = fadd(fmul(sh.s, cs.x), fmul(sh.c, cs.y));
    const int Dx = __float2int_rn(fmul(dx, 1073741824.0f));
    const int Dy = __float2int_rn(fmul(dy, 1073741824.0f));
    const int W = sh.W, H = sh.H;
    const int Px = sh.Px, Py = sh.Py;
    const int i0 = sh.ri, j0 = sh.rj;
    const bool in0 = (unsigned)i0 < (unsigned)W && (unsigned)j0 < (unsigned)H;
    const int sx = (Dx > 0) - (Dx < 0), sy = (Dy > 0) - (Dy < 0);
    const long long adx = Dx < 0 ? -(long long)Dx : (long long)Dx;
    const long long ady = Dy < 0 ? -(long long)Dy : (long long)Dy;
    // Q16 distance from the origin to the first grid line along each axis.
    const long long nx0 = Dx > 0 ? ((long long)(i0 + 1) << 16) - Px
                                 : (Dx < 0 ? (long long)Px - ((long long)i0 << 16) : 65536);
    const long long ny0 = Dy > 0 ? ((long long)(j0 + 1) << 16) - Py
                                 : (Dy < 0 ? (long long)Py - ((long long)j0 << 16) : 65536);
    // The next X crossing is strictly earlier than the next Y crossing iff
    // nx/adx < ny/ady, i.e. e = nx*ady - ny*adx < 0 (ties step Y).
    const long long e0 = nx0 * ady - ny0 * adx;
    const long long dA = ady << 16, dB = adx << 16;
    const int syW = sy * W;

    bool hit = false;
    float z_true = p.r_max;
    int cells_gt = 0;
    if (in0) {
        int k = j0 * W + i0;
        cells_gt = 1;
        if (gt_bit(s_gt, k)) {
            hit = true;
            z_true = 0.0f;
        } else {
            const int Ks = crossings_le(nx0, adx, p.Tmax) + crossings_le(ny0, ady, p.Tmax);
            int i = i0, j = j0;
            long long e = e0;
            bool lastx = false;
            for (int s = 0; s < Ks; ++s) {
                lastx = e < 0;
                if (lastx) {
                    i += sx;
                    k += sx;
                    e += dA;
                } else {
                    j += sy;
                    k += syW;
                    e -= dB;
                }
                if ((unsigned)i >= (unsigned)W || (unsigned)j >= (unsigned)H) break;
                ++cells_gt;
                if (gt_bit(s_gt, k)) {
                    hit = true;
                    break;
                }
            }
            if (hit) {
                // entry parameter of the hit cell: the crossing that entered it
                const long long n = lastx ? nx0 + ((long long)(abs(i - i0) - 1) << 16)
                                          : ny0 + ((long long)(abs(j - j0) - 1) << 16);
                const long long ad = lastx ? adx : ady;
                z_true = fmul(fmul(fdiv(__ll2float_rn(n), __ll2float_rn(ad)), 16384.0f), p.res);
            }
        }
    }
    float z = z_true;
    if (hit) {
        const float gz = det_gauss(p.key, (unsigned)sh.e, (unsigned)sh.start.gstep, (unsigned)b);
        z = fminf(fmaxf(fadd(z_true, fmul(p.sigma, gz)), 0.0f), p.r_max);
    }
    const int Tz = hit ? q16_of(z, p.res) : p.Tmax;

    int cells_upd = 0;
    if (in0) {
        const int Ku = crossings_le(nx0, adx, Tz) + crossings_le(ny0, ady, Tz);
        int i = i0, j = j0, k = j0 * W + i0;
        long long e = e0;
        for (int s = 0;; ++s) {
            const bool last = s == Ku;
            add_count<kPartial>(p, sh, i, j, k, last && hit, s_win, s_near);
            ++cells_upd;
            if (last) break;
            if (e < 0) {
                i += sx;
                k += sx;
                e += dA;
            } else {
                j += sy;
                k += syW;
                e -= dB;
            }
            if ((unsigned)i >= (unsigned)W || (unsigned)j >= (unsigned)H) break;
        }
    }
    const long long ro = sh.ray_off + b;
    p.z[ro] = z;
    if (p.flags & ASLAM_FLAG_DEBUG) {
        p.z_true[ro] = z_true;
        p.hit[ro] = hit ? 1 : 0;
    }
    if (p.out_obs) p.out_obs[(long long)sh.e * (p.b_max + 2) + b] = z;
    rc += cells_upd;
    gc += cells_gt;
    dmin_m = fminf(dmin_m, z);
    dmin_t = fminf(dmin_t, z_true);
}

// Applies (h, m) to one cell's log-odds; returns the entropy change (2^-40 nats).
__device__ __forceinline__ long long apply_cell(const Step2DParams &p, short &L, unsigned h,
                                                unsigned m) {
    const int l0 = L;
    int l1 = l0 + (int)h * p.hit_q + (int)m * p.miss_q;
    l1 = min(max(l1, -p.clamp_q), p.clamp_q);
    L = (short)l1;
    return __ldg(&p.lut[l1 + p.clamp_q]) - __ldg(&p.lut[l0 + p.clamp_q]);
}

// Applies the 8-bit counters of 8 consecutive cells (two words) to their
// int16 log-odds held in one int4.
__device__ __forceinline__ long long apply8(const Step2DParams &p, uint2 cw, int4 &lv,
                                            unsigned *dbg) {
    short *L = reinterpret_cast<short *>(&lv);
    long long dh = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const unsigned c8 = ((q < 4 ? cw.x : cw.y) >> ((q & 3) << 3)) & 0xffu;
        if (c8) dh += apply_cell(p, L[q], c8 >> 4, c8 & 0xfu);
        if (dbg) dbg[q] = ((c8 >> 4) << 16) | (c8 & 0xfu);
    }
    return dh;
}

// Applies 32-bit (hits << 16 | misses) counters of 8 consecutive cells.
__device__ __forceinline__ long long apply8_wide(const Step2DParams &p, const uint4 &c0,
                                                 const uint4 &c1, int4 &lv, unsigned *dbg) {
    short *L = reinterpret_cast<short *>(&lv);
    const unsigned c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    long long dh = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (c[q]) dh += apply_cell(p, L[q], c[q] >> 16, c[q] & 0xffffu);
        if (dbg) dbg[q] = c[q];
    }
    return dh;
}

constexpr int kUnroll = 2;

__global__ void __launch_bounds__(1024, 1) step2d_kernel(const Step2DParams p) {
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *s_gt = smem;
    unsigned *s_win = smem + p.gt_words_max;
    unsigned *s_near = s_win + p.win_words_max;
    __shared__ EnvShared sh;
    __shared__ long long r_dh[32];
    __shared__ int r_rc[32], r_gc[32];
    __shared__ float r_dm[32], r_dt[32];
    __shared__ int s_next;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const bool debug = (p.flags & ASLAM_FLAG_DEBUG) != 0;

    if (tid == 0) s_next = grab_item(p);
    for (;;) {
        __syncthreads();                 // previous env finished, s_next visible
        const int item = s_next;
        __syncthreads();                 // everyone read s_next before it is replaced
        if (item >= p.E) {
            // Every CTA grabs exactly one out-of-range item before leaving;
            // the last CTA to leave re-arms the queue for the next launch.
            if (tid == 0) {
                __threadfence();
                if (atomicAdd(p.queue + 1, 1u) == gridDim.x - 1) {
                    p.queue[0] = 0u;
                    p.queue[1] = 0u;
                    __threadfence();
                }
            }
            break;
        }
        if (tid == 0) {
            env_prologue(p, p.order[item], sh);
            s_next = grab_item(p);   // one item ahead: its data streams into L2 meanwhile
        }
        __syncthreads();

        // ---- B: reset, stage ground truth, clear counters --------------------
        const int e = sh.e, W = sh.W, H = sh.H;
        const long long ncell = (long long)W * H;
        const int nch = (int)((ncell + 7) >> 3);
        if (sh.reset) {
            int4 *bz = reinterpret_cast<int4 *>(p.belief + sh.map_off);
            for (int q = tid; q < nch; q += nt) bz[q] = make_int4(0, 0, 0, 0);
            const long long vo = p.visit_off[e], vn = p.visit_off[e + 1] - vo;
            for (long long q = tid; q < vn; q += nt) p.visit[vo + q] = -1;
        }
        {
            const int words = (int)((ncell + 31) >> 5);
            const uint4 *src = reinterpret_cast<const uint4 *>(p.gt_bits + sh.gtb_off);
            uint4 *dst = reinterpret_cast<uint4 *>(s_gt);
            for (int q = tid; q < (words + 3) >> 2; q += nt) dst[q] = __ldg(&src[q]);
            const int cw = sh.partial ? (sh.SW * sh.SH + 3) >> 2 : (int)((ncell + 3) >> 2);
            uint4 *wz = reinterpret_cast<uint4 *>(s_win);
            for (int q = tid; q < (cw + 3) >> 2; q += nt) wz[q] = make_uint4(0, 0, 0, 0);
            for (int q = tid; q < sh.NB * sh.NB; q += nt) s_near[q] = 0u;
            if (debug) {
                for (long long q = tid; q < ncell; q += nt) p.dbg_counts[sh.map_off + q] = 0u;
            }
        }
        __syncthreads();

        // ---- C: beams --------------------------------------------------------
        int rc = 0, gc = 0;
        float dmin_m = p.r_max, dmin_t = p.r_max;
        if (sh.partial) {
            for (int b = tid; b < sh.B; b += nt)
                trace_beam<true>(p, sh, b, s_gt, s_win, s_near, rc, gc, dmin_m, dmin_t);
        } else {
            for (int b = tid; b < sh.B; b += nt)
                trace_beam<false>(p, sh, b, s_gt, s_win, s_near, rc, gc, dmin_m, dmin_t);
        }
        __syncthreads();

        // ---- D: apply counters to the log-odds -------------------------------
        long long dh = 0;
        short *Lenv = p.belief + sh.map_off;
        unsigned *dbg = debug ? p.dbg_counts + sh.map_off : nullptr;
        {
            // 8-cell chunks of the shared window: the loads of kUnroll chunks
            // are issued before any of them is used.
            const int SW = sh.SW, rch = (SW + 7) >> 3;
            const int nchunk = sh.partial ? sh.SH * rch : nch;
            const uint2 *cw2 = reinterpret_cast<const uint2 *>(s_win);
            for (int q0 = tid; q0 < nchunk; q0 += nt * kUnroll) {
                uint2 cw[kUnroll];
                int4 lv[kUnroll];
                long long gk[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int q = q0 + u * nt;
                    cw[u] = make_uint2(0u, 0u);
                    gk[u] = -1;
                    if (q < nchunk) {
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
                        cw[u] = cw2[sidx];
                        if (cw[u].x | cw[u].y) {
                            gk[u] = k;
                            lv[u] = *reinterpret_cast<const int4 *>(Lenv + k);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if (gk[u] >= 0) {
                        dh += apply8(p, cw[u], lv[u], dbg ? dbg + gk[u] : nullptr);
                        *reinterpret_cast<int4 *>(Lenv + gk[u]) = lv[u];
                    }
                }
            }
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
                    dh += apply8_wide(p, c0, c1, lv, dbg ? dbg + k : nullptr);
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
                if (c) dh += apply_cell(p, Lenv[k], c >> 16, c & 0xffffu);
                if (dbg) dbg[k] = c;
            }
        }

        // ---- E: reductions, reward, observation ------------------------------
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            dh += __shfl_down_sync(0xffffffffu, dh, o);
            rc += __shfl_down_sync(0xffffffffu, rc, o);
            gc += __shfl_down_sync(0xffffffffu, gc, o);
            dmin_m = fminf(dmin_m, __shfl_down_sync(0xffffffffu, dmin_m, o));
            dmin_t = fminf(dmin_t, __shfl_down_sync(0xffffffffu, dmin_t, o));
        }
        if (lane == 0) {
            r_dh[warp] = dh;
            r_rc[warp] = rc;
            r_gc[warp] = gc;
            r_dm[warp] = dmin_m;
            r_dt[warp] = dmin_t;
        }
        __syncthreads();
        if (tid == 0) {
            EnvTotals r;
            r.dHq = 0;
            r.ray_cells = 0;
            r.gt_cells = 0;
            r.dmin_meas = p.r_max;
            r.dmin_true = p.r_max;
            for (int w = 0; w < nwarps; ++w) {
                r.dHq += r_dh[w];
                r.ray_cells += r_rc[w];
                r.gt_cells += r_gc[w];
                r.dmin_meas = fminf(r.dmin_meas, r_dm[w]);
                r.dmin_true = fminf(r.dmin_true, r_dt[w]);
            }
            finish_env(p, e, W, H, sh.start, sh.col_cell, r);
        }
        if (p.out_obs) {
            float *o = p.out_obs + (long long)e * (p.b_max + 2);
            for (int b = sh.B + tid; b < p.b_max; b += nt) o[b] = p.r_max;
        }
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

cudaError_t step2d_set_smem(size_t smem) {
    return cudaFuncSetAttribute(step2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

cudaError_t step2d_occupancy(int block, size_t smem, int *ctas_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, step2d_kernel, block, smem);
}

cudaError_t launch_step2d(const Step2DParams &p, int grid, int block, size_t smem,
                          cudaStream_t s) {
    step2d_kernel<<<grid, block, smem, s>>>(p);
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
