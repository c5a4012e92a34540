// step3d.cu -- the batched 3-D (voxel) environment step on sm_103a.
//
// Same step as the 2-D kernel (action integration, sensing, noise, per-scan
// sum-then-clamp log-odds update, entropy gain, Eq. 7-17 reward, Eq. 3
// observation), for a multi-ring LiDAR at sensor height z_s in a W x H x D
// voxel world.  One persistent CTA per environment:
//   * the env's ground truth (1 bit per voxel, 64 KiB for 128x128x32) is
//     staged in shared memory;
//   * warps take groups of 32 adjacent azimuths of one ring from a block-
//     wide counter, long rings first; one thread per beam walks the voxels
//     with an exact fixed-point 3-D traversal: three error terms e_xy, e_xz, e_yz compare the next face
//     crossings of each axis pair; ties go Z first, then Y, then X.  Every
//     step adds a multiple of 2^16 to them, so the walk carries
//     floor(e / 2^16) (same sign; a term is ax ay (t_x - t_y) scaled, both
//     next crossings within one interval, so it stays in [-2^30, 2^30]) and
//     the voxel index in 32 bits (the ground truth fits shared memory);
//   * counts: voxels within Chebyshev distance R - 1 of the sensor's voxel
//     (R from the ring and azimuth spacing, computed on the host: beyond it
//     no voxel is crossed by more than 255 beams) go to a 32-bit
//     (hits << 16 | misses) block in shared memory; every other voxel to a
//     global 16-bit (hits:8 | misses:8) counter, two per word, which never
//     carries (half the L2 footprint of 32-bit counters), plus a bitmap of
//     touched 8-voxel chunks.  The belief walk runs warp-synchronously: the 32
//     lanes of a warp are 32 adjacent azimuths of one ring, which cross the
//     same voxels near the sensor, so adjacent lanes in the same voxel are
//     merged into one atomic;
//   * the CTA then applies the touched chunks, then the near block, and sums
//     the entropy change.
#include "aslam_internal.cuh"
#include "env_common.cuh"

namespace aslam {
namespace {

struct Env3 {
    int e, W, H, Dd, B, A, R, NB;   // R: near radius (voxels), NB = 2R - 1
    int Px, Py, ri, rj, rk, col_cell;
    float c, s;
    long long map_off, gtb_off, ray_off, ncell;
    EnvStart start;
};

__device__ __forceinline__ unsigned gt_bit3(const unsigned *bits, long long k) {
    return (bits[k >> 5] >> (k & 31)) & 1u;
}

struct Walk3 {
    int i, j, k;             // voxel
    int flat;
    int exy, exz, eyz;       // floor(e / 2^16) of the axis pairs' crossing comparisons
    int last;                // axis of the last step (0 x, 1 y, 2 z)
};

struct Ray3 {
    int sx, sy, sz;
    long long ax, ay, az;    // |D| per axis (Q30)
    long long nx0, ny0, nz0;
    int stride_y, stride_z;
};

// One traversal step; returns false when it leaves the volume.
__device__ __forceinline__ bool step3(const Ray3 &r, const Env3 &sh, Walk3 &w) {
    int a;
    if (w.exy < 0) a = (w.exz < 0) ? 0 : 2;
    else a = (w.eyz < 0) ? 1 : 2;
    w.last = a;
    if (a == 0) {
        w.i += r.sx;
        w.flat += r.sx;
        w.exy += (int)r.ay;
        w.exz += (int)r.az;
        return (unsigned)w.i < (unsigned)sh.W;
    }
    if (a == 1) {
        w.j += r.sy;
        w.flat += r.sy * r.stride_y;
        w.exy -= (int)r.ax;
        w.eyz += (int)r.az;
        return (unsigned)w.j < (unsigned)sh.H;
    }
    w.k += r.sz;
    w.flat += r.sz * r.stride_z;
    w.exz -= (int)r.ax;
    w.eyz -= (int)r.ay;
    return (unsigned)w.k < (unsigned)sh.Dd;
}

__device__ __forceinline__ long long apply_cell3(const Step2DParams &p, short &L, unsigned h,
                                                 unsigned m) {
    const int l0 = L;
    int l1 = l0 + (int)h * p.hit_q + (int)m * p.miss_q;
    l1 = min(max(l1, -p.clamp_q), p.clamp_q);
    L = (short)l1;
    return __ldg(&p.lut[l1 + p.clamp_q]) - __ldg(&p.lut[l0 + p.clamp_q]);
}

// Range (in voxels) at which a ring's beams leave the slab between the floor
// and the top of the volume, at most r_max.
__device__ __forceinline__ float ring_reach(const Step2DParams &p, int Dd, int ring) {
    const float rmax_v = p.r_max / p.res;
    const float zs = (float)p.Pz * (1.0f / 65536.0f);
    const float se = p.elev_cs[ring].y;
    if (se < 0.0f) return fminf(rmax_v, zs / -se);
    if (se > 0.0f) return fminf(rmax_v, ((float)Dd - zs) / se);
    return rmax_v;
}

__global__ void __launch_bounds__(1024, 1) step3d_kernel(const Step2DParams p) {
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *s_gt = smem;
    unsigned *s_near = smem + ((p.gt_words_max + 3) & ~3);    // [NB^3], zero between envs
    __shared__ Env3 sh;
    __shared__ long long r_dh[32], r_rc[32], r_gc[32];
    __shared__ float r_dm[32], r_dt[32];
    __shared__ int s_next, s_grp;
    __shared__ short s_ring[256];   // rings, longest expected walk first

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const bool debug = (p.flags & ASLAM_FLAG_DEBUG) != 0;

    for (int q = tid; q < p.near_words_max; q += nt) s_near[q] = 0u;
    if (tid == 0) s_next = (int)atomicAdd(p.queue, 1u);
    for (;;) {
        __syncthreads();
        const int item = s_next;
        __syncthreads();
        if (item >= p.E) {
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
            const int e = p.order[item];
            const int W = p.W[e], H = p.H[e], Dd = p.Dd[e];
            sh.e = e;
            sh.W = W;
            sh.H = H;
            sh.Dd = Dd;
            sh.B = p.B[e];
            sh.A = sh.B / p.n_rings;
            sh.R = p.R8[e];
            sh.NB = 2 * sh.R - 1;
            sh.map_off = p.map_off[e];
            sh.gtb_off = p.gtb_off[e];
            sh.ray_off = p.ray_off[e];
            sh.ncell = (long long)W * H * Dd;
            sh.start = begin_env(p, e, sh.ncell);
            sh.Px = q16_of(sh.start.x, p.res);
            sh.Py = q16_of(sh.start.y, p.res);
            sh.ri = sh.Px >> 16;
            sh.rj = sh.Py >> 16;
            sh.rk = p.Pz >> 16;
            const bool inside = (unsigned)sh.ri < (unsigned)W && (unsigned)sh.rj < (unsigned)H &&
                                (unsigned)sh.rk < (unsigned)Dd;
            sh.col_cell = !inside ||
                          gt_bit3(p.gt_bits + sh.gtb_off, ((long long)sh.rk * H + sh.rj) * W + sh.ri);
            det_sincos(sh.start.th, sh.s, sh.c);
            s_grp = 0;
            s_next = (int)atomicAdd(p.queue, 1u);
        }
        __syncthreads();
        const int e = sh.e;
        const long long ncell = sh.ncell;
        // ---- reset, stage ground truth ----------------------------------------
        if (sh.start.reset) {
            int4 *bz = reinterpret_cast<int4 *>(p.belief + sh.map_off);
            for (long long q = tid; q < (ncell + 7) >> 3; q += nt) bz[q] = make_int4(0, 0, 0, 0);
            const long long vo = p.visit_off[e], vn = p.visit_off[e + 1] - vo;
            for (long long q = tid; q < vn; q += nt) p.visit[vo + q] = -1;
        }
        {
            const long long words = (ncell + 31) >> 5;
            const uint4 *src = reinterpret_cast<const uint4 *>(p.gt_bits + sh.gtb_off);
            uint4 *dst = reinterpret_cast<uint4 *>(s_gt);
            for (long long q = tid; q < (words + 3) >> 2; q += nt) dst[q] = __ldg(&src[q]);
            if (debug)
                for (long long q = tid; q < ncell; q += nt) p.dbg_counts[sh.map_off + q] = 0u;
        }
        // Rings in decreasing order of the range at which they leave the
        // slab between the floor and the top of the volume (r_max at most):
        // the warps take the long rings first, so that the groups still in
        // flight when the work runs out are short ones.  The order only
        // schedules; every count is an integer sum.
        for (int r = tid; r < p.n_rings; r += nt) {
            const float key = ring_reach(p, sh.Dd, r);
            int rank = 0;
            for (int q = 0; q < p.n_rings; ++q) {
                const float kq = ring_reach(p, sh.Dd, q);
                rank += kq > key || (kq == key && q < r);
            }
            s_ring[rank] = (short)r;
        }
        __syncthreads();

        // ---- beams -------------------------------------------------------------
        long long rc = 0, gc = 0;
        float dmin_m = p.r_max, dmin_t = p.r_max;
        const int W = sh.W, H = sh.H;
        // Work is taken a group of 32 adjacent azimuths of one ring at a time,
        // from a block-wide counter: whole warps, as the warp-synchronous
        // belief walk below needs, and balanced across the warps before the
        // CTA's barrier however the walk lengths vary.
        const int A = sh.A, gpr = (A + 31) >> 5, ngroups = p.n_rings * gpr;
        for (;;) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&s_grp, 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= ngroups) break;
            const int ring = s_ring[g / gpr];
            const int a = (g % gpr) * 32 + lane;
            const bool valid = a < A;
            const int b = ring * A + a;
            Ray3 r;
            Walk3 w0;
            bool hit = false, in0 = false;
            float z_true = p.r_max, z = p.r_max;
            int Ku = -1;
            if (valid) {
                const float2 cs = p.beam_cs[sh.ray_off + b];
                const float2 el = p.elev_cs[ring];
                const float hx = fsub(fmul(sh.c, cs.x), fmul(sh.s, cs.y));
                const float hy = fadd(fmul(sh.s, cs.x), fmul(sh.c, cs.y));
                const int Dx = __float2int_rn(fmul(fmul(el.x, hx), 1073741824.0f));
                const int Dy = __float2int_rn(fmul(fmul(el.x, hy), 1073741824.0f));
                const int Dz = __float2int_rn(fmul(el.y, 1073741824.0f));
                const int i0 = sh.ri, j0 = sh.rj, k0 = sh.rk;
                in0 = (unsigned)i0 < (unsigned)W && (unsigned)j0 < (unsigned)H &&
                      (unsigned)k0 < (unsigned)sh.Dd;
                r.sx = (Dx > 0) - (Dx < 0);
                r.sy = (Dy > 0) - (Dy < 0);
                r.sz = (Dz > 0) - (Dz < 0);
                r.ax = Dx < 0 ? -(long long)Dx : Dx;
                r.ay = Dy < 0 ? -(long long)Dy : Dy;
                r.az = Dz < 0 ? -(long long)Dz : Dz;
                r.nx0 = Dx > 0 ? ((long long)(i0 + 1) << 16) - sh.Px
                               : (Dx < 0 ? (long long)sh.Px - ((long long)i0 << 16) : 65536);
                r.ny0 = Dy > 0 ? ((long long)(j0 + 1) << 16) - sh.Py
                               : (Dy < 0 ? (long long)sh.Py - ((long long)j0 << 16) : 65536);
                r.nz0 = Dz > 0 ? ((long long)(k0 + 1) << 16) - p.Pz
                               : (Dz < 0 ? (long long)p.Pz - ((long long)k0 << 16) : 65536);
                r.stride_y = W;
                r.stride_z = W * H;
                w0.i = i0;
                w0.j = j0;
                w0.k = k0;
                w0.flat = (k0 * H + j0) * W + i0;
                w0.exy = (int)((r.nx0 * r.ay - r.ny0 * r.ax) >> 16);
                w0.exz = (int)((r.nx0 * r.az - r.nz0 * r.ax) >> 16);
                w0.eyz = (int)((r.ny0 * r.az - r.nz0 * r.ay) >> 16);
                w0.last = -1;
                if (in0) {
                    // ground truth up to the first occupied voxel
                    Walk3 w = w0;
                    int cells = 1;
                    if (gt_bit3(s_gt, w.flat)) {
                        hit = true;
                        z_true = 0.0f;
                    } else {
                        const int Ks = crossings_le(r.nx0, r.ax, p.Tmax) +
                                       crossings_le(r.ny0, r.ay, p.Tmax) +
                                       crossings_le(r.nz0, r.az, p.Tmax);
                        for (int s = 0; s < Ks; ++s) {
                            if (!step3(r, sh, w)) break;
                            ++cells;
                            if (gt_bit3(s_gt, w.flat)) {
                                hit = true;
                                break;
                            }
                        }
                        if (hit) {
                            long long n, ad;
                            if (w.last == 0) { n = r.nx0 + ((long long)(abs(w.i - i0) - 1) << 16); ad = r.ax; }
                            else if (w.last == 1) { n = r.ny0 + ((long long)(abs(w.j - j0) - 1) << 16); ad = r.ay; }
                            else { n = r.nz0 + ((long long)(abs(w.k - k0) - 1) << 16); ad = r.az; }
                            z_true = fmul(fmul(fdiv(__int2float_rn((int)n), __int2float_rn((int)ad)), 16384.0f), p.res);
                        }
                    }
                    gc += cells;
                    z = z_true;
                    if (hit) {
                        const float g = det_gauss(p.key, (unsigned)(p.env_base + e), (unsigned)sh.start.gstep, (unsigned)b);
                        z = measured_range(z_true, g, p.sigma, p.r_min, p.r_max, p.dec_scale);
                    }
                    const int Tz = hit ? q16_of(z, p.res) : p.Tmax;
                    Ku = crossings_le(r.nx0, r.ax, Tz) + crossings_le(r.ny0, r.ay, Tz) +
                         crossings_le(r.nz0, r.az, Tz);
                }
                const long long ro = sh.ray_off + b;
                p.z[ro] = z;
                if (debug) {
                    p.z_true[ro] = z_true;
                    p.hit[ro] = hit ? 1 : 0;
                }
                if (p.out_obs) p.out_obs[(long long)e * (p.b_max + 2) + b] = z;
                dmin_m = fminf(dmin_m, z);
                dmin_t = fminf(dmin_t, z_true);
            }
            // belief walk, warp-synchronous: lanes in the same voxel share one
            // atomic.  The touched-chunk bit is set only by a leader that has
            // just entered its 8-voxel chunk: the chunk of its previous voxel
            // was marked by the leader that counted that voxel one step
            // earlier (a walk's first voxel always marks, and so does the
            // first far voxel after a near one: near voxels mark nothing).
            bool active = valid && in0;
            Walk3 w = w0;
            int s = 0, prev_chunk = -1;
            for (;;) {
                const unsigned act = __ballot_sync(0xffffffffu, active);
                if (!act) break;
                // adjacent lanes (adjacent azimuths) in the same voxel form a
                // run; the run's first lane adds the whole run in one atomic
                const int vox = active ? w.flat : -1 - lane;          // inactive: unique
                const int pvox = __shfl_up_sync(0xffffffffu, vox, 1);
                const bool start = active && (lane == 0 || pvox != vox);
                const unsigned starts = __ballot_sync(0xffffffffu, start);
                const bool last = active && s == Ku;
                const unsigned hits = __ballot_sync(0xffffffffu, last && hit);
                if (active) {
                    const int chunk = w.flat >> 3;
                    const int ni = w.i - sh.ri + sh.R - 1, nj = w.j - sh.rj + sh.R - 1,
                              nk = w.k - sh.rk + sh.R - 1;
                    const bool near = (unsigned)ni < (unsigned)sh.NB &&
                                      (unsigned)nj < (unsigned)sh.NB && (unsigned)nk < (unsigned)sh.NB;
                    if (start) {
                        // the run: this lane up to the next start or inactive lane
                        const unsigned above = lane == 31 ? 0u : ~((2u << lane) - 1u);
                        const unsigned stop = (starts | ~act) & above;
                        const unsigned upto = stop ? (stop & (0u - stop)) - 1u : 0xffffffffu;
                        const unsigned run = upto & ~((1u << lane) - 1u);
                        const unsigned nh = __popc(hits & run), nm = __popc(run) - nh;
                        if (near) {
                            atomicAdd(&s_near[(nk * sh.NB + nj) * sh.NB + ni], (nh << 16) | nm);
                        } else {
                            // 16-bit field (hits:8 | misses:8) of the voxel; map_off is even
                            const long long v = sh.map_off + w.flat;
                            red_add(&p.far_cnt[v >> 1], ((nh << 8) | nm) << ((v & 1) << 4));
                            if (chunk != prev_chunk)
                                red_or(&p.far_bits[v >> 8], 1u << (chunk & 31));
                        }
                    }
                    // a near voxel marks nothing: the next far voxel of its chunk must
                    prev_chunk = near ? -1 : chunk;
                    ++rc;
                    ++s;
                    if (last) active = false;
                    else if (!step3(r, sh, w)) active = false;
                }
                // Merging pays while adjacent lanes share voxels (near the
                // sensor); once the runs are most of the active lanes the warp
                // stops merging, and every lane walks on alone.  The decision
                // is uniform (it reads ballots only).
                if (4 * __popc(starts) >= 3 * __popc(act)) break;
            }
            // each lane alone: one reduction per voxel; the chunk of a lane's
            // previous voxel is marked (by its run's leader, or by this lane)
            while (active) {
                const bool last = s == Ku;
                const int chunk = w.flat >> 3;
                const int ni = w.i - sh.ri + sh.R - 1, nj = w.j - sh.rj + sh.R - 1,
                          nk = w.k - sh.rk + sh.R - 1;
                const bool near = (unsigned)ni < (unsigned)sh.NB &&
                                  (unsigned)nj < (unsigned)sh.NB && (unsigned)nk < (unsigned)sh.NB;
                const unsigned nh = last && hit ? 1u : 0u, nm = 1u - nh;
                if (near) {
                    atomicAdd(&s_near[(nk * sh.NB + nj) * sh.NB + ni], (nh << 16) | nm);
                } else {
                    const long long v = sh.map_off + w.flat;
                    red_add(&p.far_cnt[v >> 1], ((nh << 8) | nm) << ((v & 1) << 4));
                    if (chunk != prev_chunk) red_or(&p.far_bits[v >> 8], 1u << (chunk & 31));
                }
                prev_chunk = near ? -1 : chunk;
                ++rc;
                ++s;
                if (last || !step3(r, sh, w)) active = false;
            }
        }
        __syncthreads();

        // ---- apply the touched chunks ------------------------------------------
        long long dh = 0;
        {
            short *Lenv = p.belief + sh.map_off;
            unsigned *dbg = debug ? p.dbg_counts + sh.map_off : nullptr;
            const long long nbw = (ncell + 255) >> 8;
            unsigned *bits = p.far_bits + (sh.map_off >> 8);
            for (long long wq = tid; wq < nbw; wq += nt) {
                unsigned m = __ldcg(&bits[wq]);
                if (!m) continue;
                bits[wq] = 0u;
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    const long long k = wq * 256 + bit * 8;
                    // eight 16-bit counters: 16 bytes, aligned (map_off and k are
                    // multiples of 8)
                    uint4 *cp = reinterpret_cast<uint4 *>(p.far_cnt + ((sh.map_off + k) >> 1));
                    const uint4 cw = __ldcg(cp);
                    *cp = make_uint4(0u, 0u, 0u, 0u);
                    int4 lv = *reinterpret_cast<const int4 *>(Lenv + k);
                    short *L = reinterpret_cast<short *>(&lv);
                    const unsigned c4[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const unsigned c = (c4[q >> 1] >> ((q & 1) << 4)) & 0xffffu;
                        if (c) dh += apply_cell3(p, L[q], c >> 8, c & 0xffu);
                        if (dbg) dbg[k + q] = ((c >> 8) << 16) | (c & 0xffu);
                    }
                    *reinterpret_cast<int4 *>(Lenv + k) = lv;
                }
            }
        }
        // the near block, after every far chunk (a chunk may hold voxels of both)
        __syncthreads();
        {
            short *Lenv = p.belief + sh.map_off;
            unsigned *dbg = debug ? p.dbg_counts + sh.map_off : nullptr;
            const int nb = sh.NB, nb3 = nb * nb * nb;
            for (int q = tid; q < nb3; q += nt) {
                const unsigned c = s_near[q];
                if (!c) continue;
                s_near[q] = 0u;
                const int ni = q % nb, nj = (q / nb) % nb, nk = q / (nb * nb);
                const int i = sh.ri + ni - (sh.R - 1), j = sh.rj + nj - (sh.R - 1),
                          k = sh.rk + nk - (sh.R - 1);
                // counted voxels lie in the volume
                const long long v = ((long long)k * H + j) * W + i;
                dh += apply_cell3(p, Lenv[v], c >> 16, c & 0xffffu);
                if (dbg) dbg[v] = c;
            }
        }

        // ---- reductions, reward, observation ----------------------------------
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
            EnvTotals t;
            t.dHq = 0;
            t.ray_cells = 0;
            t.gt_cells = 0;
            t.dmin_meas = p.r_max;
            t.dmin_true = p.r_max;
            for (int q = 0; q < nwarps; ++q) {
                t.dHq += r_dh[q];
                t.ray_cells += r_rc[q];
                t.gt_cells += r_gc[q];
                t.dmin_meas = fminf(t.dmin_meas, r_dm[q]);
                t.dmin_true = fminf(t.dmin_true, r_dt[q]);
            }
            finish_env(p, e, W, H, sh.start, sh.col_cell, t, false);
        }
        if (p.out_obs) {
            float *o = p.out_obs + (long long)e * (p.b_max + 2);
            for (int b = sh.B + tid; b < p.b_max; b += nt) o[b] = p.r_max;
        }
    }
}

}  // namespace

size_t step3d_static_smem() {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, step3d_kernel) == cudaSuccess ? a.sharedSizeBytes
                                                                    : (size_t)16384;
}

cudaError_t step3d_set_smem(size_t smem) {
    return cudaFuncSetAttribute(step3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

cudaError_t step3d_occupancy(int block, size_t smem, int *ctas_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, step3d_kernel, block, smem);
}

cudaError_t launch_step3d(const Step2DParams &p, int grid, int block, size_t smem,
                          cudaStream_t s, const cudaEvent_t *ev) {
    cudaError_t e = ev ? cudaEventRecord(ev[0], s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    step3d_kernel<<<grid, block, smem, s>>>(p);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    return e;
}

}  // namespace aslam
