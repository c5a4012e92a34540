// csm2d.cu -- batched correlative scan matching against each env's log-odds
// grid (Sec. III-D: a discretised (dx, dy, dth) neighbourhood of the
// predicted pose is scored against the occupancy grid; the best candidate
// is an absolute pose measurement whose information is scaled by the
// normalised score and the ambiguity margin to the second-best candidate).
//
// Score of candidate (i, j, k), i, j in [-n_xy, n_xy] cells, k in
// [-n_th, n_th] rotation steps: for every returned beam b (z_b < r_max),
// rotate its direction by th_k = th + k*dth, take the endpoint
// (x + z_b cos, y + z_b sin), its cell (floor of metres / res) shifted by
// (i, j), and add the occupancy evidence min(255, max(L, 0) >> 4) of that
// cell (0 outside the map).  All integer, so the scores, the argmax (ties:
// lowest (k, j, i) index) and the second best (best score among candidates
// more than `sep` steps away in some coordinate) are exact.
//
// One CTA per env.  The returned beams are compacted once, then the
// rotations are processed one at a time: the endpoint cells of the returned
// beams for th_k go to shared memory (one thread per beam), each thread sums
// one candidate over a slice of the beams, and the slices are added in a
// fixed order into a shared score table.
//
// When it fits, the env's evidence map (one byte per cell) is staged in
// shared memory inside a zero border of 2 n_xy cells, followed by 2 n_xy + 1
// zero rows (the sentinel block).  An endpoint cell more than n_xy cells
// outside the map scores 0 for every candidate and is pointed at the centre
// of the sentinel block; any other endpoint's candidate cells all lie in the
// bordered map.  So the per-rotation staging stores one shared address per
// beam, and each thread sums four horizontally adjacent candidates at once:
// two aligned words hold their four evidence bytes (a funnel shift by the
// address's byte offset), added as two pairs of 16-bit lanes (a thread adds
// at most ceil(1024 / 6) beams of <= 255, so a lane never carries).  The
// row stride is chosen on the host so that the words one warp reads fall in
// as few shared-memory banks per bank as it can.
#include <cmath>

#include "aslam_internal.cuh"

namespace aslam {
namespace {

constexpr int kCsmMaxN = 8;                      // |i|, |j|, |k| <= 8
constexpr int kCsmMaxCand = (2 * kCsmMaxN + 1) * (2 * kCsmMaxN + 1);
constexpr int kCsmMaxRot = 2 * kCsmMaxN + 1;
constexpr int kCsmBlock = 512;

struct CsmArgs {
    int n_xy, n_th, sep;
    float dth;
    size_t map_bytes;            // shared bytes for the staged evidence map (0: read global)
    int ws;                      // row stride of the staged map, bytes (a multiple of 4)
    bool reset_empty;            // in the step: an env resetting now has an empty map
    const float *pose_pred;      // [E, 3]
    const float *ranges;         // [sum B]
    float *pose_out;             // [E, 3]
    float *match;                // [E, 3] score_norm, margin, w
    long long *scores;           // [E, 3] best, second, best index
};

__device__ __forceinline__ unsigned evidence(short L) {
    const int v = L > 0 ? (int)L >> 4 : 0;
    return (unsigned)(v < 255 ? v : 255);
}

// evidence bytes of the two int16 cells in w, low cell in the low byte
__device__ __forceinline__ unsigned evidence2(unsigned w) {
    return evidence((short)(w & 0xffffu)) | evidence((short)(w >> 16)) << 8;
}

// column of map cell 0 in the staged rows: the 2n-cell border rounded up to
// a word, so that groups of 8 cells are stored as two aligned words
__host__ __device__ __forceinline__ int csm_col0(int n) { return (2 * n + 3) & ~3; }

__global__ void __launch_bounds__(kCsmBlock) csm2d_kernel(const Step2DParams p, const CsmArgs a) {
    extern __shared__ __align__(16) unsigned char s_map[];
    __shared__ int2 s_cell[ASLAM_MAX_BEAMS];     // staged map: .x is the shared address
    __shared__ int s_ret[ASLAM_MAX_BEAMS];       // returned beams, in beam order
    __shared__ float2 s_rot[kCsmMaxRot];         // (sin, cos) of each rotation
    __shared__ int s_wcnt[kCsmBlock / 32];
    __shared__ int s_score[kCsmMaxRot * kCsmMaxCand];
    __shared__ int s_part[kCsmBlock];
    __shared__ int s_nret;
    __shared__ unsigned long long s_red[kCsmBlock / 32];
    const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int W = p.W[e], H = p.H[e], B = p.B[e];
    const short *L = p.belief + p.map_off[e];
    const bool staged = a.map_bytes > 0;
    // inside the step the map of an env that resets now is cleared only by
    // the update kernel: it is empty for the match (no evidence anywhere)
    const bool empty = a.reset_empty && p.done[e] != 0;
    const int ws = a.ws, brd = 2 * a.n_xy, col0 = csm_col0(a.n_xy);
    if (staged) {
        uint4 *z4 = reinterpret_cast<uint4 *>(s_map);
        for (int q = tid; q < (int)(a.map_bytes >> 4); q += nt) z4[q] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        unsigned char *m0 = s_map + brd * ws + col0;
        if (!empty && (W & 7) == 0) {
            // rows of whole 8-cell groups; env grids start on 512-byte
            // boundaries, so each group is one aligned 16-byte load.  Four
            // loads per thread are in flight before their stores.
            const uint4 *L8 = reinterpret_cast<const uint4 *>(L);
            const int wv = W >> 3, nv = wv * H;
            for (int v0 = tid; v0 < nv; v0 += 4 * nt) {
                uint4 r[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (v0 + u * nt < nv) r[u] = __ldg(&L8[v0 + u * nt]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int v = v0 + u * nt;
                    if (v < nv) {
                        const int jj = v / wv, ii = v - jj * wv;
                        unsigned *d = reinterpret_cast<unsigned *>(m0 + jj * ws + 8 * ii);
                        d[0] = evidence2(r[u].x) | evidence2(r[u].y) << 16;
                        d[1] = evidence2(r[u].z) | evidence2(r[u].w) << 16;
                    }
                }
            }
        } else if (!empty) {
            // (row, column) of element q tracked incrementally (no division per cell)
            int ii = tid % W, jj = tid / W;
            const int di = nt % W, dj = nt / W;
            for (int q = tid; q < W * H; q += nt) {
                m0[jj * ws + ii] = (unsigned char)evidence(L[q]);
                ii += di;
                jj += dj;
                if (ii >= W) {
                    ii -= W;
                    ++jj;
                }
            }
        }
    }
    const float x = a.pose_pred[3 * e], y = a.pose_pred[3 * e + 1], th = a.pose_pred[3 * e + 2];
    const float *z = a.ranges + p.ray_off[e];
    const float2 *bcs = p.beam_cs + p.ray_off[e];
    const int side = 2 * a.n_xy + 1, NC = side * side, NK = 2 * a.n_th + 1;
    const int nslice = nt / NC;                  // beam slices per candidate
    const int c = tid % NC, sl = tid / NC;
    const int ci_off = c % side - a.n_xy, cj_off = c / side - a.n_xy;
    // staged map: thread (slice sl4, row cj4, group gi4) sums candidates
    // i = 4 gi4 .. 4 gi4 + 3 (those < side) of row cj4
    const int G4 = (side + 3) >> 2, NG = side * G4, nslice4 = nt / NG;
    const int sl4 = tid / NG, g4 = tid % NG, cj4 = g4 / G4, gi4 = g4 % G4;
    const int c_off4 = (cj4 - a.n_xy) * ws + 4 * gi4 - a.n_xy;
    // centre of the zero sentinel block below the bordered map
    const int sentinel = (H + 2 * brd + a.n_xy) * ws + a.n_xy;
    // the returned beams (range < r_max), compacted in beam order once
    const int lane = tid & 31, warp = tid >> 5;
    int nret = 0;
    for (int b0 = 0; b0 < B; b0 += nt) {
        const int b = b0 + tid;
        const bool ret = b < B && z[b] < p.r_max;
        const unsigned m = __ballot_sync(0xffffffffu, ret);
        if (lane == 0) s_wcnt[warp] = __popc(m);
        __syncthreads();
        int off = nret, round = 0;
        for (int w = 0; w < nt / 32; ++w) {
            if (w < warp) off += s_wcnt[w];
            round += s_wcnt[w];
        }
        if (ret) s_ret[off + __popc(m & ((1u << lane) - 1u))] = b;
        __syncthreads();
        nret += round;
    }
    if (tid == 0) s_nret = nret;
    if (tid < NK) {
        float sk, ck;
        det_sincos(fadd(th, fmul((float)(tid - a.n_th), a.dth)), sk, ck);
        s_rot[tid] = make_float2(sk, ck);
    }
    for (int k = 0; k < NK; ++k) {
        // endpoint cells of the returned beams for th_k
        __syncthreads();
        const float sk = s_rot[k].x, ck = s_rot[k].y;
        for (int q = tid; q < nret; q += nt) {
            const int b = s_ret[q];
            const float2 bc = bcs[b];
            const float cx = fsub(fmul(ck, bc.x), fmul(sk, bc.y));
            const float cy = fadd(fmul(sk, bc.x), fmul(ck, bc.y));
            const float ex = fadd(x, fmul(z[b], cx)), ey = fadd(y, fmul(z[b], cy));
            const int i = (int)floorf(fdiv(ex, p.res)), j = (int)floorf(fdiv(ey, p.res));
            if (staged) {
                const bool near = i >= -a.n_xy && i < W + a.n_xy && j >= -a.n_xy && j < H + a.n_xy;
                s_cell[q].x = near ? (j + brd) * ws + (i + col0) : sentinel;
            } else {
                s_cell[q] = make_int2(i, j);
            }
        }
        __syncthreads();
        if (staged) {
            unsigned lo = 0u, hi = 0u;          // candidates (0, 2) and (1, 3) of the group
            if (sl4 < nslice4) {
                const unsigned *words = reinterpret_cast<const unsigned *>(s_map);
                const int *addr = reinterpret_cast<const int *>(s_cell);
                for (int q = sl4; q < nret; q += nslice4) {
                    const int ad = addr[2 * q] + c_off4;
                    const unsigned v = __funnelshift_r(words[ad >> 2], words[(ad >> 2) + 1],
                                                       (unsigned)(ad & 3) << 3);
                    lo += v & 0x00ff00ffu;
                    hi += (v >> 8) & 0x00ff00ffu;
                }
            }
            __syncthreads();                      // every address is read: s_cell is free
            int *part = reinterpret_cast<int *>(s_cell);          // [nslice4][NC]
            if (sl4 < nslice4) {
                const int sums[4] = {(int)(lo & 0xffffu), (int)(hi & 0xffffu), (int)(lo >> 16),
                                     (int)(hi >> 16)};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (4 * gi4 + u < side) part[sl4 * NC + cj4 * side + 4 * gi4 + u] = sums[u];
            }
            __syncthreads();
            if (tid < NC) {
                int sum = 0;
                for (int q = 0; q < nslice4; ++q) sum += part[q * NC + tid];
                s_score[k * NC + tid] = sum;
            }
        } else {
            int acc = 0;
            if (sl < nslice) {
                for (int q = sl; q < nret; q += nslice) {
                    const int2 cc = s_cell[q];
                    const int i = cc.x + ci_off, j = cc.y + cj_off;
                    if ((unsigned)i < (unsigned)W && (unsigned)j < (unsigned)H && !empty)
                        acc += (int)evidence(L[(long long)j * W + i]);
                }
                s_part[tid] = acc;
            }
            __syncthreads();
            if (tid < NC) {
                int sum = 0;
                for (int q = 0; q < nslice; ++q) sum += s_part[q * NC + tid];
                s_score[k * NC + tid] = sum;
            }
        }
    }
    __syncthreads();
    // best: max score, ties to the lowest index (key = score << 32 | ~index)
    const int NT = NK * NC;
    auto block_max = [&](unsigned long long v) {
        for (int o = 16; o; o >>= 1) {
            const unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if ((tid & 31) == 0) s_red[tid >> 5] = v;
        __syncthreads();
        unsigned long long r = 0;
        for (int w = 0; w < nt / 32; ++w) r = s_red[w] > r ? s_red[w] : r;
        __syncthreads();
        return r;
    };
    unsigned long long best = 0;
    for (int q = tid; q < NT; q += nt) {
        const unsigned long long key = ((unsigned long long)(unsigned)s_score[q] << 32) |
                                       (unsigned long long)(0xffffffffu - (unsigned)q);
        best = key > best ? key : best;
    }
    best = block_max(best);
    const int qb = (int)(0xffffffffu - (unsigned)(best & 0xffffffffu));
    const long long sb = (long long)(best >> 32);
    const int ib = qb % side, jb = (qb / side) % side, kb = qb / NC;
    unsigned long long second = 0;
    for (int q = tid; q < NT; q += nt) {
        const int i = q % side, j = (q / side) % side, k = q / NC;
        const int d = max(max(abs(i - ib), abs(j - jb)), abs(k - kb));
        if (d > a.sep) {
            const unsigned long long v = (unsigned)s_score[q];
            second = v > second ? v : second;
        }
    }
    second = block_max(second);
    if (tid == 0) {
        const long long s2 = (long long)second;
        const int nret = s_nret;
        const double norm = nret > 0 ? (double)sb / (255.0 * (double)nret) : 0.0;
        const double margin = sb > 0 ? (double)(sb - s2) / (double)sb : 0.0;
        a.match[3 * e] = (float)norm;
        a.match[3 * e + 1] = (float)margin;
        a.match[3 * e + 2] = (float)(norm * margin);
        a.scores[3 * e] = sb;
        a.scores[3 * e + 1] = s2;
        a.scores[3 * e + 2] = qb;
        const float pi_f = (float)3.14159265358979323846;
        const float two_pi_f = (float)(2.0 * 3.14159265358979323846);
        float tho = fadd(th, fmul((float)(kb - a.n_th), a.dth));
        if (tho >= pi_f) tho = fsub(tho, two_pi_f);
        if (tho < -pi_f) tho = fadd(tho, two_pi_f);
        a.pose_out[3 * e] = fadd(x, fmul((float)(ib - a.n_xy), p.res));
        a.pose_out[3 * e + 1] = fadd(y, fmul((float)(jb - a.n_xy), p.res));
        a.pose_out[3 * e + 2] = tho;
    }
}

}  // namespace

int csm_max_n() { return kCsmMaxN; }

namespace {

// Shared-memory wavefronts of the worst warp for row stride ws (bytes): the
// lanes of one slice read the same beam, so with row stride ws / 4 words,
// lane (cj, gi) reads word w0 + cj ws / 4 + gi (and the word after it);
// lanes of different slices read other beams and are not counted.
int csm_stride_cost(int ws, int n) {
    const int side = 2 * n + 1, G4 = (side + 3) / 4, NG = side * G4, nslice = kCsmBlock / NG;
    const int wsw = ws / 4;
    int worst = 1;
    for (int w0 = 0; w0 < kCsmBlock; w0 += 32) {
        for (int sl = 0; sl < nslice; ++sl) {
            int words[32], nw = 0;
            for (int t = w0; t < w0 + 32; ++t) {
                if (t / NG != sl) continue;
                const int g = t % NG;
                words[nw++] = (g / G4) * wsw + g % G4;
            }
            for (int bank = 0; bank < 32; ++bank) {
                int distinct = 0;
                for (int u = 0; u < nw; ++u) {
                    if ((words[u] & 31) != bank) continue;
                    bool seen = false;
                    for (int v = 0; v < u; ++v) seen = seen || words[v] == words[u];
                    distinct += !seen;
                }
                worst = distinct > worst ? distinct : worst;
            }
        }
    }
    return worst;
}

}  // namespace

size_t csm_map_layout(const int *W, const int *H, int E, int n, int *ws) {
    int wmax = 0, hmax = 0;
    for (int e = 0; e < E; ++e) {
        wmax = W[e] > wmax ? W[e] : wmax;
        hmax = H[e] > hmax ? H[e] : hmax;
    }
    // bordered width in words; of the next 8 strides (a wider pad costs
    // occupancy), the first with the fewest bank conflicts across a warp's
    // candidate words
    const int w0 = (csm_col0(n) + wmax + 2 * n + 3) / 4;
    int words = w0, best = 1 << 30;
    for (int w = w0; w < w0 + 8; ++w) {
        const int c = csm_stride_cost(4 * w, n);
        if (c < best) {
            best = c;
            words = w;
        }
    }
    *ws = 4 * words;
    // bordered map rows plus the sentinel block of 2n + 1 zero rows, and 16
    // bytes for the word after the last one a candidate group reads
    const size_t bytes = (size_t)(4 * words) * (size_t)(hmax + 4 * n + 2 * n + 1) + 16;
    return (bytes + 15) & ~(size_t)15;
}

cudaError_t csm_set_smem(size_t bytes) {
    return cudaFuncSetAttribute(csm2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

cudaError_t launch_csm2d(const Step2DParams &p, int n_xy, int n_th, int sep, float dth,
                         size_t map_bytes, int ws, const float *pose_pred, const float *ranges,
                         float *pose_out, float *match, long long *scores, bool reset_empty,
                         cudaStream_t s) {
    CsmArgs a{n_xy, n_th, sep, dth, map_bytes, ws, reset_empty, pose_pred, ranges, pose_out, match,
              scores};
    csm2d_kernel<<<p.E, kCsmBlock, map_bytes, s>>>(p, a);
    return cudaGetLastError();
}

}  // namespace aslam
