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
// One CTA per env.  The env's evidence map (one byte per cell) is staged in
// shared memory when it fits, and the returned beams are compacted once;
// the rotations are processed one at a time: the endpoint cells of the
// returned beams for th_k go to shared memory (one thread per beam), then
// each thread sums one candidate over a slice of the beams, and the slices
// are added in a fixed order into a shared score table.
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

__global__ void __launch_bounds__(kCsmBlock) csm2d_kernel(const Step2DParams p, const CsmArgs a) {
    extern __shared__ __align__(16) unsigned char s_map[];
    __shared__ int2 s_cell[ASLAM_MAX_BEAMS];
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
    // rows padded by 4 bytes: vertically adjacent cells fall in different banks
    const int ws = W + 4;
    if (staged) {
        // (row, column) of element q tracked incrementally (no division per cell)
        int ii = tid % W, jj = tid / W;
        const int di = nt % W, dj = nt / W;
        for (long long q = tid; q < (long long)W * H; q += nt) {
            s_map[(long long)jj * ws + ii] = empty ? (unsigned char)0 : (unsigned char)evidence(L[q]);
            ii += di;
            jj += dj;
            if (ii >= W) {
                ii -= W;
                ++jj;
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
            s_cell[q] = make_int2((int)floorf(fdiv(ex, p.res)), (int)floorf(fdiv(ey, p.res)));
        }
        __syncthreads();
        int acc = 0;
        if (sl < nslice) {
            for (int q = sl; q < nret; q += nslice) {
                const int2 cc = s_cell[q];
                const int i = cc.x + ci_off, j = cc.y + cj_off;
                if ((unsigned)i < (unsigned)W && (unsigned)j < (unsigned)H) {
                    const long long kk = (long long)j * W + i;
                    acc += staged ? (int)s_map[(long long)j * ws + i]
                                  : (empty ? 0 : (int)evidence(L[kk]));
                }
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

size_t csm_map_bytes(int W, int H) {
    const size_t n = (size_t)(W + 4) * H;               // padded rows
    return (n + 15) & ~(size_t)15;
}

cudaError_t csm_set_smem(size_t bytes) {
    return cudaFuncSetAttribute(csm2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

cudaError_t launch_csm2d(const Step2DParams &p, int n_xy, int n_th, int sep, float dth,
                         size_t map_bytes, const float *pose_pred, const float *ranges,
                         float *pose_out, float *match, long long *scores, bool reset_empty,
                         cudaStream_t s) {
    CsmArgs a{n_xy, n_th, sep, dth, map_bytes, reset_empty, pose_pred, ranges, pose_out, match,
              scores};
    csm2d_kernel<<<p.E, kCsmBlock, map_bytes, s>>>(p, a);
    return cudaGetLastError();
}

}  // namespace aslam
