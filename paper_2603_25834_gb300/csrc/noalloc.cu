// noalloc.cu -- aslam_scan_update_noalloc: integrate one LiDAR scan per
// environment into caller-owned log-odds grids without allocating anything.
//
// Who needs this: code that runs where it may not allocate device memory --
// e.g. a plugin handed fixed buffers by a host framework that owns the
// allocator, or a pipeline whose memory budget is frozen after start-up.
// Such a caller has its maps, poses and output buffers already; what it
// cannot provide is per-call scratch.  This entry point takes that scratch
// from a fixed array in the library's own device data, so it calls no
// cudaMalloc / cudaFree (nor any allocating library routine).
//
// Limits and sharing:
//   * the scratch array holds at most kMaxCells 32-bit counters (16 MiB),
//     the offsets and sizes of at most kMaxEnvs grids and one beam table
//     (1024 beams); larger requests are rejected with ASLAM_ERR_INVALID_ARG;
//   * every GPU that loads the library holds the array until the process
//     exits;
//   * every call on a device uses the same array: each call clears the part
//     it needs first, but calls that overlap on the GPU (different streams,
//     or host threads racing) corrupt each other -- serialise them;
//   * the first call on each device looks the array's device address up
//     (cudaGetSymbolAddress) with that device current;
//   * every call copies its tables from host memory (some of it on the
//     call's own stack) with cudaMemcpyAsync, so a call made while `stream`
//     is being captured is rejected with ASLAM_ERR_UNSUPPORTED.
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>

#include "aslam_internal.cuh"

namespace aslam {
namespace {

constexpr long long kMaxCells = 1LL << 22;          // 4,194,304 cells (16 MiB of counters)
constexpr int kMaxEnvs = 2048;
constexpr size_t kOffAt = 0;                         // int64 [E+1] grid offsets
constexpr size_t kWAt = 16640;                       // int32 [E] widths
constexpr size_t kHAt = kWAt + 4 * kMaxEnvs;         // int32 [E] heights
constexpr size_t kBeamAt = kHAt + 4 * kMaxEnvs;      // float2 [B] beam directions
constexpr size_t kCntAt = 41216;                     // uint32 [cells] (hits << 16 | misses)
constexpr size_t kScratchBytes = kCntAt + 4 * (size_t)kMaxCells;
static_assert(kOffAt + 8 * (kMaxEnvs + 1) <= kWAt, "offset table overlaps the widths");
static_assert(kBeamAt + 8 * ASLAM_MAX_BEAMS <= kCntAt, "beam table overlaps the counters");
static_assert(kCntAt % 256 == 0, "counters must start 256-byte aligned");

// The scratch array.  In host code this name is only a stand-in for the
// device address, which comes from cudaGetSymbolAddress (scratch_ptr()).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};
thread_local std::string g_na_error;

struct ScanParams {
    int E, B, hit_q, miss_q, clamp_q, Tmax;
    long long cells;
    float res, r_max, sigma;
    uint2 key;
    int env_base;
    float r_min, dec_scale;
    const uint8_t *gt;
    const float *pose;
    const int *step;
    short *belief;
    float *ranges;
    const long long *off;      // scratch
    const int *Wd, *Hd;        // scratch
    const float2 *beams;       // scratch
    unsigned *cnt;             // scratch
};

// One thread per beam: ground-truth traversal to the first occupied cell,
// range noise, then a traversal to the measured endpoint that adds one miss
// to every crossed cell and a hit to the endpoint of a returned beam (the
// same definitions as the batched step, with global counters).
__global__ void scan_rays_kernel(const ScanParams p) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)p.E * p.B) return;
    const int e = (int)(r / p.B), b = (int)(r - (long long)e * p.B);
    const long long off = p.off[e];
    const int W = p.Wd[e], H = p.Hd[e];
    const float x = p.pose[3 * e], y = p.pose[3 * e + 1], th = p.pose[3 * e + 2];
    float s, c;
    det_sincos(th, s, c);
    const float2 cs = p.beams[b];
    const int Px = q16_of(x, p.res), Py = q16_of(y, p.res);
    const int Dx = __float2int_rn(fmul(fsub(fmul(c, cs.x), fmul(s, cs.y)), 1073741824.0f));
    const int Dy = __float2int_rn(fmul(fadd(fmul(s, cs.x), fmul(c, cs.y)), 1073741824.0f));
    const int i0 = Px >> 16, j0 = Py >> 16;
    float z = p.r_max;
    if ((unsigned)i0 < (unsigned)W && (unsigned)j0 < (unsigned)H) {
        const int sx = (Dx > 0) - (Dx < 0), sy = (Dy > 0) - (Dy < 0);
        const long long adx = Dx < 0 ? -(long long)Dx : Dx, ady = Dy < 0 ? -(long long)Dy : Dy;
        const long long nx0 = Dx > 0 ? ((long long)(i0 + 1) << 16) - Px
                                     : (Dx < 0 ? (long long)Px - ((long long)i0 << 16) : 65536);
        const long long ny0 = Dy > 0 ? ((long long)(j0 + 1) << 16) - Py
                                     : (Dy < 0 ? (long long)Py - ((long long)j0 << 16) : 65536);
        const long long e0 = nx0 * ady - ny0 * adx, dA = ady << 16, dB = adx << 16;
        // ground truth
        bool hit = false;
        float z_true = p.r_max;
        int i = i0, j = j0;
        if (p.gt[off + (long long)j0 * W + i0]) {
            hit = true;
            z_true = 0.0f;
        } else {
            const int Ks = crossings_le(nx0, adx, p.Tmax) + crossings_le(ny0, ady, p.Tmax);
            long long ee = e0;
            bool lastx = false;
            for (int st = 0; st < Ks; ++st) {
                lastx = ee < 0;
                if (lastx) { i += sx; ee += dA; } else { j += sy; ee -= dB; }
                if ((unsigned)i >= (unsigned)W || (unsigned)j >= (unsigned)H) break;
                if (p.gt[off + (long long)j * W + i]) { hit = true; break; }
            }
            if (hit) {
                const long long n = lastx ? nx0 + ((long long)(abs(i - i0) - 1) << 16)
                                          : ny0 + ((long long)(abs(j - j0) - 1) << 16);
                const long long ad = lastx ? adx : ady;
                z_true = fmul(fmul(fdiv(__int2float_rn((int)n), __int2float_rn((int)ad)), 16384.0f), p.res);
            }
        }
        z = z_true;
        if (hit) {
            const float g = det_gauss(p.key, (unsigned)(p.env_base + e), (unsigned)p.step[e], (unsigned)b);
            z = measured_range(z_true, g, p.sigma, p.r_min, p.r_max, p.dec_scale);
        }
        const int Tz = hit ? q16_of(z, p.res) : p.Tmax;
        // belief
        const int Ku = crossings_le(nx0, adx, Tz) + crossings_le(ny0, ady, Tz);
        i = i0;
        j = j0;
        long long ee = e0;
        for (int st = 0;; ++st) {
            const bool last = st == Ku;
            red_add(&p.cnt[off + (long long)j * W + i], (last && hit) ? 0x10000u : 1u);
            if (last) break;
            if (ee < 0) { i += sx; ee += dA; } else { j += sy; ee -= dB; }
            if ((unsigned)i >= (unsigned)W || (unsigned)j >= (unsigned)H) break;
        }
    }
    p.ranges[(long long)e * p.B + b] = z;
}

// One thread per cell: L' = clamp(L + hits*HIT + misses*MISS), once per scan.
__global__ void scan_apply_kernel(const ScanParams p) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < p.cells;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned c = p.cnt[k];
        if (!c) continue;
        int l = p.belief[k] + (int)(c >> 16) * p.hit_q + (int)(c & 0xffffu) * p.miss_q;
        p.belief[k] = (short)min(max(l, -p.clamp_q), p.clamp_q);
    }
}

aslam_status na_fail(aslam_status s, const std::string &m) {
    g_na_error = m;
    set_thread_error(m.c_str());
    return s;
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
aslam_status scratch_ptr(unsigned char **out) {
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return na_fail(ASLAM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(ASLAM_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        ce = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (ce != cudaSuccess || !ptr)
            return na_fail(ASLAM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
        g_scratch_ptr[dev] = (unsigned char *)ptr;
    }
    *out = g_scratch_ptr[dev];
    return ASLAM_OK;
}

}  // namespace
}  // namespace aslam

using namespace aslam;

extern "C" aslam_status aslam_scan_update_noalloc(const aslam_config *cfg, const uint8_t *d_gt,
                                                  const int64_t *h_gt_off, const float *d_pose,
                                                  const int32_t *d_step, int16_t *d_belief,
                                                  float *d_ranges, void *stream) {
    if (!cfg || cfg->struct_size != sizeof(aslam_config) || cfg->version != ASLAM_CONFIG_VERSION)
        return na_fail(ASLAM_ERR_INVALID_ARG, "bad config struct");
    const int E = cfg->n_envs;
    if (E < 1 || E > kMaxEnvs)
        return na_fail(ASLAM_ERR_INVALID_ARG, "n_envs out of [1, 2048] (the static scratch maximum)");
    if (cfg->env_base < 0 || (long long)cfg->env_base + E > 2147483647LL)
        return na_fail(ASLAM_ERR_INVALID_ARG, "env_base out of [0, 2^31 - 1 - n_envs]");
    if (!cfg->h_map_w || !cfg->h_map_h || !cfg->h_n_beams || !h_gt_off || !d_gt || !d_pose ||
        !d_step || !d_belief || !d_ranges)
        return na_fail(ASLAM_ERR_INVALID_ARG, "NULL pointer argument");
    const int B = cfg->h_n_beams[0];
    if (B < 1 || B > ASLAM_MAX_BEAMS) return na_fail(ASLAM_ERR_INVALID_ARG, "n_beams out of [1, 1024]");
    long long cells = 0;
    for (int e = 0; e < E; ++e) {
        if (cfg->h_n_beams[e] != B)
            return na_fail(ASLAM_ERR_INVALID_ARG, "every env must have the same beam count here");
        const int W = cfg->h_map_w[e], H = cfg->h_map_h[e];
        if (W < 1 || H < 1 || W > ASLAM_MAX_MAP_SIDE || H > ASLAM_MAX_MAP_SIDE)
            return na_fail(ASLAM_ERR_INVALID_ARG, "map side out of [1, ASLAM_MAX_MAP_SIDE]");
        if (h_gt_off[e] != cells || h_gt_off[e + 1] - h_gt_off[e] != (int64_t)W * H)
            return na_fail(ASLAM_ERR_INVALID_ARG, "h_gt_off must be the packed prefix sum of W*H");
        cells += (long long)W * H;
    }
    if (cells > kMaxCells)
        return na_fail(ASLAM_ERR_INVALID_ARG,
                       "total grid cells exceed the static scratch maximum of 4194304");
    if (!(cfg->res_m > 0.0f) || !(cfg->r_max_m > 0.0f) || (double)cfg->r_max_m / cfg->res_m > 16384.0)
        return na_fail(ASLAM_ERR_INVALID_ARG, "res_m / r_max_m out of range");
    if (cfg->l_clamp_q < 1 || cfg->l_clamp_q > 32767 || !(cfg->noise_sigma_m >= 0.0f))
        return na_fail(ASLAM_ERR_INVALID_ARG, "l_clamp_q or noise_sigma_m out of range");
    // hits * l_hit_q + misses * l_miss_q stays inside a 32-bit int for up to
    // 2^15 beams per cell only with increments of at most 16 bits
    if (std::abs(cfg->l_hit_q) > 32767 || std::abs(cfg->l_miss_q) > 32767)
        return na_fail(ASLAM_ERR_INVALID_ARG, "|l_hit_q|, |l_miss_q| must be <= 32767");
    if (cfg->range_decimals < -1 || cfg->range_decimals > 6 || !(cfg->r_min_m >= 0.0f) ||
        !(cfg->r_min_m <= cfg->r_max_m))
        return na_fail(ASLAM_ERR_INVALID_ARG, "range_decimals or r_min_m out of range");

    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t qe = cudaStreamIsCapturing(s, &cap);
    if (qe != cudaSuccess)
        return na_fail(ASLAM_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(qe));
    if (cap != cudaStreamCaptureStatusNone)
        return na_fail(ASLAM_ERR_UNSUPPORTED,
                       "stream is being captured: this call copies host tables and cannot be captured");
    unsigned char *base = nullptr;
    aslam_status st = scratch_ptr(&base);
    if (st != ASLAM_OK) return st;

    // Beam directions, as the batched step builds them (host fp64 -> fp32).
    float2 tab[ASLAM_MAX_BEAMS];
    const double two_pi = 2.0 * 3.14159265358979323846;
    const double fov = (double)cfg->fov_rad;
    const bool full_turn = fov <= 0.0 || fov >= two_pi - 1e-9;
    for (int k = 0; k < B; ++k) {
        double a;
        if (full_turn) a = (two_pi * (double)k) / (double)B;
        else if (B == 1) a = 0.0;
        else a = -0.5 * fov + ((double)k * fov) / (double)(B - 1);
        tab[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    // Pageable host sources: each copy is staged before the call returns.
    cudaError_t ce = cudaMemcpyAsync(base + kOffAt, h_gt_off, 8 * (size_t)(E + 1),
                                     cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(base + kWAt, cfg->h_map_w, 4 * (size_t)E, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(base + kHAt, cfg->h_map_h, 4 * (size_t)E, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(base + kBeamAt, tab, 8 * (size_t)B, cudaMemcpyHostToDevice, s);
    // The counters must start at zero: clear the part this call uses.
    if (ce == cudaSuccess) ce = cudaMemsetAsync(base + kCntAt, 0, 4 * (size_t)cells, s);
    if (ce != cudaSuccess) return na_fail(ASLAM_ERR_CUDA, std::string("scratch upload: ") + cudaGetErrorString(ce));

    ScanParams p;
    p.E = E;
    p.B = B;
    p.hit_q = cfg->l_hit_q;
    p.miss_q = cfg->l_miss_q;
    p.clamp_q = cfg->l_clamp_q;
    p.Tmax = (int)lrintf((cfg->r_max_m / cfg->res_m) * 65536.0f);
    p.cells = cells;
    p.res = cfg->res_m;
    p.r_max = cfg->r_max_m;
    p.sigma = cfg->noise_sigma_m;
    p.key = make_uint2((unsigned)cfg->seed, (unsigned)(cfg->seed >> 32));
    p.env_base = cfg->env_base;
    p.r_min = cfg->r_min_m;
    p.dec_scale = range_scale(cfg->range_decimals);
    p.gt = d_gt;
    p.pose = d_pose;
    p.step = d_step;
    p.belief = d_belief;
    p.ranges = d_ranges;
    p.off = reinterpret_cast<const long long *>(base + kOffAt);
    p.Wd = reinterpret_cast<const int *>(base + kWAt);
    p.Hd = reinterpret_cast<const int *>(base + kHAt);
    p.beams = reinterpret_cast<const float2 *>(base + kBeamAt);
    p.cnt = reinterpret_cast<unsigned *>(base + kCntAt);
    const long long rays = (long long)E * B;
    scan_rays_kernel<<<(unsigned)((rays + 127) / 128), 128, 0, s>>>(p);
    scan_apply_kernel<<<(unsigned)std::min<long long>((cells + 255) / 256, 4096), 256, 0, s>>>(p);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return na_fail(ASLAM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(ce));
    return ASLAM_OK;
}
