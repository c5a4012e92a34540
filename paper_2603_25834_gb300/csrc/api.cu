// api.cu -- host implementation of the libaslam C ABI (include/aslam.h).
//
// The library owns no device memory: every device array lives in the
// caller's workspace at offsets computed by `build_layout`, identically in
// aslam_workspace_bytes and aslam_create_batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "aslam_internal.cuh"

using namespace aslam;

namespace {

thread_local std::string g_thread_error;

constexpr size_t kAlign = 256;
constexpr int kCellPad = 256;    // env grids start on 512-byte (int16) boundaries

struct HostInfo {
    int E = 0, b_max = 0, r8_max = 1, dims = 2, n_rings = 1;
    std::vector<int> W, H, B, Vw, Vh, R8, D;
    std::vector<long long> map_off, gtb_off, ray_off, visit_off;
    int gt_words_max = 0;
};

struct Offsets {
    size_t W, H, B, Vw, Vh, R8, Dd, elev, order, map_off, gtb_off, ray_off, visit_off, src_off;
    size_t beam_cs, beam_df, lut, gt_bits;
    size_t x, y, th, u_prev, t, g, ep, done, Hq;
    size_t belief, visit, spawn;
    size_t z, z_true, hit, dbg, ray_cells, gt_cells, terms, reward;
    size_t far_cnt, far_bits, ray_code, env_sense, bundles, queue, err, tune_actions;
    size_t io_in, io_out;        // aslam_step_host staging: [3E] in, [E (b_max + 3)] out
    size_t pose_cov, u_scan;
    size_t win_x, win_odo, win_meas, win_minfo, win_n, slam_pred, slam_odo, csm_pose, csm_match,
        csm_scores, slam_upd_w, slam_gn_pose;
    size_t total;
};

size_t pad_to(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Does a step evaluate the soft range model in the step (in-step U or the
// match correction)?  Those kernels read the beams' fp64 directions.
bool soft_dirs(const aslam_config *c) {
    return c->dims == 2 && (c->u_mode == ASLAM_U_SCANMATCH ||
                            (c->u_mode == ASLAM_U_FIXEDLAG && c->slam_gn_iters > 0));
}

// Visit-workspace dims (Eq. 9 counts cells over a workspace much larger than the map):
// twice the map extent per axis, in visit cells, computed in fp32.
void visit_dims(int W, int H, float res, float vc, int *Vw, int *Vh) {
    float ew = 2.0f * ((float)W * res), eh = 2.0f * ((float)H * res);
    int a = (int)std::ceil(ew / vc), b = (int)std::ceil(eh / vc);
    *Vw = a < 1 ? 1 : a;
    *Vh = b < 1 ? 1 : b;
}

// Smallest Chebyshev distance d (>= 2) from the robot's cell beyond which no
// cell can be crossed by more than 15 of the B beams: a cell at distance d
// has its centre >= d - 1/2 cells away and lies in a disc of radius
// sqrt(2)/2 about it, so the beams crossing it span an angle of at most
// 2*asin(0.70711/(d - 1/2)) (+2e-6 rad for fp32 direction rounding).
int near_radius(int B, double fov) {
    if (B <= 15) return 1;
    const double two_pi = 2.0 * 3.14159265358979323846;
    const bool full_turn = fov <= 0.0 || fov >= two_pi - 1e-9;
    const double dbeta = full_turn ? two_pi / B : fov / (double)(B - 1);
    for (int d = 2; d < 4096; ++d) {
        const double x = 0.70711 / ((double)d - 0.5);
        if (x >= 1.0) continue;
        const int n = (int)std::floor((2.0 * std::asin(x) + 2e-6) / dbeta) + 1;
        if (n <= 15) return d;
    }
    return 4096;
}

// 3-D: smallest Chebyshev distance d (>= 2) from the sensor's voxel beyond
// which no voxel can be crossed by more than 255 of the rings x azimuths
// beams.  A voxel at distance d has its centre >= d - 1/2 voxels from the
// sensor and lies in a ball of radius sqrt(3)/2 about it, so every beam
// crossing it is within alpha = asin(0.86603 / (d - 1/2)) of one direction,
// and any two of them within 2 alpha of each other.  Two beams differ in
// angle by at least their elevation difference, so they come from at most
// floor(2 alpha / de) + 1 rings (de: ring spacing); two beams of one ring at
// elevation e and azimuth difference dphi are 2 asin(cos(e) sin(dphi / 2))
// apart, so one ring contributes at most floor(2 asin(sin(alpha) /
// cos(e_abs)) / dphi_a) + 1 of them (e_abs: the largest |elevation|, dphi_a:
// the azimuth spacing), +2e-6 rad for the fp32 direction rounding.
int near_radius_3d(int A, int R, double el_min, double el_max) {
    const double two_pi = 2.0 * 3.14159265358979323846;
    const double dphi = two_pi / std::max(A, 1);
    const double de = R > 1 ? (el_max - el_min) / (double)(R - 1) : 0.0;
    const double cmin = std::cos(std::max(std::fabs(el_min), std::fabs(el_max)));
    for (int d = 2; d < 4096; ++d) {
        const double x = 0.86603 / ((double)d - 0.5);
        if (x >= 1.0) continue;
        const double alpha = std::asin(x) + 1e-6;
        const long long rings = R > 1 ? std::min<long long>(R, (long long)std::floor(2.0 * alpha / de) + 1) : 1;
        const double sa = std::sin(alpha) / cmin;
        const long long az = sa >= 1.0 ? A
                                        : std::min<long long>(A, (long long)std::floor((2.0 * std::asin(sa) + 2e-6) / dphi) + 1);
        if (rings * az <= 255) return d;
    }
    return 4096;
}

bool validate(const aslam_config *c, std::string *msg) {
    auto fail = [&](const char *m) { *msg = m; return false; };
    if (!c) return fail("config is NULL");
    if (c->struct_size != sizeof(aslam_config)) return fail("config struct_size mismatch");
    if (c->version != ASLAM_CONFIG_VERSION) return fail("config version mismatch");
    if (c->n_envs < 1) return fail("n_envs must be >= 1");
    if (c->env_base < 0 || (long long)c->env_base + c->n_envs > 2147483647LL)
        return fail("env_base out of [0, 2^31 - 1 - n_envs]");
    if (c->dims != 2 && c->dims != 3) return fail("dims must be 2 or 3");
    if (c->dims == 3) {
        if (!c->h_map_d) return fail("h_map_d is NULL for a 3-D batch");
        if (c->n_rings < 1 || c->n_rings > 256) return fail("n_rings out of [1, 256]");
        if (!(c->elev_min_rad <= c->elev_max_rad)) return fail("elev_min_rad exceeds elev_max_rad");
        for (int e = 0; e < c->n_envs; ++e) {
            if (c->h_map_d[e] < 1 || c->h_map_d[e] > 4096) return fail("map depth out of [1, 4096]");
            if (c->h_map_w[e] % 8) return fail("3-D maps need a width that is a multiple of 8");
            if ((long long)c->h_map_w[e] * c->h_map_h[e] * c->h_map_d[e] > (1LL << 30))
                return fail("3-D map larger than 2^30 voxels");
        }
    }
    if (c->n_spawn < 1) return fail("n_spawn must be >= 1");
    if (!c->h_map_w || !c->h_map_h || !c->h_n_beams) return fail("map dims / beams arrays are NULL");
    for (int e = 0; e < c->n_envs; ++e) {
        if (c->h_map_w[e] < 1 || c->h_map_w[e] > ASLAM_MAX_MAP_SIDE || c->h_map_h[e] < 1 ||
            c->h_map_h[e] > ASLAM_MAX_MAP_SIDE)
            return fail("map side out of [1, ASLAM_MAX_MAP_SIDE]");
        if (c->h_n_beams[e] < 0 || c->h_n_beams[e] > ASLAM_MAX_BEAMS)
            return fail("n_beams out of [0, ASLAM_MAX_BEAMS]");
        if (c->dims == 2 && (long long)c->h_map_w[e] * c->h_map_h[e] > 1600LL * 1024)
            return fail("2-D map larger than 1638400 cells");
    }
    {
        // every real-valued field must be finite (NaN fails every comparison
        // below, but +-Inf would pass the sign checks)
        const double vals[] = {c->res_m, c->r_max_m, c->fov_rad, c->noise_sigma_m, c->dt_s,
                               c->v_max, c->w_max, c->d_crash, c->d_full, c->visit_cell_m,
                               c->logodds_scale, c->lam_col, c->lam_explore, c->lam_abs,
                               c->lam_delta, c->kappa, c->u_hi, c->r_min_m, c->sensor_z_m,
                               c->elev_min_rad, c->elev_max_rad, c->uq_step_m,
                               c->uq_range_sigma_m, c->uq_u_scale, c->csm_dth_rad,
                               c->uq_odo_sigma[0], c->uq_odo_sigma[1], c->uq_odo_sigma[2],
                               c->uq_prior_sigma[0], c->uq_prior_sigma[1], c->uq_prior_sigma[2],
                               c->slam_meas_info[0], c->slam_meas_info[1], c->slam_meas_info[2],
                               c->slam_prior_info[0], c->slam_prior_info[1],
                               c->slam_prior_info[2]};
        for (double v : vals)
            if (!std::isfinite(v)) return fail("a real-valued config field is NaN or infinite");
    }
    if (!(c->res_m > 0.0f) || !(c->r_max_m > 0.0f)) return fail("res_m and r_max_m must be > 0");
    if ((double)c->r_max_m / c->res_m > 16384.0) return fail("r_max_m / res_m must be <= 16384 cells");
    if (!(c->dt_s >= 0.0f) || !(c->v_max >= 0.0f) || !(c->w_max >= 0.0f))
        return fail("dt_s, v_max, w_max must be >= 0");
    if (!(c->noise_sigma_m >= 0.0f)) return fail("noise_sigma_m must be >= 0");
    if (!(c->r_min_m >= 0.0f) || !(c->r_min_m <= c->r_max_m))
        return fail("r_min_m must be in [0, r_max_m]");
    if (c->range_decimals < -1 || c->range_decimals > 6) return fail("range_decimals out of [-1, 6]");
    if (c->u_mode != ASLAM_U_CALLER && c->u_mode != ASLAM_U_SCANMATCH &&
        c->u_mode != ASLAM_U_FIXEDLAG)
        return fail("unknown u_mode");
    if (c->u_mode == ASLAM_U_FIXEDLAG) {
        if (c->slam_window < 1 || c->slam_window > 16) return fail("slam_window out of [1, 16]");
        if (c->slam_iters < 0 || c->slam_iters > 20) return fail("slam_iters out of [0, 20]");
        if (c->csm_n_xy < 0 || c->csm_n_xy > 8 || c->csm_n_th < 0 || c->csm_n_th > 8)
            return fail("csm_n_xy and csm_n_th must be in [0, 8]");
        if (c->csm_sep < 0 || !(c->csm_dth_rad > 0.0f)) return fail("need csm_sep >= 0, csm_dth_rad > 0");
        for (int q = 0; q < 3; ++q)
            if (!(c->slam_meas_info[q] > 0.0f) || !(c->slam_prior_info[q] > 0.0f))
                return fail("slam_meas_info and slam_prior_info must be > 0");
        if (c->slam_weighted_update != 0 && c->slam_weighted_update != 1)
            return fail("slam_weighted_update must be 0 or 1");
        if (c->slam_gn_iters < 0 || c->slam_gn_iters > 10) return fail("slam_gn_iters out of [0, 10]");
    }
    if (c->u_mode != ASLAM_U_CALLER) {
        if (c->dims != 2) return fail("an in-step u_mode needs dims = 2");
        if (c->uq_samples < 1 || c->uq_samples > ASLAM_SOFT_MAX_SAMPLES)
            return fail("uq_samples out of [1, ASLAM_SOFT_MAX_SAMPLES]");
        if (!(c->uq_step_m >= 0.0f) || !(c->uq_range_sigma_m > 0.0f) || !(c->uq_u_scale >= 0.0f))
            return fail("need uq_step_m >= 0, uq_range_sigma_m > 0, uq_u_scale >= 0");
        for (int i = 0; i < 3; ++i)
            if (!(c->uq_odo_sigma[i] > 0.0f) || !(c->uq_prior_sigma[i] > 0.0f))
                return fail("uq_odo_sigma and uq_prior_sigma must be > 0");
    }
    if (c->l_clamp_q < 1 || c->l_clamp_q > 8192) return fail("l_clamp_q out of [1, 8192]");
    if (std::abs(c->l_hit_q) > 32767 || std::abs(c->l_miss_q) > 32767)
        return fail("|l_hit_q|, |l_miss_q| must be <= 32767");
    if (c->t_episode < 1) return fail("t_episode must be >= 1");
    if (!(c->d_full > c->d_crash)) return fail("d_full must exceed d_crash");
    if (!(c->visit_cell_m > 0.0f)) return fail("visit_cell_m must be > 0");
    if (!(c->kappa > 0.0) || !(c->u_hi > 0.0)) return fail("kappa and u_hi must be > 0");
    if (!(c->logodds_scale > 0.0f)) return fail("logodds_scale must be > 0");
    if (c->reward_mode != ASLAM_REWARD_ENTROPY && c->reward_mode != ASLAM_REWARD_COMPOSITE)
        return fail("unknown reward_mode");
    if (c->threads_per_cta != 0 &&
        (c->threads_per_cta < 128 || c->threads_per_cta > 1024 || c->threads_per_cta % 32))
        return fail("threads_per_cta must be 0 or a multiple of 32 in [128, 1024]");
    if (c->window_cells != 0 && (c->window_cells < 64 || c->window_cells % 8))
        return fail("window_cells must be 0 or a multiple of 8 >= 64");
    return true;
}

void host_info(const aslam_config *c, HostInfo *hi) {
    const int E = c->n_envs;
    hi->E = E;
    hi->dims = c->dims;
    hi->n_rings = c->dims == 3 ? c->n_rings : 1;
    hi->W.assign(c->h_map_w, c->h_map_w + E);
    hi->H.assign(c->h_map_h, c->h_map_h + E);
    hi->B.assign(c->h_n_beams, c->h_n_beams + E);
    hi->D.assign(E, 1);
    if (c->dims == 3) {
        hi->D.assign(c->h_map_d, c->h_map_d + E);
        for (int e = 0; e < E; ++e) hi->B[e] *= c->n_rings;   // beams = rings x azimuths
    }
    hi->Vw.resize(E);
    hi->Vh.resize(E);
    hi->R8.resize(E);
    hi->r8_max = 1;
    hi->map_off.assign(E + 1, 0);
    hi->gtb_off.assign(E + 1, 0);
    hi->ray_off.assign(E + 1, 0);
    hi->visit_off.assign(E + 1, 0);
    hi->gt_words_max = 0;
    hi->b_max = *std::max_element(hi->B.begin(), hi->B.end());
    for (int e = 0; e < E; ++e) {
        const long long n = (long long)hi->W[e] * hi->H[e] * hi->D[e];
        const long long words = (long long)pad_to((size_t)((n + 31) / 32), 4);
        hi->map_off[e + 1] = hi->map_off[e] + (long long)pad_to((size_t)n, kCellPad);
        hi->gtb_off[e + 1] = hi->gtb_off[e] + words;
        hi->ray_off[e + 1] = hi->ray_off[e] + hi->B[e];
        visit_dims(hi->W[e], hi->H[e], c->res_m, c->visit_cell_m, &hi->Vw[e], &hi->Vh[e]);
        hi->visit_off[e + 1] = hi->visit_off[e] + (long long)hi->Vw[e] * hi->Vh[e];
        hi->gt_words_max = std::max(hi->gt_words_max, (int)words);
        hi->R8[e] = c->dims == 3 ? near_radius_3d(hi->B[e] / hi->n_rings, hi->n_rings,
                                                  (double)c->elev_min_rad, (double)c->elev_max_rad)
                                 : near_radius(hi->B[e], (double)c->fov_rad);
        hi->r8_max = std::max(hi->r8_max, hi->R8[e]);
    }
}

Offsets build_layout(const aslam_config *c, const HostInfo &hi) {
    Offsets o{};
    size_t cur = 0;
    auto add = [&](size_t bytes) {
        size_t at = pad_to(cur, kAlign);
        cur = at + bytes;
        return at;
    };
    const size_t E = hi.E;
    const size_t cells = (size_t)hi.map_off[E];
    const size_t rays = (size_t)std::max<long long>(hi.ray_off[E], 1);
    const bool debug = (c->flags & ASLAM_FLAG_DEBUG) != 0;
    o.W = add(4 * E);
    o.H = add(4 * E);
    o.B = add(4 * E);
    o.Vw = add(4 * E);
    o.Vh = add(4 * E);
    o.R8 = add(4 * E);
    o.Dd = add(4 * E);
    o.elev = add(8 * (size_t)hi.n_rings);
    o.order = add(4 * E);
    o.map_off = add(8 * (E + 1));
    o.gtb_off = add(8 * (E + 1));
    o.ray_off = add(8 * (E + 1));
    o.visit_off = add(8 * (E + 1));
    o.src_off = add(8 * (E + 1));
    o.beam_cs = add(8 * rays);
    o.beam_df = add(soft_dirs(c) ? 16 * rays : 0);
    o.lut = add(8 * (2 * (size_t)c->l_clamp_q + 1));
    o.gt_bits = add(4 * (size_t)hi.gtb_off[E]);
    o.x = add(4 * E);
    o.y = add(4 * E);
    o.th = add(4 * E);
    o.u_prev = add(4 * E);
    o.t = add(4 * E);
    o.g = add(4 * E);
    o.ep = add(4 * E);
    o.done = add(4 * E);
    o.Hq = add(8 * E);
    o.belief = add(2 * cells);
    o.visit = add(4 * (size_t)hi.visit_off[E]);
    o.spawn = add(12 * E * (size_t)c->n_spawn);
    o.z = add(4 * rays);
    o.z_true = add(debug ? 4 * rays : 0);
    o.hit = add(debug ? rays : 0);
    o.dbg = add(debug ? 4 * cells : 0);
    o.ray_cells = add(8 * E);
    o.gt_cells = add(8 * E);
    o.terms = add(4 * E * kTerms);
    o.reward = add(4 * E);
    o.far_cnt = add(4 * cells);
    o.far_bits = add(cells / 64);
    o.ray_code = add(4 * rays);
    o.env_sense = add(env_sense_bytes() * E);
    {
        size_t nb = 0;
        const int sb = sense_block(hi.gt_words_max);
        // at least one bundle per env: its first bundle integrates the env
        for (int e = 0; e < hi.E; ++e) nb += std::max<size_t>(1, (size_t)(hi.B[e] + sb - 1) / sb);
        o.bundles = add(8 * std::max<size_t>(nb, 1));
    }
    o.queue = add(16);         // {next item, CTAs finished, sensing CTAs finished}
    o.err = add(4);
    o.tune_actions = add(8 * E);
    o.io_in = add(12 * E);                                   // actions [E, 2], U [E]
    o.io_out = add(4 * E * ((size_t)hi.b_max + 3));          // reward [E], obs [E, b_max + 2]
    const bool uq = c->u_mode == ASLAM_U_SCANMATCH || c->u_mode == ASLAM_U_FIXEDLAG;
    const bool sl = c->u_mode == ASLAM_U_FIXEDLAG;
    o.pose_cov = add(uq ? 48 * E : 0);
    o.u_scan = add(uq ? 4 * E : 0);
    const size_t win = sl ? 12 * E * (size_t)c->slam_window : 0;
    o.win_x = add(win);
    o.win_odo = add(win);
    o.win_meas = add(win);
    o.win_minfo = add(win);
    o.win_n = add(sl ? 4 * E : 0);
    o.slam_pred = add(sl ? 12 * E : 0);
    o.slam_odo = add(sl ? 12 * E : 0);
    o.csm_pose = add(sl ? 12 * E : 0);
    o.csm_match = add(sl ? 12 * E : 0);
    o.csm_scores = add(sl ? 24 * E : 0);
    o.slam_upd_w = add(sl ? 4 * E : 0);
    o.slam_gn_pose = add(sl && c->slam_gn_iters > 0 ? 12 * E : 0);
    o.total = pad_to(cur, kAlign);
    return o;
}

}  // namespace

void aslam::set_thread_error(const char *msg) { g_thread_error = msg ? msg : ""; }

struct aslam_batch {
    aslam_config cfg;
    HostInfo hi;
    Offsets off;
    Step2DParams p;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    int sm_count = 0, smem_optin = 0;
    int block = 0, window = 0, grid = 0;
    size_t smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
    std::vector<int> order;
    // per-kernel timing (aslam_profile_begin/end): (kernels + 1) events per step
    std::vector<cudaEvent_t> prof_ev;
    int prof_cap = 0, prof_n = 0;
    // staged-map layout of aslam_csm for the last search width (-1: none)
    int csm_n = -1, csm_ws = 0;
    size_t csm_bytes = 0;
};

namespace {

aslam_status fail_b(aslam_batch *b, aslam_status s, const std::string &m) {
    if (b) b->err = m;
    g_thread_error = m;
    return s;
}

aslam_status cuda_fail(aslam_batch *b, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail_b(b, ASLAM_ERR_CUDA, m);
}

#define CK(call, where)                                        \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return cuda_fail(b, _e, where); \
    } while (0)

template <class T>
T *at(aslam_batch *b, size_t off) {
    return reinterpret_cast<T *>(b->ws + off);
}

}  // namespace

namespace aslam {
// 10^d as an fp32 scale of the range rounding (exact for d <= 10), 0 for none.
float range_scale(int d) {
    if (d < 0) return 0.0f;
    float s = 1.0f;
    for (int i = 0; i < d; ++i) s *= 10.0f;
    return s;
}
}  // namespace aslam

namespace {

int step_kernels(const aslam_batch *b) {
    if (b->hi.dims == 3) return kStep3DKernels;
    if (b->p.u_mode == ASLAM_U_FIXEDLAG) return kStep2DKernels + (b->p.slam_gn_iters > 0 ? 5 : 4);
    return kStep2DKernels + (b->p.u_mode == ASLAM_U_SCANMATCH ? 1 : 0);
}

void release_profile(aslam_batch *b) {
    for (cudaEvent_t e : b->prof_ev) cudaEventDestroy(e);
    b->prof_ev.clear();
    b->prof_cap = b->prof_n = 0;
}

// Shared-memory needs of a window side S: words of 8-bit counters for the
// largest env (the whole map when it fits in S x S, else an S x S window).
bool plan_window(const HostInfo &hi, int S, int *win_words, std::string *msg) {
    int ww = 0;
    for (int e = 0; e < hi.E; ++e) {
        const long long n = (long long)hi.W[e] * hi.H[e];
        long long need;
        if (n <= (long long)S * S) {
            need = (n + 3) / 4;
        } else {
            const int SW = std::min(S, hi.W[e]), SH = std::min(S, hi.H[e]);
            if (hi.W[e] % 8) {
                *msg = "a map larger than the shared window needs a width that is a multiple of 8";
                return false;
            }
            if (SW < 2 * hi.R8[e] + 14 || SH < 2 * hi.R8[e] + 14) {
                *msg = "shared window too small for the beam count";
                return false;
            }
            need = ((long long)SW * SH + 3) / 4;
        }
        ww = std::max(ww, (int)pad_to((size_t)need, 16));   // the apply reads 16 words at a time
    }
    *win_words = ww;
    return true;
}

int near_words(const HostInfo &hi) {
    const int nb = 2 * hi.r8_max - 1;
    return (int)pad_to((size_t)nb * nb, 4);
}

// Shared words of the update kernel's per-beam table (Q30 direction, walk
// code and the walk's decision term at the origin), of its chunk map / touched-chunk list (4 words per thread),
// and of the entropy half table (int64 per |L| = 0..clamp).
int geo_words(const HostInfo &hi) {
    return (int)(pad_to(2 * (size_t)hi.b_max, 4) + 2 * pad_to((size_t)hi.b_max, 4));
}
int list_words(int block) { return 4 * block; }
int lut_words(int clamp_q) { return (int)pad_to(2 * ((size_t)clamp_q + 1), 4); }

int auto_window(const HostInfo &hi, int smem_optin, int clamp_q, int block) {
    long long budget_words = (smem_optin - (long long)update2d_static_smem()) / 4 -
                             geo_words(hi) - list_words(block) - near_words(hi) - lut_words(clamp_q);
    int S = (int)std::floor(std::sqrt(4.0 * (double)budget_words));
    S &= ~7;
    return std::max(64, std::min(S, ASLAM_MAX_MAP_SIDE));
}

aslam_status configure_launch(aslam_batch *b, int block, int S) {
    if (b->hi.dims == 3) {
        // voxel batches: ground-truth bits in shared memory, global counters
        // ground-truth bits, then the 32-bit near block (a cube of side 2R - 1)
        const long long nb = 2LL * b->hi.r8_max - 1;
        const long long near = nb * nb * nb;
        if (nb > 31)
            return fail_b(b, ASLAM_ERR_UNSUPPORTED, "beams too dense for the voxel near block");
        const size_t smem = 4 * ((size_t)pad_to((size_t)b->hi.gt_words_max, 4) + pad_to((size_t)near, 4));
        if (smem + step3d_static_smem() > (size_t)b->smem_optin)
            return fail_b(b, ASLAM_ERR_UNSUPPORTED, "voxel map too large for shared memory");
        b->p.near_words_max = (int)pad_to((size_t)near, 4);
        CK(step3d_set_smem(smem), "cudaFuncSetAttribute");
        int per_sm = 0;
        CK(step3d_occupancy(block, smem, &per_sm), "occupancy");
        if (per_sm < 1) return fail_b(b, ASLAM_ERR_INVALID_ARG, "launch configuration does not fit an SM");
        b->block = block;
        b->window = 0;
        b->smem = smem;
        b->grid = std::min(b->hi.E, b->sm_count * per_sm);
        b->p.gt_words_max = b->hi.gt_words_max;
        return ASLAM_OK;
    }
    int ww = 0;
    std::string msg;
    if (!plan_window(b->hi, S, &ww, &msg)) return fail_b(b, ASLAM_ERR_UNSUPPORTED, msg);
    const size_t smem = 4 * ((size_t)lut_words(b->p.clamp_q) + geo_words(b->hi) +
                             list_words(block) + ww + near_words(b->hi));
    if (smem + update2d_static_smem() > (size_t)b->smem_optin)
        return fail_b(b, ASLAM_ERR_INVALID_ARG, "shared-memory window does not fit this device");
    CK(step2d_set_smem(smem), "cudaFuncSetAttribute");
    int per_sm = 0;
    CK(step2d_occupancy(block, smem, &per_sm), "occupancy");
    if (per_sm < 1) return fail_b(b, ASLAM_ERR_INVALID_ARG, "launch configuration does not fit an SM");
    b->block = block;
    b->window = S;
    b->smem = smem;
    b->grid = std::min(b->hi.E, b->sm_count * per_sm);
    b->p.window = S;
    b->p.gt_words_max = b->hi.gt_words_max;
    b->p.win_words_max = ww;
    b->p.near_words_max = near_words(b->hi);
    b->p.lut_words = lut_words(b->p.clamp_q);
    b->p.geo_words = geo_words(b->hi);
    b->p.list_words = list_words(block);
    return ASLAM_OK;
}

int default_block(const HostInfo &hi) {
    if (hi.dims == 3) return 1024;
    int t = (std::min(hi.b_max, 512) + 31) / 32 * 32;
    return std::max(128, t);
}

aslam_status reset_all(aslam_batch *b, cudaStream_t s) {
    const size_t cells = (size_t)b->hi.map_off[b->hi.E];
    CK(cudaMemsetAsync(b->p.belief, 0, 2 * cells, s), "memset belief");
    CK(cudaMemsetAsync(b->p.visit, 0xff, 4 * (size_t)b->hi.visit_off[b->hi.E], s), "memset visit");
    CK(cudaMemsetAsync(b->p.far_cnt, 0, 4 * cells, s), "memset far counters");
    CK(cudaMemsetAsync(b->p.far_bits, 0, cells / 64, s), "memset far bitmap");
    CK(cudaMemsetAsync(b->p.queue, 0, 16, s), "memset queue");
    if (b->p.dbg_counts) CK(cudaMemsetAsync(b->p.dbg_counts, 0, 4 * cells, s), "memset debug");
    CK(launch_init_state(b->p, s), "init state");
    return ASLAM_OK;
}

}  // namespace

extern "C" {

aslam_status aslam_config_init(aslam_config *c) {
    if (!c) return ASLAM_ERR_INVALID_ARG;
    std::memset(c, 0, sizeof(*c));
    c->struct_size = sizeof(aslam_config);
    c->version = ASLAM_CONFIG_VERSION;
    c->n_envs = 1;
    c->dims = 2;
    c->n_spawn = 1;
    c->reward_mode = ASLAM_REWARD_ENTROPY;
    c->res_m = 0.05f;
    c->r_max_m = 12.0f;
    c->fov_rad = 0.0f;
    c->noise_sigma_m = 0.01f;
    c->dt_s = 0.1f;
    c->v_max = 0.5f;
    c->w_max = 1.0f;
    c->d_crash = 0.15f;
    c->d_full = 0.5f;
    c->visit_cell_m = 0.5f;
    c->l_hit_q = 870;
    c->l_miss_q = -410;
    c->l_clamp_q = 3584;
    c->t_episode = 2048;
    c->logodds_scale = 1.0f / 1024.0f;
    c->lam_col = 10.0;
    c->lam_explore = 1.0;
    c->lam_abs = 0.1;
    c->lam_delta = 1.0;
    c->kappa = 0.05;
    c->u_hi = 1.0;
    c->seed = 20260325ull;
    c->r_min_m = 0.0f;
    c->range_decimals = -1;
    c->u_mode = ASLAM_U_CALLER;
    c->uq_samples = 64;
    c->uq_step_m = 0.0f;
    c->uq_range_sigma_m = 0.01f;
    for (int i = 0; i < 3; ++i) {
        c->uq_odo_sigma[i] = 0.01f;
        c->uq_prior_sigma[i] = 0.01f;
    }
    c->uq_u_scale = 0.0f;
    c->slam_window = 8;
    c->slam_iters = 3;
    c->csm_n_xy = 5;
    c->csm_n_th = 5;
    c->csm_sep = 1;
    c->csm_dth_rad = 0.01f;
    c->slam_meas_info[0] = c->slam_meas_info[1] = 4e4f;     // sigma 5 mm at full confidence
    c->slam_meas_info[2] = 1e6f;                             // sigma 1 mrad
    for (int q = 0; q < 3; ++q) c->slam_prior_info[q] = 1e4f;
    c->slam_weighted_update = 0;
    c->slam_gn_iters = 0;
    return ASLAM_OK;
}

aslam_status aslam_workspace_bytes(const aslam_config *cfg, size_t *bytes) {
    std::string msg;
    if (!bytes) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "bytes is NULL");
    if (!validate(cfg, &msg)) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, msg);
    try {
        HostInfo hi;
        host_info(cfg, &hi);
        *bytes = build_layout(cfg, hi).total;
    } catch (const std::bad_alloc &) {
        return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "host allocation failed");
    }
    return ASLAM_OK;
}

aslam_status aslam_create_batch(const aslam_config *cfg, void *d_workspace, size_t bytes,
                                const uint8_t *d_gt, const int64_t *h_gt_off,
                                const float *d_spawn, void *stream, aslam_batch **out) {
    std::string msg;
    if (!out) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!validate(cfg, &msg)) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, msg);
    if (!d_gt || !h_gt_off || !d_spawn) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "NULL input pointer");
    if (!d_workspace || ((uintptr_t)d_workspace % kAlign))
        return fail_b(nullptr, ASLAM_ERR_WORKSPACE, "workspace is NULL or not 256-byte aligned");
    aslam_batch *b = new (std::nothrow) aslam_batch();
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "host allocation failed");
    cudaStream_t s = (cudaStream_t)stream;
    try {
        b->cfg = *cfg;
        host_info(cfg, &b->hi);
        b->off = build_layout(cfg, b->hi);
        for (int e = 0; e < cfg->n_envs; ++e) {
            if (h_gt_off[e + 1] - h_gt_off[e] !=
                (int64_t)cfg->h_map_w[e] * cfg->h_map_h[e] * b->hi.D[e]) {
                delete b;
                return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "h_gt_off does not match W*H");
            }
        }
    } catch (const std::bad_alloc &) {
        delete b;
        return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "host allocation failed");
    }
    if (bytes < b->off.total) {
        delete b;
        return fail_b(nullptr, ASLAM_ERR_WORKSPACE, "workspace smaller than aslam_workspace_bytes()");
    }
    b->ws = (char *)d_workspace;
    b->ws_bytes = bytes;
    aslam_status st = ASLAM_OK;
    do {
        int dev = 0;
        cudaError_t ce = cudaGetDevice(&dev);
        if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (ce == cudaSuccess)
            ce = cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (ce != cudaSuccess) { st = cuda_fail(b, ce, "device query"); break; }

        const HostInfo &hi = b->hi;
        const Offsets &o = b->off;
        const int E = hi.E;
        Step2DParams &p = b->p;
        std::memset(&p, 0, sizeof(p));
        p.E = E;
        p.b_max = hi.b_max;
        p.n_spawn = cfg->n_spawn;
        p.flags = cfg->flags;
        p.reward_mode = cfg->reward_mode;
        p.hit_q = cfg->l_hit_q;
        p.miss_q = cfg->l_miss_q;
        p.clamp_q = cfg->l_clamp_q;
        p.t_episode = cfg->t_episode;
        p.Tmax = (int)lrintf((cfg->r_max_m / cfg->res_m) * 65536.0f);
        p.res = cfg->res_m;
        p.r_max = cfg->r_max_m;
        p.sigma = cfg->noise_sigma_m;
        p.r_min = cfg->r_min_m;
        p.dec_scale = range_scale(cfg->range_decimals);
        p.dt = cfg->dt_s;
        p.v_max = cfg->v_max;
        p.w_max = cfg->w_max;
        p.d_crash = cfg->d_crash;
        p.d_full = cfg->d_full;
        p.visit_cell = cfg->visit_cell_m;
        p.logodds_scale = cfg->logodds_scale;
        p.u_mode = cfg->u_mode;
        if (cfg->u_mode == ASLAM_U_SCANMATCH || cfg->u_mode == ASLAM_U_FIXEDLAG) {
            p.uq_K = cfg->uq_samples;
            p.uq_ds = cfg->uq_step_m > 0.0f ? cfg->uq_step_m : cfg->res_m;
            p.uq_inv_s2 = 1.0 / ((double)cfg->uq_range_sigma_m * cfg->uq_range_sigma_m);
            double qdet = 1.0;
            for (int i = 0; i < 3; ++i) {
                p.uq_q[i] = (double)cfg->uq_odo_sigma[i] * cfg->uq_odo_sigma[i];
                p.uq_prior[i] = (double)cfg->uq_prior_sigma[i] * cfg->uq_prior_sigma[i];
                qdet *= p.uq_q[i];
            }
            p.uq_scale = cfg->uq_u_scale > 0.0f ? (double)cfg->uq_u_scale : std::cbrt(qdet);
            p.pose_cov = at<double>(b, o.pose_cov);
            p.u_scan = at<float>(b, o.u_scan);
        }
        if (cfg->u_mode == ASLAM_U_FIXEDLAG) {
            p.slam_L = cfg->slam_window;
            p.slam_iters = cfg->slam_iters;
            p.csm_n_xy = cfg->csm_n_xy;
            p.csm_n_th = cfg->csm_n_th;
            p.csm_sep = cfg->csm_sep;
            p.csm_dth = cfg->csm_dth_rad;
            p.slam_weighted = cfg->slam_weighted_update;
            p.slam_gn_iters = cfg->slam_gn_iters;
            for (int q = 0; q < 3; ++q) {
                p.slam_meas_info[q] = cfg->slam_meas_info[q];
                p.slam_prior_info[q] = cfg->slam_prior_info[q];
                p.slam_wo[q] = 1.0 / ((double)cfg->uq_odo_sigma[q] * cfg->uq_odo_sigma[q]);
            }
            const size_t need = csm_map_layout(hi.W.data(), hi.H.data(), E, p.csm_n_xy, &p.csm_ws);
            p.csm_map_bytes = need <= 160 * 1024 ? need : 0;
            if (p.csm_map_bytes > 0) {
                ce = csm_set_smem(p.csm_map_bytes);
                if (ce != cudaSuccess) { st = cuda_fail(b, ce, "create: csm shared memory"); break; }
            }
            p.win_x = at<float>(b, o.win_x);
            p.win_odo = at<float>(b, o.win_odo);
            p.win_meas = at<float>(b, o.win_meas);
            p.win_minfo = at<float>(b, o.win_minfo);
            p.win_n = at<int>(b, o.win_n);
            p.slam_pred = at<float>(b, o.slam_pred);
            p.slam_odo = at<float>(b, o.slam_odo);
            p.csm_pose = at<float>(b, o.csm_pose);
            p.csm_match = at<float>(b, o.csm_match);
            p.csm_scores = at<long long>(b, o.csm_scores);
            p.slam_upd_w = at<float>(b, o.slam_upd_w);
            p.slam_gn_pose = cfg->slam_gn_iters > 0 ? at<float>(b, o.slam_gn_pose) : nullptr;
        }
        p.lam_col = (float)cfg->lam_col;
        p.lam_explore = (float)cfg->lam_explore;
        p.lam_abs = (float)cfg->lam_abs;
        p.lam_delta = (float)cfg->lam_delta;
        p.kappa = (float)cfg->kappa;
        p.u_hi = (float)cfg->u_hi;
        p.key = make_uint2((unsigned)cfg->seed, (unsigned)(cfg->seed >> 32));
        p.env_base = cfg->env_base;
        p.W = at<int>(b, o.W);
        p.H = at<int>(b, o.H);
        p.B = at<int>(b, o.B);
        p.Vw = at<int>(b, o.Vw);
        p.Vh = at<int>(b, o.Vh);
        p.R8 = at<int>(b, o.R8);
        p.Dd = at<int>(b, o.Dd);
        p.elev_cs = at<float2>(b, o.elev);
        p.dims = hi.dims;
        p.n_rings = hi.n_rings;
        p.Pz = cfg->dims == 3 ? (int)lrintf((cfg->sensor_z_m / cfg->res_m) * 65536.0f) : 0;
        p.order = at<int>(b, o.order);
        p.map_off = at<long long>(b, o.map_off);
        p.gtb_off = at<long long>(b, o.gtb_off);
        p.ray_off = at<long long>(b, o.ray_off);
        p.visit_off = at<long long>(b, o.visit_off);
        p.beam_cs = at<float2>(b, o.beam_cs);
        p.beam_df = soft_dirs(cfg) ? at<float4>(b, o.beam_df) : nullptr;
        p.lut = at<long long>(b, o.lut);
        p.gt_bits = at<unsigned>(b, o.gt_bits);
        p.x = at<float>(b, o.x);
        p.y = at<float>(b, o.y);
        p.th = at<float>(b, o.th);
        p.u_prev = at<float>(b, o.u_prev);
        p.t = at<int>(b, o.t);
        p.g = at<int>(b, o.g);
        p.ep = at<int>(b, o.ep);
        p.done = at<int>(b, o.done);
        p.Hq = at<long long>(b, o.Hq);
        p.belief = at<short>(b, o.belief);
        p.visit = at<int>(b, o.visit);
        p.spawn = at<float>(b, o.spawn);
        p.z = at<float>(b, o.z);
        const bool debug = (cfg->flags & ASLAM_FLAG_DEBUG) != 0;
        p.z_true = debug ? at<float>(b, o.z_true) : nullptr;
        p.hit = debug ? at<unsigned char>(b, o.hit) : nullptr;
        p.dbg_counts = debug ? at<unsigned>(b, o.dbg) : nullptr;
        p.ray_cells = at<long long>(b, o.ray_cells);
        p.gt_cells = at<long long>(b, o.gt_cells);
        p.terms = at<float>(b, o.terms);
        p.reward = at<float>(b, o.reward);
        p.far_cnt = at<unsigned>(b, o.far_cnt);
        p.far_bits = at<unsigned>(b, o.far_bits);
        p.ray_code = at<int>(b, o.ray_code);
        p.env_sense = at<void>(b, o.env_sense);
        // the smallest chunk; an env's later chunks must also start outside
        // its near block, so the kernel takes at least 2*R8 of the env.
        // Timed with the later chunks claimed per warp: a floor of 12 / 16 /
        // 20 cells -> step 0.1157 / 0.1164 / 0.1172 ms at 750 paper-scale
        // envs, 0.6410 / 0.6407 / 0.6421 ms at 4096 uneven envs
        p.chunk = 12;
        p.queue = at<unsigned>(b, o.queue);
        p.err = at<unsigned>(b, o.err);

        // Host-built tables: beam directions, entropy table, work order.
        std::vector<float2> cs((size_t)std::max<long long>(hi.ray_off[E], 1));
        std::vector<float4> df(soft_dirs(cfg) ? cs.size() : 0);
        const double two_pi = 2.0 * 3.14159265358979323846;
        const double fov = (double)cfg->fov_rad;
        const bool full_turn = fov <= 0.0 || fov >= two_pi - 1e-9;
        for (int e = 0; e < E; ++e) {
            // 2-D: B beams over the field of view; 3-D: rings x azimuths over a
            // full turn, beam b = ring * A + azimuth
            const int A = hi.B[e] / hi.n_rings;
            for (int k = 0; k < hi.B[e]; ++k) {
                double a;
                if (hi.dims == 3) a = (two_pi * (double)(k % A)) / (double)A;
                else if (full_turn) a = (two_pi * (double)k) / (double)A;
                else if (A == 1) a = 0.0;
                else a = -0.5 * fov + ((double)k * fov) / (double)(A - 1);
                cs[(size_t)hi.ray_off[e] + k] = make_float2((float)std::cos(a), (float)std::sin(a));
                if (soft_dirs(cfg)) {
                    // the soft range model of the in-step U walks the beam at
                    // its fp64 angle: (cos, sin) as hi + lo pairs of floats
                    const double ca = std::cos(a), sa = std::sin(a);
                    const float ch = (float)ca, sh = (float)sa;
                    df[(size_t)hi.ray_off[e] + k] = make_float4(ch, (float)(ca - (double)ch), sh,
                                                                (float)(sa - (double)sh));
                }
            }
        }
        std::vector<float2> elev((size_t)hi.n_rings);
        for (int r = 0; r < hi.n_rings; ++r) {
            const double lo = (double)cfg->elev_min_rad, hi_el = (double)cfg->elev_max_rad;
            const double el = hi.n_rings == 1 ? lo : lo + ((double)r * (hi_el - lo)) / (double)(hi.n_rings - 1);
            elev[(size_t)r] = make_float2((float)std::cos(el), (float)std::sin(el));
        }
        // Entropy of a cell with log-odds l = L * scale, in 2^-40 nats, by
        // the stable form h = l * q + log1p(e^-l), q = e^-l / (1 + e^-l).
        const int C = cfg->l_clamp_q;
        std::vector<long long> lut(2 * (size_t)C + 1);
        for (int L = -C; L <= C; ++L) {
            const double l = std::fabs((double)L * (double)cfg->logodds_scale);
            const double ex = std::exp(-l);
            const double h = l * (ex / (1.0 + ex)) + std::log1p(ex);
            lut[(size_t)(L + C)] = std::llrint(h * kLutScale);
        }
        // Longest-first work order: cost ~ beams x cells a beam can cross.
        b->order.resize(E);
        std::iota(b->order.begin(), b->order.end(), 0);
        std::vector<double> cost(E);
        const double rcell = (double)cfg->r_max_m / cfg->res_m;
        for (int e = 0; e < E; ++e)
            cost[e] = (double)std::max(hi.B[e], 1) *
                      std::min(rcell, std::sqrt((double)hi.W[e] * hi.W[e] + (double)hi.H[e] * hi.H[e] +
                                                (double)hi.D[e] * hi.D[e]));
        std::stable_sort(b->order.begin(), b->order.end(),
                         [&](int a, int c2) { return cost[a] > cost[c2]; });
        // sensing bundles of sense_block() beams, costliest envs first; an
        // env without beams still gets one (it integrates the env's action)
        std::vector<int2> bundles;
        p.sense_block = sense_block(hi.gt_words_max);
        for (int q = 0; q < E; ++q) {
            const int e = b->order[q];
            bundles.push_back(make_int2(e, 0));
            for (int b0 = p.sense_block; b0 < hi.B[e]; b0 += p.sense_block)
                bundles.push_back(make_int2(e, b0));
        }
        p.n_bundles = (int)bundles.size();
        p.bundles = at<int2>(b, o.bundles);

        auto h2d = [&](void *dst, const void *src, size_t n) {
            return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
        };
        std::vector<long long> src_off(h_gt_off, h_gt_off + E + 1);
        cudaError_t e1 = cudaSuccess;
        if (e1 == cudaSuccess) e1 = h2d((void *)p.W, hi.W.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess) e1 = h2d((void *)p.H, hi.H.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess) e1 = h2d((void *)p.B, hi.B.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess) e1 = h2d((void *)p.Vw, hi.Vw.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess) e1 = h2d((void *)p.Vh, hi.Vh.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess) e1 = h2d((void *)p.R8, hi.R8.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess) e1 = h2d((void *)p.Dd, hi.D.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess) e1 = h2d((void *)p.elev_cs, elev.data(), 8 * elev.size());
        if (e1 == cudaSuccess) e1 = h2d((void *)p.order, b->order.data(), 4 * (size_t)E);
        if (e1 == cudaSuccess && !bundles.empty())
            e1 = h2d((void *)p.bundles, bundles.data(), 8 * bundles.size());
        if (e1 == cudaSuccess) e1 = h2d((void *)p.map_off, hi.map_off.data(), 8 * (size_t)(E + 1));
        if (e1 == cudaSuccess) e1 = h2d((void *)p.gtb_off, hi.gtb_off.data(), 8 * (size_t)(E + 1));
        if (e1 == cudaSuccess) e1 = h2d((void *)p.ray_off, hi.ray_off.data(), 8 * (size_t)(E + 1));
        if (e1 == cudaSuccess) e1 = h2d((void *)p.visit_off, hi.visit_off.data(), 8 * (size_t)(E + 1));
        if (e1 == cudaSuccess) e1 = h2d(at<void>(b, o.src_off), src_off.data(), 8 * (size_t)(E + 1));
        if (e1 == cudaSuccess) e1 = h2d((void *)p.beam_cs, cs.data(), 8 * cs.size());
        if (e1 == cudaSuccess && !df.empty()) e1 = h2d((void *)p.beam_df, df.data(), 16 * df.size());
        if (e1 == cudaSuccess) e1 = h2d((void *)p.lut, lut.data(), 8 * lut.size());
        if (e1 == cudaSuccess)
            e1 = cudaMemcpyAsync((void *)p.spawn, d_spawn, 12 * (size_t)E * cfg->n_spawn,
                                 cudaMemcpyDeviceToDevice, s);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(p.err, 0, 4, s);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(p.queue, 0, 16, s);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(at<void>(b, o.tune_actions), 0, 8 * (size_t)E, s);
        if (e1 == cudaSuccess)
            e1 = launch_pack_gt(d_gt, at<long long>(b, o.src_off), p.W, p.H, p.Dd, p.gtb_off,
                                (unsigned *)p.gt_bits, E, s);
        if (e1 != cudaSuccess) { st = cuda_fail(b, e1, "create: upload"); break; }
        st = reset_all(b, s);
        if (st != ASLAM_OK) break;
        const int block = cfg->threads_per_cta ? cfg->threads_per_cta : default_block(hi);
        const int S = cfg->window_cells ? cfg->window_cells
                                         : auto_window(hi, b->smem_optin, cfg->l_clamp_q, block);
        st = configure_launch(b, block, S);
        if (st != ASLAM_OK) break;
        ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { st = cuda_fail(b, ce, "create: synchronize"); break; }
    } while (0);
    if (st != ASLAM_OK) {
        g_thread_error = b->err;
        delete b;
        return st;
    }
    *out = b;
    return ASLAM_OK;
}

aslam_status aslam_step_fused(aslam_batch *b, const float *d_actions, const float *d_u,
                              float *d_reward, float *d_obs, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    if (!d_actions) return fail_b(b, ASLAM_ERR_INVALID_ARG, "d_actions is NULL");
    Step2DParams p = b->p;
    p.actions = d_actions;
    p.u_in = d_u;
    p.out_reward = d_reward;
    p.out_obs = d_obs;
    const cudaEvent_t *ev = nullptr;
    if (b->prof_n < b->prof_cap) {
        ev = &b->prof_ev[(size_t)b->prof_n * (step_kernels(b) + 1)];
        ++b->prof_n;
    }
    if (b->hi.dims == 3)
        CK(launch_step3d(p, b->grid, b->block, b->smem, (cudaStream_t)stream, ev), "aslam_step");
    else
        CK(launch_step2d(p, b->grid, b->block, b->smem, (cudaStream_t)stream, ev), "aslam_step");
    return ASLAM_OK;
}

aslam_status aslam_step(aslam_batch *b, const float *d_actions, const float *d_u, void *stream) {
    return aslam_step_fused(b, d_actions, d_u, nullptr, nullptr, stream);
}

// The device address of page-locked host memory (mapped into the device's
// address space), or NULL for any other host memory.
static float *mapped_host(const float *h) {
    if (!h) return nullptr;
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, const_cast<float *>(h), 0) != cudaSuccess) {
        (void)cudaGetLastError();        // not page-locked: not an error of this call
        return nullptr;
    }
    return static_cast<float *>(d);
}

aslam_status aslam_step_host(aslam_batch *b, const float *h_actions, const float *h_u,
                             float *h_reward, float *h_obs, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    if (!h_actions) return fail_b(b, ASLAM_ERR_INVALID_ARG, "h_actions is NULL");
    const size_t E = (size_t)b->hi.E;
    const cudaStream_t s = (cudaStream_t)stream;
    float *d_in = at<float>(b, b->off.io_in);
    float *d_out = at<float>(b, b->off.io_out);
    // Page-locked buffers are read and written by the kernels in place (over
    // NVLink-C2C on a Grace-Blackwell node): the inputs by one thread per
    // sensing CTA and the finishing warp, the outputs as each kernel produces
    // them, so no copy sits before or after the step.  Any other host memory
    // goes through the workspace's staging arrays with copies.
    const float *d_act = mapped_host(h_actions);
    if (!d_act) {
        CK(cudaMemcpyAsync(d_in, h_actions, 8 * E, cudaMemcpyHostToDevice, s), "aslam_step_host: actions");
        d_act = d_in;
    }
    const float *d_u = mapped_host(h_u);
    if (h_u && !d_u) {
        CK(cudaMemcpyAsync(d_in + 2 * E, h_u, 4 * E, cudaMemcpyHostToDevice, s), "aslam_step_host: U");
        d_u = d_in + 2 * E;
    }
    float *m_reward = mapped_host(h_reward), *m_obs = mapped_host(h_obs);
    const aslam_status st =
        aslam_step_fused(b, d_act, d_u, h_reward ? (m_reward ? m_reward : d_out) : nullptr,
                         h_obs ? (m_obs ? m_obs : d_out + E) : nullptr, stream);
    if (st != ASLAM_OK) return st;
    if (h_reward && !m_reward)
        CK(cudaMemcpyAsync(h_reward, d_out, 4 * E, cudaMemcpyDeviceToHost, s), "aslam_step_host: reward");
    if (h_obs && !m_obs)
        CK(cudaMemcpyAsync(h_obs, d_out + E, 4 * E * ((size_t)b->hi.b_max + 2), cudaMemcpyDeviceToHost, s),
           "aslam_step_host: obs");
    return ASLAM_OK;
}

aslam_status aslam_reward(aslam_batch *b, float *d_reward, void *stream) {
    if (!b || !d_reward) return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL argument");
    CK(launch_gather_reward(b->p, d_reward, (cudaStream_t)stream), "aslam_reward");
    return ASLAM_OK;
}

aslam_status aslam_reward_terms(aslam_batch *b, float *d_terms, void *stream) {
    if (!b || !d_terms) return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL argument");
    CK(cudaMemcpyAsync(d_terms, b->p.terms, 4 * (size_t)b->hi.E * kTerms,
                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "aslam_reward_terms");
    return ASLAM_OK;
}

aslam_status aslam_observe(aslam_batch *b, float *d_obs, void *stream) {
    if (!b || !d_obs) return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL argument");
    CK(launch_gather_obs(b->p, d_obs, (cudaStream_t)stream), "aslam_observe");
    return ASLAM_OK;
}

aslam_status aslam_reset(aslam_batch *b, const uint8_t *d_mask, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    CK(launch_mark_done(b->p.done, d_mask, b->hi.E, (cudaStream_t)stream), "aslam_reset");
    return ASLAM_OK;
}

aslam_status aslam_get_state(aslam_batch *b, aslam_state_ptrs *o) {
    if (!b || !o) return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL argument");
    const Step2DParams &p = b->p;
    o->x = p.x;
    o->y = p.y;
    o->th = p.th;
    o->u_prev = p.u_prev;
    o->t = p.t;
    o->g = p.g;
    o->ep = p.ep;
    o->done = p.done;
    o->belief = p.belief;
    o->z = p.z;
    o->z_true = p.z_true;
    o->hit = p.hit;
    o->counts = p.dbg_counts;
    o->ray_cells = reinterpret_cast<int64_t *>(p.ray_cells);
    o->gt_cells = reinterpret_cast<int64_t *>(p.gt_cells);
    o->terms = p.terms;
    o->h_map_off = reinterpret_cast<const int64_t *>(b->hi.map_off.data());
    o->h_ray_off = reinterpret_cast<const int64_t *>(b->hi.ray_off.data());
    o->b_max = b->hi.b_max;
    o->pose_cov = p.pose_cov;
    o->slam_window = p.win_x;
    o->slam_count = p.win_n;
    o->slam_match = p.csm_match;
    o->slam_scores = reinterpret_cast<int64_t *>(p.csm_scores);
    o->slam_match_pose = p.csm_pose;
    o->slam_gn_pose = p.slam_gn_pose;
    return ASLAM_OK;
}

aslam_status aslam_sync_status(aslam_batch *b, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, b->p.err, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream), "status read");
    CK(cudaStreamSynchronize((cudaStream_t)stream), "status synchronize");
    if (h & kErrChecks) return fail_b(b, ASLAM_ERR_DEVICE, "a device-side check failed");
    return ASLAM_OK;
}

aslam_status aslam_capture_graph(aslam_batch *b, const float *d_actions, const float *d_u,
                                 float *d_reward, float *d_obs, void *stream) {
    if (!b || !d_actions) return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return fail_b(b, ASLAM_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    Step2DParams p = b->p;
    p.actions = d_actions;
    p.u_in = d_u;
    p.out_reward = d_reward;
    p.out_obs = d_obs;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t le = b->hi.dims == 3 ? launch_step3d(p, b->grid, b->block, b->smem, s)
                                     : launch_step2d(p, b->grid, b->block, b->smem, s);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(s, &g);
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(b, le, "capture launch"); }
    if (ee != cudaSuccess) return cuda_fail(b, ee, "end capture");
    b->graph = g;
    CK(cudaGraphInstantiate(&b->gexec, g, 0), "graph instantiate");
    return ASLAM_OK;
}

aslam_status aslam_graph_step(aslam_batch *b, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    if (!b->gexec) return fail_b(b, ASLAM_ERR_STATE, "no captured graph");
    CK(cudaGraphLaunch(b->gexec, (cudaStream_t)stream), "graph launch");
    return ASLAM_OK;
}

aslam_status aslam_autotune(aslam_batch *b, int32_t *h_best, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int b_max = b->hi.b_max;
    std::vector<int> blocks, windows;
    for (int t : {128, 256, 384, 512, 768, 1024})
        if (t >= 64 && (t <= 1024)) blocks.push_back(t);
    // the largest window of each block size (its chunk list grows with the block)
    for (int blk : blocks) {
        const int Sa = auto_window(b->hi, b->smem_optin, b->p.clamp_q, blk);
        for (int S : {Sa, 320, 256, 224, 192, 160, 128})
            if (S <= Sa && std::find(windows.begin(), windows.end(), S) == windows.end()) windows.push_back(S);
    }
    std::sort(windows.begin(), windows.end(), std::greater<int>());
    if (b->hi.dims == 3) {
        windows.assign(1, 0);
        blocks.assign({256, 512, 1024});
    }
    (void)b_max;
    const int keep_block = b->block, keep_window = b->window;
    float best_ms = 1e30f;
    int best_block = keep_block, best_window = keep_window;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const float *acts = at<float>(b, b->off.tune_actions);
    aslam_status st = ASLAM_OK;
    for (int S : windows) {
        for (int blk : blocks) {
            if (configure_launch(b, blk, S) != ASLAM_OK) continue;
            st = reset_all(b, s);
            if (st != ASLAM_OK) break;
            Step2DParams p = b->p;
            p.actions = acts;
            auto launch = [&]() {
                return b->hi.dims == 3 ? launch_step3d(p, b->grid, b->block, b->smem, s)
                                       : launch_step2d(p, b->grid, b->block, b->smem, s);
            };
            cudaError_t ce = launch();
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
            for (int r = 0; r < 3 && ce == cudaSuccess; ++r) ce = launch();
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess) { st = cuda_fail(b, ce, "autotune"); break; }
            if (ms < best_ms) { best_ms = ms; best_block = blk; best_window = S; }
        }
        if (st != ASLAM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != ASLAM_OK) return st;
    st = configure_launch(b, best_block, best_window);
    if (st != ASLAM_OK) return st;
    st = reset_all(b, s);
    if (st != ASLAM_OK) return st;
    CK(cudaStreamSynchronize(s), "autotune synchronize");
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (h_best) { h_best[0] = best_block; h_best[1] = best_window; }
    return ASLAM_OK;
}

}  // extern "C"

namespace {
struct Region { void *ptr; size_t bytes; };
std::vector<Region> state_regions(aslam_batch *b) {
    const Step2DParams &p = b->p;
    const size_t E = b->hi.E;
    std::vector<Region> r = {{p.x, 4 * E}, {p.y, 4 * E}, {p.th, 4 * E}, {p.u_prev, 4 * E},
                             {p.t, 4 * E}, {p.g, 4 * E}, {p.ep, 4 * E}, {p.done, 4 * E},
                             {p.Hq, 8 * E}, {p.belief, 2 * (size_t)b->hi.map_off[E]},
                             {p.visit, 4 * (size_t)b->hi.visit_off[E]}};
    if (p.pose_cov) r.push_back({p.pose_cov, 48 * E});
    if (p.win_n) {
        const size_t w = 12 * E * (size_t)p.slam_L;
        r.push_back({p.win_x, w});
        r.push_back({p.win_odo, w});
        r.push_back({p.win_meas, w});
        r.push_back({p.win_minfo, w});
        r.push_back({p.win_n, 4 * E});
    }
    return r;
}
}  // namespace

extern "C" {

aslam_status aslam_state_bytes(aslam_batch *b, size_t *bytes) {
    if (!b || !bytes) return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL argument");
    size_t n = 0;
    for (const Region &r : state_regions(b)) n += r.bytes;
    *bytes = n;
    return ASLAM_OK;
}

aslam_status aslam_save_state(aslam_batch *b, void *h_buf, size_t bytes, void *stream) {
    size_t need = 0;
    aslam_status st = aslam_state_bytes(b, &need);
    if (st != ASLAM_OK) return st;
    if (!h_buf || bytes < need) return fail_b(b, ASLAM_ERR_INVALID_ARG, "state buffer too small");
    char *dst = (char *)h_buf;
    for (const Region &r : state_regions(b)) {
        CK(cudaMemcpyAsync(dst, r.ptr, r.bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream), "save");
        dst += r.bytes;
    }
    CK(cudaStreamSynchronize((cudaStream_t)stream), "save synchronize");
    return ASLAM_OK;
}

aslam_status aslam_load_state(aslam_batch *b, const void *h_buf, size_t bytes, void *stream) {
    size_t need = 0;
    aslam_status st = aslam_state_bytes(b, &need);
    if (st != ASLAM_OK) return st;
    if (!h_buf || bytes < need) return fail_b(b, ASLAM_ERR_INVALID_ARG, "state buffer too small");
    const char *src = (const char *)h_buf;
    for (const Region &r : state_regions(b)) {
        CK(cudaMemcpyAsync(r.ptr, src, r.bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream), "load");
        src += r.bytes;
    }
    CK(cudaStreamSynchronize((cudaStream_t)stream), "load synchronize");
    return ASLAM_OK;
}

aslam_status aslam_flgn_config_init(aslam_flgn_config *c) {
    if (!c) return ASLAM_ERR_INVALID_ARG;
    c->struct_size = sizeof(aslam_flgn_config);
    c->n_envs = 1;
    c->window = 8;
    c->iters = 3;
    for (int q = 0; q < 3; ++q) c->odo_info[q] = 1.0f / (0.01f * 0.01f);
    c->u_scale = 1e-4f;
    return ASLAM_OK;
}

aslam_status aslam_fixed_lag_gn(const aslam_flgn_config *c, float *d_x, const float *d_odo,
                                const float *d_meas, const float *d_meas_info,
                                const float *d_prior, const float *d_prior_info, float *d_cov,
                                float *d_u, int32_t *d_status, void *stream) {
    auto fail = [](const char *m) {
        set_thread_error(m);
        return ASLAM_ERR_INVALID_ARG;
    };
    if (!c || c->struct_size != sizeof(aslam_flgn_config)) return fail("flgn config NULL or struct_size mismatch");
    if (c->n_envs < 1) return fail("n_envs must be >= 1");
    if (c->window < 1 || c->window > flgn_max_window()) return fail("window out of [1, 16]");
    if (c->iters < 0 || c->iters > 20) return fail("iters out of [0, 20]");
    for (int q = 0; q < 3; ++q)
        if (!(c->odo_info[q] > 0.0f)) return fail("odo_info must be > 0");
    if (!(c->u_scale > 0.0f)) return fail("u_scale must be > 0");
    if (!d_x || !d_meas || !d_meas_info || !d_prior || !d_prior_info || (c->window > 1 && !d_odo))
        return fail("NULL pointer argument");
    cudaError_t e = launch_flgn(c->n_envs, c->window, c->iters, c->odo_info, c->u_scale, d_x,
                                d_odo, d_meas, d_meas_info, d_prior, d_prior_info, d_cov, d_u,
                                d_status, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return ASLAM_ERR_CUDA;
    }
    return ASLAM_OK;
}

aslam_status aslam_csm_config_init(aslam_csm_config *c) {
    if (!c) return ASLAM_ERR_INVALID_ARG;
    c->struct_size = sizeof(aslam_csm_config);
    c->n_xy = 5;
    c->n_th = 5;
    c->sep = 1;
    c->dth_rad = 0.01f;
    return ASLAM_OK;
}

aslam_status aslam_csm(aslam_batch *b, const aslam_csm_config *c, const float *d_pose_pred,
                       const float *d_ranges, float *d_pose_out, float *d_match,
                       int64_t *d_scores, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    if (!c || c->struct_size != sizeof(aslam_csm_config))
        return fail_b(b, ASLAM_ERR_INVALID_ARG, "csm config NULL or struct_size mismatch");
    if (b->hi.dims != 2) return fail_b(b, ASLAM_ERR_INVALID_ARG, "aslam_csm needs a 2-D batch");
    if (c->n_xy < 0 || c->n_xy > csm_max_n() || c->n_th < 0 || c->n_th > csm_max_n())
        return fail_b(b, ASLAM_ERR_INVALID_ARG, "n_xy and n_th must be in [0, 8]");
    if (c->sep < 0 || !(c->dth_rad > 0.0f))
        return fail_b(b, ASLAM_ERR_INVALID_ARG, "need sep >= 0 and dth_rad > 0");
    if (!d_pose_pred || !d_pose_out || !d_match || !d_scores)
        return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL pointer argument");
    // stage the evidence maps in shared memory when the largest one fits
    if (b->csm_n != c->n_xy) {
        b->csm_bytes = csm_map_layout(b->hi.W.data(), b->hi.H.data(), b->hi.E, c->n_xy, &b->csm_ws);
        b->csm_n = c->n_xy;
    }
    const int ws = b->csm_ws;
    const size_t budget = 160 * 1024;
    const size_t map_bytes = b->csm_bytes <= budget ? b->csm_bytes : 0;
    if (map_bytes > 0) CK(csm_set_smem(map_bytes), "aslam_csm: shared memory");
    CK(launch_csm2d(b->p, c->n_xy, c->n_th, c->sep, c->dth_rad, map_bytes, ws, d_pose_pred,
                    d_ranges ? d_ranges : b->p.z, d_pose_out, d_match,
                    reinterpret_cast<long long *>(d_scores), false, (cudaStream_t)stream),
       "aslam_csm");
    return ASLAM_OK;
}

aslam_status aslam_bridge_u(aslam_batch *b, const float *d_u_old, const float *d_u_new, int64_t t,
                            int64_t t_bridge, float *d_u_out, float *d_obs, void *stream) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    if (!d_u_old || !d_u_new) return fail_b(b, ASLAM_ERR_INVALID_ARG, "d_u_old / d_u_new is NULL");
    if (!d_u_out && !d_obs) return fail_b(b, ASLAM_ERR_INVALID_ARG, "no output (d_u_out, d_obs)");
    if (t < 0 || t_bridge < 1) return fail_b(b, ASLAM_ERR_INVALID_ARG, "need t >= 0 and t_bridge >= 1");
    // alpha_t = min(1, t / T_bridge) (Eq. 21), in fp64, rounded once to fp32
    const double a = (double)t / (double)t_bridge;
    const float alpha = (float)(a < 1.0 ? a : 1.0);
    CK(launch_bridge_u(d_u_old, d_u_new, alpha, b->hi.E, d_u_out, d_obs, b->hi.b_max + 2,
                       b->hi.b_max + 1, (cudaStream_t)stream), "aslam_bridge_u");
    return ASLAM_OK;
}

aslam_status aslam_profile_begin(aslam_batch *b, int32_t max_steps) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    if (max_steps < 1 || max_steps > (1 << 20))
        return fail_b(b, ASLAM_ERR_INVALID_ARG, "max_steps must be in [1, 2^20]");
    release_profile(b);
    const size_t n = (size_t)max_steps * (step_kernels(b) + 1);
    b->prof_ev.reserve(n);
    for (size_t i = 0; i < n; ++i) {
        cudaEvent_t e;
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) {
            release_profile(b);
            return cuda_fail(b, ce, "aslam_profile_begin");
        }
        b->prof_ev.push_back(e);
    }
    b->prof_cap = max_steps;
    return ASLAM_OK;
}

aslam_status aslam_profile_end(aslam_batch *b, double *h_ms, int32_t *h_n_kernels,
                               int32_t *h_n_steps) {
    if (!b) return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "batch is NULL");
    if (!h_ms || !h_n_kernels || !h_n_steps) return fail_b(b, ASLAM_ERR_INVALID_ARG, "NULL argument");
    if (b->prof_cap == 0) return fail_b(b, ASLAM_ERR_STATE, "no aslam_profile_begin");
    const int nk = step_kernels(b);
    for (int k = 0; k < ASLAM_MAX_STEP_KERNELS; ++k) h_ms[k] = 0.0;
    aslam_status st = ASLAM_OK;
    if (b->prof_n > 0) {
        cudaError_t ce = cudaEventSynchronize(b->prof_ev[(size_t)b->prof_n * (nk + 1) - 1]);
        for (int i = 0; i < b->prof_n && ce == cudaSuccess; ++i) {
            const cudaEvent_t *ev = &b->prof_ev[(size_t)i * (nk + 1)];
            for (int k = 0; k < nk && ce == cudaSuccess; ++k) {
                float ms = 0.0f;
                ce = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
                h_ms[k] += ms;
            }
        }
        if (ce != cudaSuccess) st = cuda_fail(b, ce, "aslam_profile_end");
    }
    *h_n_kernels = nk;
    *h_n_steps = b->prof_n;
    release_profile(b);
    return st;
}

const char *aslam_kernel_name(const aslam_batch *b, int32_t k) {
    static const char *const k2[] = {"sense2d_kernel", "update2d_kernel"};
    static const char *const k2u[] = {"sense2d_kernel", "uq2d_kernel", "update2d_kernel"};
    if (!b || k < 0) return nullptr;
    if (b->hi.dims == 3) return k == 0 ? "step3d_kernel" : nullptr;
    static const char *const k2s[] = {"sense2d_kernel",
                                      "slam_predict2d_kernel", "csm2d_kernel",
                                      "slam_window2d_kernel", "slam_replan2d_kernel",
                                      "update2d_kernel"};
    static const char *const k2g[] = {"sense2d_kernel",
                                      "slam_predict2d_kernel", "csm2d_kernel",
                                      "slam_correct2d_kernel", "slam_window2d_kernel",
                                      "slam_replan2d_kernel", "update2d_kernel"};
    if (b->p.u_mode == ASLAM_U_SCANMATCH) return k < kStep2DKernels + 1 ? k2u[k] : nullptr;
    if (b->p.u_mode == ASLAM_U_FIXEDLAG && b->p.slam_gn_iters > 0)
        return k < kStep2DKernels + 5 ? k2g[k] : nullptr;
    if (b->p.u_mode == ASLAM_U_FIXEDLAG) return k < kStep2DKernels + 4 ? k2s[k] : nullptr;
    return k < kStep2DKernels ? k2[k] : nullptr;
}

void aslam_destroy_batch(aslam_batch *b) {
    if (!b) return;
    release_profile(b);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

const char *aslam_status_string(aslam_status s) {
    switch (s) {
        case ASLAM_OK: return "ok";
        case ASLAM_ERR_INVALID_ARG: return "invalid argument";
        case ASLAM_ERR_CUDA: return "CUDA error";
        case ASLAM_ERR_WORKSPACE: return "workspace error";
        case ASLAM_ERR_TIMEOUT: return "reserved (no device waits in this build)";
        case ASLAM_ERR_STATE: return "invalid state";
        case ASLAM_ERR_UNSUPPORTED: return "unsupported";
        case ASLAM_ERR_DEVICE: return "device-side check failed";
    }
    return "unknown status";
}

const char *aslam_last_error(const aslam_batch *b) {
    if (b) return b->err.c_str();
    return g_thread_error.c_str();
}

aslam_status aslam_debug_detmath(const float *d_x, const float *d_u, int32_t n, float *d_sin,
                                 float *d_cos, float *d_log, float *d_cos2pi, uint64_t seed,
                                 float *d_gauss, void *stream) {
    aslam_batch *b = nullptr;
    if (n < 0 || (n > 0 && (!d_x || !d_u || !d_sin || !d_cos || !d_log || !d_cos2pi || !d_gauss)))
        return fail_b(nullptr, ASLAM_ERR_INVALID_ARG, "bad detmath arguments");
    if (n == 0) return ASLAM_OK;
    CK(launch_detmath(d_x, d_u, n, d_sin, d_cos, d_log, d_cos2pi,
                      make_uint2((unsigned)seed, (unsigned)(seed >> 32)), d_gauss,
                      (cudaStream_t)stream), "detmath");
    return ASLAM_OK;
}

}  // extern "C"
