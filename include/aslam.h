/*
 * aslam.h -- C ABI of libaslam, the GB300 (sm_103a) batched Active-SLAM
 * environment step of "Massive Parallel Deep Reinforcement Learning for
 * Active SLAM" (arXiv 2603.25834).
 *
 * One call advances E independent robots by one control period: action
 * integration (Eq. 4, Sec. IV-A robot), LiDAR raycasting into each robot's
 * ground-truth world (Sec. IV-A sensor), the inverse-sensor log-odds update
 * of each robot's occupancy grid (Sec. III-D), and the per-environment
 * reward (Sec. III-E, Eq. 7-17; or the map-entropy information gain, Table I
 * "Map entropy") and observation (Eq. 3).  A differentiable soft-range
 * raycaster with its adjoint and a batched scan-to-map Gauss-Newton pose
 * correction (Sec. III-D, Eq. 5-6) sit beside the step.
 *
 * Conventions shared by every call:
 *   - Device pointers ("d_") are CUDA global-memory addresses on the current
 *     device; host pointers ("h_") are ordinary process memory.  The caller
 *     owns every buffer it passes; the library never allocates device
 *     memory (no cudaMalloc) and keeps no pointer to caller buffers beyond
 *     the call, except the workspace given to aslam_create_batch.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Every call is stream-ordered and asynchronous unless stated.
 *   - Argument errors are detected before any launch and leave device state
 *     untouched; the call returns a non-zero status and aslam_last_error()
 *     gives a message.  Device-side failures set a sticky error word that the
 *     next aslam_sync_status() returns.
 *   - A batch is thread-compatible, not thread-safe: calls on one batch must
 *     not overlap in time from several host threads.
 *
 * Grid conventions (both dims): cell (i, j) covers [i*res, (i+1)*res) x
 * [j*res, (j+1)*res) in metres, flat index j*W + i (3-D: (k*H + j)*W + i);
 * a ground-truth byte != 0 is occupied.  Beam b of B over a full turn sits
 * at angle th + b*2*pi/B; over a front arc of width fov at th - fov/2 +
 * b*fov/(B-1).  Log-odds are int16 in units of logodds_scale (1/1024).
 */
#ifndef ASLAM_H
#define ASLAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aslam_batch aslam_batch;   /* opaque host-side handle */

typedef enum {
    ASLAM_OK = 0,
    ASLAM_ERR_INVALID_ARG = 1,   /* a size, pointer or value is out of range */
    ASLAM_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    ASLAM_ERR_WORKSPACE = 3,     /* workspace missing, misaligned or too small */
    ASLAM_ERR_TIMEOUT = 4,       /* reserved: no kernel of this build waits on another */
    ASLAM_ERR_STATE = 5,         /* call not valid in the batch's current state */
    ASLAM_ERR_UNSUPPORTED = 6,   /* valid request this build does not support */
    ASLAM_ERR_DEVICE = 7         /* a device-side check failed (sticky error word) */
} aslam_status;

/* Config flags. */
#define ASLAM_FLAG_DEBUG   0x1   /* keep per-beam true ranges/hit flags and per-cell counts */
/* Device-side consistency checks: every grid index of the 2-D sensing and
 * update walks is checked before the access (a failed check skips it), and
 * non-finite actions or U_t are reported.  A failed check sets the batch's
 * sticky error word (aslam_sync_status -> ASLAM_ERR_DEVICE); no kernel traps.
 * Results are unchanged when every check passes; the checked walks are slower. */
#define ASLAM_FLAG_CHECKS  0x2

/* Reward selection (aslam_reward). */
#define ASLAM_REWARD_ENTROPY   0  /* H_{t-1} - H_t of the robot's map, nats */
#define ASLAM_REWARD_COMPOSITE 1  /* Eq. 7 */

/* Per-env reward terms written by aslam_reward_terms, [E, ASLAM_N_TERMS] fp32. */
#define ASLAM_N_TERMS 12
/* 0 dH = H_{t-1} - H_t   1 dcells (Eq. 9)    2 I (Eq. 10)     3 alpha_hug (Eq. 15)
 * 4 R_explore* (Eq. 16)  5 R_abs (Eq. 13)    6 R_delta* (Eq. 17)
 * 7 R_t (Eq. 7)          8 collision (0/1)   9 d_min of the measured ranges
 * 10 d_min of the noise-free ranges          11 H_t (nats) */

#define ASLAM_CONFIG_VERSION 2u

/*
 * Batch configuration (POD).  Fill with aslam_config_init() and override.
 * The defaults are the values the paper fixes (Sec. IV-A: sigma = 0.01 m,
 * d_crash = 0.15 m, T_episode = 2048; dt = 0.1 s from "3000 timesteps (5
 * minutes)") and, where the paper leaves a value open, documented choices.
 */
typedef struct {
    uint32_t struct_size;          /* sizeof(aslam_config) */
    uint32_t version;              /* ASLAM_CONFIG_VERSION */
    int32_t n_envs;                /* E >= 1 */
    int32_t dims;                  /* 2: planar grids; 3: voxel volumes (fields at the end) */
    int32_t n_spawn;               /* spawn poses per env, >= 1 */
    int32_t reward_mode;           /* ASLAM_REWARD_* */
    const int32_t *h_map_w;        /* HOST [E]: grid width W (cells), >= 1 */
    const int32_t *h_map_h;        /* HOST [E]: grid height H (cells), >= 1 */
    const int32_t *h_n_beams;      /* HOST [E]: beams B, 0..ASLAM_MAX_BEAMS */
    float res_m;                   /* cell size (m) */
    float r_max_m;                 /* max range (m) */
    float fov_rad;                 /* 0 or >= 2*pi: full turn; else front arc */
    float noise_sigma_m;           /* range noise std (m) */
    float dt_s;                    /* control period (s) */
    float v_max;                   /* |v| clamp, v in [0, v_max] (m/s) */
    float w_max;                   /* w in [-w_max, w_max] (rad/s) */
    float d_crash;                 /* collision distance (m) */
    float d_full;                  /* Eq. 15 full-clearance distance (m) */
    float visit_cell_m;            /* Eq. 9 workspace cell size (m) */
    int32_t l_hit_q;               /* hit increment, logodds_scale units (870) */
    int32_t l_miss_q;              /* miss increment (-410) */
    int32_t l_clamp_q;             /* |L| clamp (3584) */
    int32_t t_episode;             /* episode length in steps */
    float logodds_scale;           /* log-odds per int16 unit (1/1024) */
    int32_t threads_per_cta;       /* 0 = library default / autotuned */
    double lam_col, lam_explore, lam_abs, lam_delta, kappa, u_hi;   /* Eq. 7-17 */
    uint64_t seed;                 /* noise stream key (Philox4x32-10) */
    int32_t flags;                 /* ASLAM_FLAG_* */
    int32_t window_cells;          /* side of the shared-memory counter window; 0 = auto */
    /* 3-D voxel variant (dims = 3): W x H x D voxels, a multi-ring LiDAR of
     * n_rings elevations evenly spaced over [elev_min, elev_max] (both ends
     * included) times h_n_beams[e] azimuths over a full turn, mounted at
     * sensor_z_m; beam index b = ring * azimuths + azimuth.  W must be a
     * multiple of 8.  Ignored for dims = 2. */
    const int32_t *h_map_d;        /* HOST [E]: depth D (voxels) */
    int32_t n_rings;
    float sensor_z_m, elev_min_rad, elev_max_rad;
    /* Global index of env 0 (>= 0, env_base + n_envs <= 2^31 - 1): the
     * range-noise counter of env e is env_base + e, so a batch holding envs
     * [lo, hi) of a larger set, created with env_base = lo, draws the same
     * noise as those envs do in one batch of the whole set (default 0). */
    int32_t env_base;
    /* Sensor quantisation of Sec. IV-A (0.1 m minimum range, ranges
     * reported to 0.01 m).  A returned beam's measured range is
     * z = clip(round(z_true + sigma*n, range_decimals), r_min_m, r_max_m),
     * the rounding done as rint(z * 10^d) / 10^d in fp32 (half to even);
     * range_decimals = -1 (default) skips it, r_min_m = 0 (default) clips
     * at 0.  A beam with no return reports r_max_m unrounded. */
    float r_min_m;                 /* 0 <= r_min_m <= r_max_m */
    int32_t range_decimals;        /* -1 (off) or 0..6 */
    /* In-step pose uncertainty (Sec. III-D, Eq. 5-6), 2-D only.  With
     * u_mode = ASLAM_U_SCANMATCH the step computes U_t itself (the caller's
     * d_u is ignored): the scan-match information of the soft expected-range
     * model on the map before this scan, A = sum_b J_b J_b^T / sigma_r^2
     * (J_b = d r_b / d(x, y, th) at the robot's pose; uq_samples samples of
     * uq_step_m), is fused with the previous pose covariance propagated by
     * one step of odometry noise Q = diag(uq_odo_sigma^2):
     * Sigma_t = ((Sigma_{t-1} + Q)^-1 + A)^-1, Sigma = diag(uq_prior_sigma^2)
     * after a reset; U_t = det(Sigma_t)^(1/3) / uq_u_scale (0: det(Q)^(1/3)).
     * U_t then enters the reward (Eq. 7-17) and the observation (Eq. 3). */
    int32_t u_mode;                /* ASLAM_U_CALLER (default) or ASLAM_U_SCANMATCH */
    int32_t uq_samples;            /* 1 .. ASLAM_SOFT_MAX_SAMPLES (default 64) */
    float uq_step_m;               /* >= 0; 0 = res_m */
    float uq_range_sigma_m;        /* > 0 (default 0.01) */
    float uq_odo_sigma[3];         /* > 0: x, y (m), theta (rad) per step (default 0.01) */
    float uq_prior_sigma[3];       /* > 0 (default 0.01) */
    float uq_u_scale;              /* >= 0 (default 0) */
    /* The SLAM backbone in the step (u_mode = ASLAM_U_FIXEDLAG, 2-D only;
     * Sec. III-D).  Each step: the pose predicted from the window's newest
     * estimate and this step's odometry (v dt, 0, w dt) is matched against
     * the map before this scan (aslam_csm with the csm_* parameters); the
     * match enters a sliding window of slam_window poses as a pose factor of
     * information w * slam_meas_info, the odometry as a factor of
     * information 1 / uq_odo_sigma^2, and the oldest pose is anchored at its
     * current estimate with slam_prior_info; slam_iters Gauss-Newton steps
     * (aslam_fixed_lag_gn) give the newest pose's marginal covariance Sigma_t
     * and U_t = det(Sigma_t)^(1/3) / (uq_u_scale or det(Q)^(1/3)).  An env's
     * window restarts at its reset; its first scan adds no pose factor.  With
     * slam_weighted_update = 1 the scan's log-odds increments are scaled by
     * the normalised match score s (1 for an episode's first scan):
     * L' = clamp(L + rint(s * (h*HIT + m*MISS))) (fp32).  After the
     * optimisation the aligned scan is integrated: every beam's measured
     * range is walked from the window's newest optimised pose (its heading
     * rotating the beams), not from the sensing pose; ray_cells counts those
     * walks.  The sensing pose stays the robot's state (motion, collision,
     * visit grid). */
    int32_t slam_window;           /* 1 .. 16 (default 8) */
    int32_t slam_iters;            /* 0 .. 20 (default 3) */
    int32_t csm_n_xy, csm_n_th;    /* 0 .. 8 (default 5, 5) */
    int32_t csm_sep;               /* >= 0 (default 1) */
    float csm_dth_rad;             /* > 0 (default 0.01) */
    float slam_meas_info[3];       /* > 0 (default 4e4 m^-2, 4e4 m^-2, 1e6 rad^-2) */
    float slam_prior_info[3];      /* > 0 (default 1e4) */
    int32_t slam_weighted_update;  /* 0 (default) or 1 */
    /* Scan-to-map Gauss-Newton correction of the match inside the step
     * (u_mode = ASLAM_U_FIXEDLAG; Sec. III-D, Eq. 5): slam_gn_iters damped
     * steps xi <- xi - (J^T J + 1e-6 I)^-1 J^T e of the soft expected-range
     * model (uq_samples samples of uq_step_m, the belief before this scan in
     * nats) from the correlative match, over the beams whose measured range
     * lies within the model's reach and within two cells of the model's range
     * at the match.  An iterate outside the matcher's search box
     * (+-(csm_n_xy + 1) cells, +-(csm_n_th + 1) csm_dth_rad) keeps the match;
     * otherwise the result, rounded to 1 mm and 1 mrad, replaces the match as
     * the window's pose measurement.  An episode's first scan keeps the
     * match.  0 (default) switches the correction off. */
    int32_t slam_gn_iters;         /* 0 .. 10 */
} aslam_config;

#define ASLAM_U_CALLER    0
#define ASLAM_U_SCANMATCH 1
#define ASLAM_U_FIXEDLAG  2

#define ASLAM_MAX_BEAMS 1024
#define ASLAM_MAX_MAP_SIDE 8192

/* Borrowed device views of the batch state (valid until destroy). */
typedef struct {
    float *x, *y, *th;             /* [E] pose (m, m, rad in [-pi, pi)) */
    float *u_prev;                 /* [E] U_{t-1} */
    int32_t *t;                    /* [E] step within the episode */
    int32_t *g;                    /* [E] global step count (noise counter) */
    int32_t *ep;                   /* [E] episode count */
    int32_t *done;                 /* [E] 1 after a collision or t == T_episode */
    int16_t *belief;               /* [map_off[E]] log-odds, env e at map_off[e] */
    float *z;                      /* [ray_off[E]] measured ranges of the last step */
    float *z_true;                 /* [ray_off[E]] noise-free ranges (DEBUG flag) */
    uint8_t *hit;                  /* [ray_off[E]] 1 if the beam returned (DEBUG flag) */
    uint32_t *counts;              /* [map_off[E]] last step's (hits<<16 | misses) (DEBUG) */
    int64_t *ray_cells;            /* [E] cells updated by the last step */
    int64_t *gt_cells;             /* [E] ground-truth cells read by the last step */
    float *terms;                  /* [E, ASLAM_N_TERMS] last step's reward terms */
    const int64_t *h_map_off;      /* HOST [E+1] cell offsets of each env's grid */
    const int64_t *h_ray_off;      /* HOST [E+1] offsets of each env's beams */
    int32_t b_max;                 /* max beams over envs (observation row = b_max + 2) */
    double *pose_cov;              /* [E, 6] (xx, xy, xt, yy, yt, tt) with ASLAM_U_SCANMATCH or
                                    * ASLAM_U_FIXEDLAG, else NULL */
    float *slam_window;            /* [E, L, 3] pose estimates, oldest first (ASLAM_U_FIXEDLAG) */
    int32_t *slam_count;           /* [E] poses in each window */
    float *slam_match;             /* [E, 3] this step's (score_norm, margin, w) */
    int64_t *slam_scores;          /* [E, 3] this step's (best, second, best index) */
    float *slam_match_pose;        /* [E, 3] this step's matched pose */
    float *slam_gn_pose;           /* [E, 3] this step's corrected match (slam_gn_iters > 0),
                                    * else NULL */
} aslam_state_ptrs;

/* Fill `cfg` with defaults (version, struct_size, constants). */
aslam_status aslam_config_init(aslam_config *cfg);

/* Device workspace bytes a batch with this config needs (host-only call). */
aslam_status aslam_workspace_bytes(const aslam_config *cfg, size_t *bytes);

/*
 * Create a batch over a caller-owned device workspace of at least
 * aslam_workspace_bytes() bytes, 256-byte aligned, which must stay valid and
 * untouched until aslam_destroy_batch.
 *   d_gt     device uint8 ground-truth grids, env e at h_gt_off[e] (row-major
 *            W x H); read during this call only (packed into the workspace).
 *   h_gt_off host int64 [E+1] offsets into d_gt.
 *   d_spawn  device float [E, n_spawn, 3] spawn poses (x, y, th); copied.
 * All envs start at spawn pose 0 with an all-unknown map (L = 0).
 * Synchronises `stream` before returning.
 */
aslam_status aslam_create_batch(const aslam_config *cfg, void *d_workspace, size_t bytes,
                                const uint8_t *d_gt, const int64_t *h_gt_off,
                                const float *d_spawn, void *stream, aslam_batch **out);

/*
 * One environment step for every env (Sec. III-C/D/E, IV-A):
 *   d_actions device float [E, 2] (v, w), clamped to [0, v_max] x [-w_max, w_max];
 *   d_u       device float [E] uncertainty U_t from the SLAM backend, or NULL (0).
 * Envs flagged done by the previous step are first reset to their next spawn
 * pose with a cleared map.  Results stay in the workspace for
 * aslam_reward / aslam_observe / aslam_reward_terms.
 */
aslam_status aslam_step(aslam_batch *b, const float *d_actions, const float *d_u, void *stream);

/* aslam_step that also writes the reward [E] and observation [E, b_max+2]
 * directly (either may be NULL). */
aslam_status aslam_step_fused(aslam_batch *b, const float *d_actions, const float *d_u,
                              float *d_reward, float *d_obs, void *stream);

/* aslam_step_fused from and to HOST memory: h_actions [E, 2] and h_u [E]
 * (may be NULL) in, the reward [E] and observation [E, b_max+2] (either may
 * be NULL) out, in order on `stream`.  A page-locked buffer (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory) is read or written by the step's
 * kernels in place, through its device mapping; any other buffer is copied
 * through a staging area of the workspace (the CUDA runtime may then stage
 * and block).  The results are valid once the stream has been synchronised,
 * and the inputs must stay unchanged and every buffer valid until then.
 * Errors as aslam_step_fused, plus ASLAM_ERR_CUDA for a failed copy. */
aslam_status aslam_step_host(aslam_batch *b, const float *h_actions, const float *h_u,
                             float *h_reward, float *h_obs, void *stream);

/* Reward of the last step, [E] fp32, selected by cfg.reward_mode. */
aslam_status aslam_reward(aslam_batch *b, float *d_reward, void *stream);

/* All reward terms of the last step, [E, ASLAM_N_TERMS] fp32. */
aslam_status aslam_reward_terms(aslam_batch *b, float *d_terms, void *stream);

/* Observation of the last step (Eq. 3): [E, b_max + 2] fp32 rows
 * [z_0 .. z_{B-1}, r_max padding up to b_max, yaw, U_t]. */
aslam_status aslam_observe(aslam_batch *b, float *d_obs, void *stream);

/* Reset the envs whose d_mask byte is non-zero (NULL: all) on the next step
 * boundary: marks them done so the next aslam_step resets them. */
aslam_status aslam_reset(aslam_batch *b, const uint8_t *d_mask, void *stream);

/* Borrowed device pointers to the batch state (host call, no sync). */
aslam_status aslam_get_state(aslam_batch *b, aslam_state_ptrs *out);

/* Synchronise `stream` and return ASLAM_ERR_DEVICE if a device-side check
 * has fired since create (ASLAM_FLAG_CHECKS, or a singular fixed-lag window
 * of ASLAM_U_FIXEDLAG); the word stays set. */
aslam_status aslam_sync_status(aslam_batch *b, void *stream);

/*
 * Capture one aslam_step_fused into a CUDA graph bound to these pointers
 * (which must then hold the next step's inputs at every replay), and replay
 * it with aslam_graph_step.  `stream` must not be capturing already.
 */
aslam_status aslam_capture_graph(aslam_batch *b, const float *d_actions, const float *d_u,
                                 float *d_reward, float *d_obs, void *stream);
aslam_status aslam_graph_step(aslam_batch *b, void *stream);

/*
 * Pick threads-per-CTA and the shared-memory counter window by timing
 * candidate launches on this batch's own worlds (zero actions from the
 * current poses), then reset every env.  Synchronises `stream`.
 * h_best (optional, int32[2]) receives {threads_per_cta, window_cells}.
 */
aslam_status aslam_autotune(aslam_batch *b, int32_t *h_best, void *stream);

/* Checkpoint: bytes of the mutable state; save to / load from host memory.
 * Synchronises `stream`.  A loaded state continues bit-exactly. */
aslam_status aslam_state_bytes(aslam_batch *b, size_t *bytes);
aslam_status aslam_save_state(aslam_batch *b, void *h_buf, size_t bytes, void *stream);
aslam_status aslam_load_state(aslam_batch *b, const void *h_buf, size_t bytes, void *stream);

/*
 * Batched correlative scan matching (Sec. III-D: a discretised (dx, dy, dth)
 * neighbourhood of the predicted pose is evaluated against the log-odds
 * grid; the best candidate is an absolute pose measurement whose
 * information is scaled by the normalised match score and the ambiguity
 * margin between the best and second-best candidates).  2-D batches only.
 *
 * Candidates: translations (i, j) in [-n_xy, n_xy]^2 whole cells and
 * rotations k in [-n_th, n_th] steps of dth_rad.  For each returned beam
 * (range < r_max) its direction is rotated by th_k = th + k*dth (fp32, the
 * library's sin/cos), its endpoint (x, y) + z*(cos, sin) is taken to a cell
 * by floor(metres / res) and shifted by (i, j); the candidate's score is the
 * sum over beams of the cell's occupancy evidence min(255, max(L, 0) >> 4)
 * (0 outside the map).  Best: the highest score, ties to the lowest index
 * ((k + n_th)(2n_xy+1) + (j + n_xy))(2n_xy+1) + (i + n_xy); second: the
 * highest score of the candidates more than `sep` steps from the best in
 * some coordinate.  With N returned beams: score_norm = best / (255 N),
 * margin = (best - second) / best, w = score_norm * margin (each 0 when
 * its denominator is 0), evaluated in fp64 and stored as fp32.
 *
 *   d_pose_pred [E, 3]  predicted poses (x, y, th)
 *   d_ranges    [sum B] ranges, or NULL for the batch's last measured ranges
 *   d_pose_out  [E, 3]  (x + i*res, y + j*res, th_k wrapped to [-pi, pi))
 *   d_match     [E, 3]  (score_norm, margin, w)
 *   d_scores    [E, 3]  int64 (best, second, best index)
 */
typedef struct {
    uint32_t struct_size;          /* sizeof(aslam_csm_config) */
    int32_t n_xy;                  /* 0..8 */
    int32_t n_th;                  /* 0..8 */
    int32_t sep;                   /* >= 0 */
    float dth_rad;                 /* > 0 */
} aslam_csm_config;

/* Defaults: n_xy = 5, n_th = 5, sep = 1, dth_rad = 0.01. */
aslam_status aslam_csm_config_init(aslam_csm_config *cfg);
aslam_status aslam_csm(aslam_batch *b, const aslam_csm_config *cfg, const float *d_pose_pred,
                       const float *d_ranges, float *d_pose_out, float *d_match,
                       int64_t *d_scores, void *stream);

/*
 * Batched fixed-lag window Gauss-Newton (Sec. III-D, Eq. 5-6): per env a
 * sliding window of L planar poses x_i = (x, y, th) with
 *   a prior factor      r = x_0 - p                       information diag(d_prior_info)
 *   odometry factors    r = (R(th_i)^T (t_{i+1} - t_i) - u_xy,
 *                            wrap(th_{i+1} - th_i - u_th))  information diag(odo_info)
 *   pose factors        r = x_i - z_i                      information diag(d_meas_info)
 * (angle residuals wrapped to [-pi, pi); a zero information row disables a
 * factor, e.g. a pose without a scan match).  `iters` Gauss-Newton steps
 * x <- x + H^-1 (-g) in fp64, then at the final estimate the marginal
 * covariance of the newest pose, Sigma_last = the last 3x3 block of H^-1
 * (Eq. 6), and U = det(Sigma_last)^(1/3) / u_scale.
 *   d_x         [E, L, 3] fp32, in: initial estimate, out: optimised window
 *   d_odo       [E, L-1, 3]   d_meas, d_meas_info [E, L, 3]
 *   d_prior, d_prior_info     [E, 3]
 *   d_cov [E, 9], d_u [E], d_status [E] (0 ok, 1 singular normal matrix;
 *   then cov and U are NaN): optional outputs.
 */
typedef struct {
    uint32_t struct_size;          /* sizeof(aslam_flgn_config) */
    int32_t n_envs;                /* E >= 1 */
    int32_t window;                /* L in [1, 16] */
    int32_t iters;                 /* 0 .. 20 */
    float odo_info[3];             /* > 0: x, y (m^-2), th (rad^-2) */
    float u_scale;                 /* > 0 */
} aslam_flgn_config;

/* Defaults: 1 env, L = 8, 3 iterations, odometry std 0.01 m / 0.01 rad,
 * u_scale = 1e-4 (one step of that odometry noise). */
aslam_status aslam_flgn_config_init(aslam_flgn_config *cfg);
aslam_status aslam_fixed_lag_gn(const aslam_flgn_config *cfg, float *d_x, const float *d_odo,
                                const float *d_meas, const float *d_meas_info,
                                const float *d_prior, const float *d_prior_info, float *d_cov,
                                float *d_u, int32_t *d_status, void *stream);

/*
 * Uncertainty bridge for SLAM-agnostic fine-tuning (Sec. III-G, Eq. 21-22):
 * alpha = min(1, t / t_bridge) (fp64, rounded once to fp32) and, per env,
 * U = alpha * U_new + (1 - alpha) * U_old in fp32.  d_u_old / d_u_new:
 * device float [E] (the training backend's and the external estimator's
 * uncertainty); t >= 0 is the fine-tuning step, t_bridge >= 1.  Writes
 * d_u_out [E] (optional) and/or the U slot (column b_max + 1) of the
 * observation rows d_obs [E, b_max + 2] (optional); at least one is needed.
 * The reward is not touched: the bridge changes only what the policy sees.
 */
aslam_status aslam_bridge_u(aslam_batch *b, const float *d_u_old, const float *d_u_new, int64_t t,
                            int64_t t_bridge, float *d_u_out, float *d_obs, void *stream);

/*
 * Per-kernel device timing of aslam_step / aslam_step_fused (graph replays
 * are not timed).  aslam_profile_begin creates CUDA events for the next
 * max_steps (1 .. 2^20) steps; each of those steps records one event before
 * its first kernel and one after each kernel, on its own stream.
 * aslam_profile_end waits for the last recorded event, writes the summed
 * device time in ms of kernel k to h_ms[k] (host double
 * [ASLAM_MAX_STEP_KERNELS], zero past the last kernel), the number of
 * kernels a step launches to *h_n_kernels and the number of timed steps to
 * *h_n_steps, and releases the events; ASLAM_ERR_STATE without a begin.
 * aslam_kernel_name(b, k) is the name of kernel k ("sense2d_kernel", which
 * also integrates the actions, then "uq2d_kernel" with ASLAM_U_SCANMATCH or
 * "slam_predict2d_kernel", "csm2d_kernel", "slam_window2d_kernel",
 * "slam_replan2d_kernel" with ASLAM_U_FIXEDLAG, then "update2d_kernel"; 3-D:
 * "step3d_kernel"), NULL
 * past the last.  A static string, owned by the library.
 */
#define ASLAM_MAX_STEP_KERNELS 8
aslam_status aslam_profile_begin(aslam_batch *b, int32_t max_steps);
aslam_status aslam_profile_end(aslam_batch *b, double *h_ms, int32_t *h_n_kernels,
                               int32_t *h_n_steps);
const char *aslam_kernel_name(const aslam_batch *b, int32_t k);

/* Release the host handle (the caller frees the workspace). */
void aslam_destroy_batch(aslam_batch *b);

const char *aslam_status_string(aslam_status s);
/* Last error message of this batch (b != NULL) or of the calling thread. */
const char *aslam_last_error(const aslam_batch *b);

/* Test hook: evaluate the library's deterministic fp32 sin/cos, log,
 * cos(2*pi*u) and Gaussian draw on n device inputs (outputs [n] each). */
aslam_status aslam_debug_detmath(const float *d_x, const float *d_u, int32_t n,
                                 float *d_sin, float *d_cos, float *d_log, float *d_cos2pi,
                                 uint64_t seed, float *d_gauss, void *stream);

/* ------------------------------------------------------------------------
 * Differentiable soft expected-range raycaster and scan-to-map Gauss-Newton
 * (Sec. III-D: pose estimate by Gauss-Newton on the scan residuals, Eq. 5,
 * and the pose covariance block from the inverse Gauss-Newton Hessian,
 * Eq. 6).  Grids are identical in size for all envs: fp32 natural log-odds
 * d_logodds[E, H, W] (row-major, cell (i, j) centred at ((i+.5)res, (j+.5)res),
 * bilinear between centres, clamped to the edge outside the map).  Beam b
 * casts K samples s_k = (k+1)*ds; p_k = sigmoid(bilinear log-odds);
 * T_0 = 1, T_{k+1} = T_k (1 - p_k); r = sum_k T_k p_k s_k + T_K * K*ds.
 * ------------------------------------------------------------------------ */
#define ASLAM_SOFT_MAX_SAMPLES 256

typedef struct {
    uint32_t struct_size;          /* sizeof(aslam_soft_config) */
    int32_t n_envs;                /* E >= 1 */
    int32_t map_w, map_h;          /* grid W, H (cells) for every env */
    int32_t n_beams;               /* B in [1, ASLAM_MAX_BEAMS] */
    int32_t n_samples;             /* K in [1, ASLAM_SOFT_MAX_SAMPLES] */
    float res_m;                   /* cell size (m) */
    float sample_step_m;           /* ds (m); the no-return range is K*ds */
    float fov_rad;                 /* 0 or >= 2*pi: full turn; else front arc */
    float gn_damping;              /* mu added to the diagonal of J^T J */
    float range_sigma_m;           /* range noise std: Sigma = sigma^2 (J^T J + mu I)^-1 */
} aslam_soft_config;

/* Defaults: 1 env, 256 x 256 @ 0.05 m, 360 beams, 64 samples of 0.05 m,
 * mu = 1e-6, sigma = 0.01 m. */
aslam_status aslam_soft_config_init(aslam_soft_config *cfg);

/* Soft ranges: d_pose [E, 3] (x, y, th) -> d_ranges [E, B]. */
aslam_status aslam_soft_range_fwd(const aslam_soft_config *cfg, const float *d_logodds,
                                  const float *d_pose, float *d_ranges, void *stream);

/* Ranges (optional, may be NULL) and their Jacobian d_jac [E, B, 3] w.r.t.
 * (x, y, th), by forward-mode differentiation. */
aslam_status aslam_soft_range_jac(const aslam_soft_config *cfg, const float *d_logodds,
                                  const float *d_pose, float *d_ranges, float *d_jac,
                                  void *stream);

/* Adjoint of sum(d_grad_ranges * r): d_grad_pose [E, 3] is overwritten;
 * d_grad_logodds [E, H, W] (optional) is ACCUMULATED into (+=, atomic fp32
 * adds, so the summation order varies from run to run).  The transmittance
 * of every beam is recomputed inside this call (nothing is kept from
 * aslam_soft_range_fwd). */
aslam_status aslam_soft_range_bwd(const aslam_soft_config *cfg, const float *d_logodds,
                                  const float *d_pose, const float *d_grad_ranges,
                                  float *d_grad_pose, float *d_grad_logodds, void *stream);

/* Gauss-Newton scan-to-map correction (Eq. 5): from d_pose_in [E, 3], `iters`
 * (0..100) damped steps xi <- xi - (J^T J + mu I)^{-1} J^T (r(xi) - z) on the
 * measured ranges d_z [E, B]; writes d_pose_out [E, 3] and, evaluated at
 * the final pose, the covariance block d_cov [E, 3, 3] = sigma^2 (J^T J +
 * mu I)^{-1} (Eq. 6, optional) and the scalar uncertainty
 * d_u [E] = det(Sigma)^(1/3) (D-optimality, optional). */
aslam_status aslam_gn_correct(const aslam_soft_config *cfg, const float *d_logodds,
                              const float *d_pose_in, const float *d_z, int32_t iters,
                              float *d_pose_out, float *d_cov, float *d_u, void *stream);

/*
 * Allocation-free single-scan update.  The paper has no counterpart: this
 * is an integration aid for callers that may not allocate device memory
 * (code running inside a host framework that owns the allocator, or with a
 * memory budget frozen after start-up).  It integrates one scan per
 * environment -- raycast from the given pose, range noise, miss/hit counts,
 * one clamp per scan -- exactly as aslam_step does for a robot that did not
 * move, but keeps its per-cell counters in a fixed array inside the library
 * (16 MiB, held by every GPU that loads the library until the process
 * exits) instead of a workspace.  It calls no cudaMalloc/cudaFree.
 *   cfg        constants (res_m, r_max_m, fov_rad, noise_sigma_m, l_*_q, seed)
 *              and HOST h_map_w/h_map_h/h_n_beams [n_envs]; every env must
 *              have the same beam count B.
 *   d_gt       device uint8 ground-truth grids, packed: env e at h_gt_off[e].
 *   h_gt_off   HOST int64 [n_envs+1] prefix sums of W*H (h_gt_off[0] = 0).
 *   d_pose     device float [n_envs, 3] scan pose (x, y, th).
 *   d_step     device int32 [n_envs] noise counter (aslam_step's global step).
 *   d_belief   device int16 log-odds, same layout as d_gt, updated in place.
 *   d_ranges   device float [n_envs, B] measured ranges (output).
 * Limits: n_envs <= 2048, total cells <= 4194304, B <= 1024; larger requests
 * return ASLAM_ERR_INVALID_ARG.  The first call on a device looks up the
 * array's device address with that device current.  Every call copies its
 * small tables from host memory, so a call made while `stream` is being
 * captured into a CUDA graph returns ASLAM_ERR_UNSUPPORTED.  All calls share
 * the array (each clears what it uses first), so calls that overlap on the
 * GPU race: serialise them.
 */
aslam_status aslam_scan_update_noalloc(const aslam_config *cfg, const uint8_t *d_gt,
                                       const int64_t *h_gt_off, const float *d_pose,
                                       const int32_t *d_step, int16_t *d_belief,
                                       float *d_ranges, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ASLAM_H */
