/*
 * aslam_oracle.c -- plain, slow CPU oracle of the batched Active-SLAM
 * environment step (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may load this library.  The product path never does.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes, in the order the method defines it:
 *   - action integration with the unicycle model of the differential-drive
 *     robot (Sec. III-C action space Eq. 4; Sec. IV-A robot; dt = 0.1 s);
 *   - the LiDAR sensor of Sec. IV-A: each beam's range is the distance to
 *     the first occupied ground-truth cell along the beam, plus Gaussian
 *     noise N(0, sigma^2), optionally rounded to a number of decimal places
 *     (Sec. IV-A gives the sensor a resolution of 0.01 m), clipped to
 *     [r_min, r_max] (Sec. IV-A: minimum range 0.1 m); a beam that meets no
 *     obstacle within r_max reports r_max;
 *   - the log-odds occupancy-grid update of Sec. III-D: cells the beam
 *     crosses before its measured endpoint receive a "miss" increment, the
 *     endpoint cell a "hit" increment when the beam returned, and every cell
 *     is clamped, after summing all of one scan's increments;
 *   - the map entropy H = sum_cells h(p) (the information measure Table I
 *     lists as "Map entropy"), recomputed from scratch over the whole map;
 *   - the reward of Sec. III-E, Eq. 7-17, term by term, and the observation
 *     vector of Eq. 3.
 *
 * Geometry is defined on exact fixed-point numbers so that the set of
 * traversed cells is unique: the ray origin is in Q16 cell units, the
 * direction in Q30; the walk visits cells in the order in which the exact
 * rational ray parameter crosses grid lines (ties: the horizontal line, i.e.
 * the Y crossing, first).  All comparisons are exact 128-bit products.
 * Values that decide integers (pose, directions, noise, range endpoints) are
 * computed in fp32 with a fixed sequence of IEEE operations and the
 * project's own sin/cos/log polynomials; everything else is fp64.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ------------------------------------------------------------------------ */
/* Deterministic fp32 elementary functions (own polynomials, IEEE + - * /).  */
/* ------------------------------------------------------------------------ */

/* Taylor coefficients of sin and cos (1/n!, rounded to float once). */
#define ORC_S1 ((float)(-1.0 / 6.0))
#define ORC_S2 ((float)(1.0 / 120.0))
#define ORC_S3 ((float)(-1.0 / 5040.0))
#define ORC_S4 ((float)(1.0 / 362880.0))
#define ORC_C1 ((float)(-1.0 / 2.0))
#define ORC_C2 ((float)(1.0 / 24.0))
#define ORC_C3 ((float)(-1.0 / 720.0))
#define ORC_C4 ((float)(1.0 / 40320.0))
#define ORC_C5 ((float)(-1.0 / 3628800.0))

/* sin and cos of r, |r| <= pi/4, by the truncated Taylor series. */
static void orc_sincos_poly(float r, float *s, float *c)
{
    float r2 = r * r;
    float p = ORC_S3 + r2 * ORC_S4;
    p = ORC_S2 + r2 * p;
    p = ORC_S1 + r2 * p;
    float r3 = r * r2;
    *s = r + r3 * p;
    float q = ORC_C4 + r2 * ORC_C5;
    q = ORC_C3 + r2 * q;
    q = ORC_C2 + r2 * q;
    q = ORC_C1 + r2 * q;
    *c = 1.0f + r2 * q;
}

/* sin/cos of an fp32 angle: quadrant reduction in fp64 (x - k*pi/2), then
 * the polynomial on the fp32 remainder. */
void orc_sincosf(float x, float *s, float *c)
{
    const double two_over_pi = 0.63661977236758134308;
    const double pi_over_2 = 1.57079632679489661923;
    double k = rint((double)x * two_over_pi);
    double kp = k * pi_over_2;
    float r = (float)((double)x - kp);
    float ps, pc;
    orc_sincos_poly(r, &ps, &pc);
    int q = ((int)k) & 3;
    switch (q) {
    case 0: *s = ps;  *c = pc;  break;
    case 1: *s = pc;  *c = -ps; break;
    case 2: *s = -ps; *c = -pc; break;
    default: *s = -pc; *c = ps; break;
    }
}

/* cos(2*pi*u) for u in [0, 1): exact quarter-turn reduction on u. */
float orc_cos2pi(float u)
{
    const float two_pi = (float)(2.0 * 3.14159265358979323846);
    float q = rintf(u * 4.0f);
    float r = u - q * 0.25f;           /* exact, |r| <= 1/8 */
    float a = r * two_pi;
    float ps, pc;
    orc_sincos_poly(a, &ps, &pc);
    switch (((int)q) & 3) {
    case 0: return pc;
    case 1: return -ps;
    case 2: return -pc;
    default: return ps;
    }
}

/* Natural log of a positive normal float: u = m * 2^e with m in
 * [sqrt(1/2), sqrt(2)), ln m = 2 atanh((m-1)/(m+1)) by its odd series. */
float orc_logf(float u)
{
    uint32_t bits;
    memcpy(&bits, &u, 4);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    uint32_t mb = (bits & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (mb > 0x3fb504f3u) {             /* m > sqrt(2) */
        m = m * 0.5f;
        e += 1;
    }
    const float ln2_hi = 0.693145751953125f;          /* 16 significant bits */
    const float ln2_lo = (float)(0.69314718055994530942 - 0.693145751953125);
    float f = m - 1.0f;
    float s = f / (m + 1.0f);
    float s2 = s * s;
    float p = (float)(1.0 / 9.0) + s2 * (float)(1.0 / 11.0);
    p = (float)(1.0 / 7.0) + s2 * p;
    p = (float)(1.0 / 5.0) + s2 * p;
    p = (float)(1.0 / 3.0) + s2 * p;
    float two_s = s + s;
    float lnm = two_s + two_s * (s2 * p);
    float fe = (float)e;
    return (fe * ln2_lo + lnm) + fe * ln2_hi;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon et al., SC'11).              */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normal draw for (seed, env, global step, beam): Box-Muller on
 * the first two Philox words, u1 in (0, 1], u2 in [0, 1). */
float orc_gauss(uint64_t seed, uint32_t env, uint32_t step, uint32_t beam)
{
    uint32_t ctr[4] = {beam, env, step, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    float u1 = (float)((r[0] >> 8) + 1u) * (1.0f / 16777216.0f);
    float u2 = (float)(r[1] >> 8) * (1.0f / 16777216.0f);
    float l = orc_logf(u1);
    float rad = sqrtf(-2.0f * l);
    return rad * orc_cos2pi(u2);
}

/* ------------------------------------------------------------------------ */
/* Exact grid traversal (2-D).                                               */
/* ------------------------------------------------------------------------ */

static int64_t orc_floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0)))
        q -= 1;
    return q;
}

/* Q16 distance from the origin coordinate P to the first grid line the
 * ray meets along an axis with direction component D (unused when D == 0). */
static int64_t orc_first_gap(int32_t P, int32_t D)
{
    int64_t cell = orc_floordiv(P, 65536);
    if (D > 0)
        return (cell + 1) * 65536 - (int64_t)P;
    return (int64_t)P - cell * 65536;
}

/* Is the crossing with Q16 numerator n on an axis with |D| = ad within
 * ray parameter T (Q16 cells)?  t = n * 2^14 / ad  <=  T / 2^16. */
static int orc_within(int64_t n, int64_t ad, int64_t T)
{
    return (i128)n * ((i128)1 << 30) <= (i128)T * (i128)ad;
}

/* Walk the cells of one ray up to parameter T (Q16 cells).  Writes the flat
 * indices of the visited in-map cells (origin first) and, per cell, the Q16
 * numerator and |D| of the crossing that entered it (0, 0 for the origin).
 * Stops at the first crossing that would leave the W x H map and reports it
 * through *left.  Returns the number of cells written. */
int orc_walk2d(int32_t Px, int32_t Py, int32_t Dx, int32_t Dy, int64_t T,
               int32_t W, int32_t H, int64_t *cells, int64_t *enter_n,
               int64_t *enter_ad, int cap, int *left)
{
    int64_t i = orc_floordiv(Px, 65536), j = orc_floordiv(Py, 65536);
    int n_out = 0;
    *left = 0;
    if (i < 0 || i >= W || j < 0 || j >= H) {
        *left = 1;
        return 0;
    }
    int sx = (Dx > 0) - (Dx < 0), sy = (Dy > 0) - (Dy < 0);
    int64_t adx = Dx < 0 ? -(int64_t)Dx : Dx, ady = Dy < 0 ? -(int64_t)Dy : Dy;
    int64_t nx = orc_first_gap(Px, Dx), ny = orc_first_gap(Py, Dy);
    if (n_out < cap) {
        cells[n_out] = j * W + i;
        enter_n[n_out] = 0;
        enter_ad[n_out] = 0;
    }
    n_out++;
    for (;;) {
        int have_x = sx != 0 && orc_within(nx, adx, T);
        int have_y = sy != 0 && orc_within(ny, ady, T);
        if (!have_x && !have_y)
            break;
        int take_x;
        if (have_x && have_y)      /* strictly earlier X crossing; ties go to Y */
            take_x = (i128)nx * ady < (i128)ny * adx;
        else
            take_x = have_x;
        int64_t en, ea;
        if (take_x) {
            i += sx; en = nx; ea = adx; nx += 65536;
        } else {
            j += sy; en = ny; ea = ady; ny += 65536;
        }
        if (i < 0 || i >= W || j < 0 || j >= H) {
            *left = 1;
            break;
        }
        if (n_out < cap) {
            cells[n_out] = j * W + i;
            enter_n[n_out] = en;
            enter_ad[n_out] = ea;
        }
        n_out++;
    }
    return n_out;
}

/* ------------------------------------------------------------------------ */
/* Sensor geometry.                                                          */
/* ------------------------------------------------------------------------ */

/* Beam angle of beam b of B over the field of view: a full turn without a
 * duplicate at 2*pi, or a front arc with both ends included (Sec. IV-A
 * spaces the rays evenly over the field of view). */
static double orc_beam_angle(int b, int B, double fov)
{
    const double two_pi = 2.0 * 3.14159265358979323846;
    if (fov <= 0.0 || fov >= two_pi - 1e-9)
        return (two_pi * (double)b) / (double)B;
    if (B == 1)
        return 0.0;
    return -0.5 * fov + ((double)b * fov) / (double)(B - 1);
}

void orc_beam_dirs(int B, double fov, float *cb, float *sb)
{
    for (int b = 0; b < B; ++b) {
        double a = orc_beam_angle(b, B, fov);
        cb[b] = (float)cos(a);
        sb[b] = (float)sin(a);
    }
}

/* Ray origin in Q16 cell units and direction in Q30 for a robot at (x, y)
 * with heading (c, s) = (cos th, sin th) and beam (cb, sb). */
void orc_ray_setup(float x, float y, float c, float s, float cb, float sb, float res,
                   int32_t *Px, int32_t *Py, int32_t *Dx, int32_t *Dy)
{
    *Px = (int32_t)lrintf((x / res) * 65536.0f);
    *Py = (int32_t)lrintf((y / res) * 65536.0f);
    float dx = c * cb - s * sb;
    float dy = s * cb + c * sb;
    *Dx = (int32_t)lrintf(dx * 1073741824.0f);
    *Dy = (int32_t)lrintf(dy * 1073741824.0f);
}

/* Metric range of a crossing with Q16 numerator n on an axis with |D| = ad. */
static float orc_range_of(int64_t n, int64_t ad, float res)
{
    if (ad == 0)
        return 0.0f;
    float t = ((float)n / (float)ad) * 16384.0f;
    return t * res;
}

static int32_t orc_q16_of_range(float z, float res)
{
    return (int32_t)lrintf((z / res) * 65536.0f);
}

/* ------------------------------------------------------------------------ */
/* Entropy of a log-odds cell (nats), plain formula.                          */
/* ------------------------------------------------------------------------ */
double orc_cell_entropy(double l)
{
    double p = 1.0 / (1.0 + exp(-l));
    return -p * log(p) - (1.0 - p) * log(1.0 - p);
}

double orc_map_entropy(const int16_t *L, int64_t n, double scale)
{
    double h = 0.0;
    for (int64_t k = 0; k < n; ++k)
        h += orc_cell_entropy((double)L[k] * scale);
    return h;
}

/* ------------------------------------------------------------------------ */
/* The batched 2-D environment step.                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n_envs;
    int32_t b_max;             /* row length of the per-beam outputs */
    int32_t n_spawn;
    int32_t hit_q, miss_q, clamp_q;
    int32_t t_episode;
    int32_t pad0;
    uint64_t seed;
    float res, r_max, fov, sigma, dt, v_max, w_max, d_crash, d_full, visit_cell;
    float r_min;               /* minimum range (m); returned ranges are clipped up to it */
    float dec_scale;           /* 10^decimals of the range rounding, 0 for none */
    double logodds_scale;
    double lam_col, lam_explore, lam_abs, lam_delta, kappa, u_hi;
    const int32_t *map_w, *map_h, *n_beams;
    const int64_t *map_off;    /* [E+1] */
    const int64_t *visit_off;  /* [E+1] */
    const int32_t *env_id;     /* [E] index of each env in the noise stream, or NULL */
    /* in-step pose uncertainty (u_mode 1): see orc_scan_uncertainty */
    int32_t u_mode, uq_samples;
    float uq_step, uq_range_sigma, uq_odo[3], uq_prior[3], uq_u_scale;
    /* SLAM backbone in the step (u_mode 2): see orc_slam_backbone */
    int32_t slam_window, slam_iters, csm_n_xy, csm_n_th, csm_sep;
    float csm_dth, slam_meas_info[3], slam_prior_info[3];
    int32_t slam_weighted;
    int32_t slam_gn_iters;     /* scan-to-map Gauss-Newton steps on the match (0: none) */
} orc_cfg;

typedef struct {
    const uint8_t *gt;
    int16_t *belief;
    float *x, *y, *th, *u_prev;
    int32_t *t, *g, *ep;
    uint8_t *done;
    int32_t *visit;
    const float *spawn;        /* [E, n_spawn, 3] */
    double *sigma;             /* [E, 6] pose covariance (xx, xy, xt, yy, yt, tt), u_mode 1 and 2 */
    float *win_x, *win_odo, *win_meas, *win_minfo;   /* [E, L, 3] window (u_mode 2) */
    int32_t *win_n;            /* [E] poses in the window */
    float *slam_match, *slam_pose;                    /* [E, 3] this step's scan match */
    int64_t *slam_scores;      /* [E, 3] */
    float *slam_upd_w;         /* [E] this step's map-update weight */
    float *slam_gn_pose;       /* [E, 3] this step's corrected match (or NULL) */
} orc_state;

enum { ORC_NT = 12 };          /* reward terms per env */

typedef struct {
    float *z, *z_true;         /* [E, b_max] */
    uint8_t *hit;              /* [E, b_max] */
    int32_t *cnt_h, *cnt_m;    /* [sum W*H] or NULL: this step's hit/miss counts */
    double *terms;             /* [E, ORC_NT] */
    float *reward_ent, *reward_comp;
    float *obs;                /* [E, b_max + 2] */
    int64_t *ray_cells, *gt_cells;
} orc_out;

/* Measured range of a returned beam (Sec. IV-A sensor): noise, then rounding
 * to 1/dec_scale m (round half to even on the scaled value) when dec_scale
 * > 0, then the clip to [r_min, r_max].  fp32, one IEEE operation at a time. */
float orc_measured_range(float z_true, float g, float sigma, float r_min, float r_max,
                         float dec_scale)
{
    float z = z_true + sigma * g;
    if (dec_scale > 0.0f) {
        float scaled = z * dec_scale;
        z = rintf(scaled) / dec_scale;
    }
    return fminf(fmaxf(z, r_min), r_max);
}

/* Uncertainty bridge of the SLAM-agnostic fine-tuning wrapper (Sec. III-G,
 * Eq. 21-22): alpha_t = min(1, t / T_bridge), evaluated in
 * fp64 and rounded once to fp32; U = alpha * U_new + (1 - alpha) * U_old in
 * fp32. */
float orc_bridge_alpha(int64_t t, int64_t t_bridge)
{
    double a = (double)t / (double)t_bridge;
    return (float)(a < 1.0 ? a : 1.0);
}

float orc_bridge_u(float u_old, float u_new, float alpha)
{
    float w_new = alpha * u_new;
    float w_old = (1.0f - alpha) * u_old;
    return w_new + w_old;
}

void orc_visit_dims(int32_t W, int32_t H, float res, float vc, int32_t *Vw, int32_t *Vh)
{
    int32_t a = (int32_t)ceilf((2.0f * ((float)W * res)) / vc);
    int32_t b = (int32_t)ceilf((2.0f * ((float)H * res)) / vc);
    *Vw = a < 1 ? 1 : a;
    *Vh = b < 1 ? 1 : b;
}

static double orc_clip(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

static void orc_reset_env(const orc_cfg *cfg, orc_state *st, int e)
{
    int64_t off = cfg->map_off[e], n = cfg->map_off[e + 1] - off;
    st->ep[e] += 1;
    int k = st->ep[e] % cfg->n_spawn;
    const float *sp = st->spawn + ((int64_t)e * cfg->n_spawn + k) * 3;
    st->x[e] = sp[0];
    st->y[e] = sp[1];
    st->th[e] = sp[2];
    st->t[e] = 0;
    st->u_prev[e] = 0.0f;
    st->done[e] = 0;
    memset(st->belief + off, 0, (size_t)n * sizeof(int16_t));
    for (int64_t v = cfg->visit_off[e]; v < cfg->visit_off[e + 1]; ++v)
        st->visit[v] = -1;
    if (st->win_n)
        st->win_n[e] = 0;
    if (st->sigma) {
        double *S = st->sigma + 6 * (int64_t)e;
        S[0] = (double)cfg->uq_prior[0] * cfg->uq_prior[0];
        S[1] = S[2] = S[4] = 0.0;
        S[3] = (double)cfg->uq_prior[1] * cfg->uq_prior[1];
        S[5] = (double)cfg->uq_prior[2] * cfg->uq_prior[2];
    }
}

/* ---- in-step pose uncertainty (Sec. III-D, Eq. 5-6) ------------------------ */

typedef struct {
    int32_t W, H, B, K;
    double res, ds, fov;
} orc_soft_cfg;                /* as in soft_range_oracle.c (same library) */

double orc_soft_range(const orc_soft_cfg *c, const float *L, double x, double y, double th,
                      int b, double gr, double *grad_pose, double *grad_map);

static double orc_det3(const double *M)
{
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* Inverse of a 3x3 matrix by its adjugate. */
static void orc_inv3(const double *M, double *R)
{
    double d = orc_det3(M);
    R[0] = (M[4] * M[8] - M[5] * M[7]) / d;
    R[1] = (M[2] * M[7] - M[1] * M[8]) / d;
    R[2] = (M[1] * M[5] - M[2] * M[4]) / d;
    R[3] = (M[5] * M[6] - M[3] * M[8]) / d;
    R[4] = (M[0] * M[8] - M[2] * M[6]) / d;
    R[5] = (M[2] * M[3] - M[0] * M[5]) / d;
    R[6] = (M[3] * M[7] - M[4] * M[6]) / d;
    R[7] = (M[1] * M[6] - M[0] * M[7]) / d;
    R[8] = (M[0] * M[4] - M[1] * M[3]) / d;
}

/* The pose uncertainty of one env after this step's scan, from the map as
 * it stands before the scan is integrated.  Scan-match information of the
 * soft expected-range model (the Gauss-Newton Hessian of Eq. 5, Eq. 6):
 * A = sum_b J_b J_b^T / sigma_r^2, J_b = d r_b / d(x, y, th) at the robot's
 * pose, over the log-odds L * logodds_scale (nats).  It is fused with the
 * previous covariance propagated by one step of odometry noise Q (the last
 * block of a two-pose window): Sigma_t = ((Sigma_{t-1} + Q)^-1 + A)^-1.
 * U_t = det(Sigma_t)^(1/3) / u_scale, u_scale = det(Q)^(1/3) unless given.
 * Updates st->sigma and returns U_t. */
static double orc_scan_uncertainty(const orc_cfg *cfg, orc_state *st, int e, float x, float y,
                                   float th)
{
    const int32_t W = cfg->map_w[e], H = cfg->map_h[e], B = cfg->n_beams[e];
    const int64_t off = cfg->map_off[e], n = (int64_t)W * H;
    float *Lf = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k)
        Lf[k] = (float)((double)st->belief[off + k] * cfg->logodds_scale);
    orc_soft_cfg sc;
    sc.W = W;
    sc.H = H;
    sc.B = B;
    sc.K = cfg->uq_samples;
    sc.res = cfg->res;
    sc.ds = cfg->uq_step > 0.0f ? (double)cfg->uq_step : (double)cfg->res;
    sc.fov = cfg->fov;
    double A[9] = {0};
    for (int b = 0; b < B; ++b) {
        double J[3] = {0.0, 0.0, 0.0};
        orc_soft_range(&sc, Lf, (double)x, (double)y, (double)th, b, 1.0, J, NULL);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                A[3 * i + j] += J[i] * J[j];
    }
    free(Lf);
    const double s2 = (double)cfg->uq_range_sigma * cfg->uq_range_sigma;
    double *S = st->sigma + 6 * (int64_t)e;
    double P[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    for (int i = 0; i < 3; ++i)
        P[4 * i] += (double)cfg->uq_odo[i] * cfg->uq_odo[i];
    double Pi[9], Info[9], Sn[9];
    orc_inv3(P, Pi);
    for (int k = 0; k < 9; ++k)
        Info[k] = Pi[k] + A[k] / s2;
    orc_inv3(Info, Sn);
    S[0] = Sn[0];
    S[1] = 0.5 * (Sn[1] + Sn[3]);
    S[2] = 0.5 * (Sn[2] + Sn[6]);
    S[3] = Sn[4];
    S[4] = 0.5 * (Sn[5] + Sn[7]);
    S[5] = Sn[8];
    double scale = cfg->uq_u_scale;
    if (!(scale > 0.0))
        scale = cbrt((double)cfg->uq_odo[0] * cfg->uq_odo[0] * cfg->uq_odo[1] * cfg->uq_odo[1] *
                     cfg->uq_odo[2] * cfg->uq_odo[2]);
    return cbrt(orc_det3(Sn)) / scale;
}

void orc_csm(const int16_t *belief, int32_t W, int32_t H, float res, float r_max, int32_t B,
             double fov, const float *z, float x, float y, float th, int32_t n, int32_t m,
             int32_t sep, float dth, float *pose_out, float *match, int64_t *scores);
int orc_fixed_lag_gn(int L, int iters, double *x, const double *odo, const double *meas,
                     const double *wm, const double *prior, const double *wp, const double *wo,
                     double *cov_last);

/* Scan-to-map Gauss-Newton correction of a matched pose (Sec. III-D, Eq. 5)
 * on the soft expected-range model of the belief before this scan (the
 * model of orc_soft_range: cfg->uq_samples samples of uq_step, the log-odds
 * in nats).  Residuals e_b = r_b(xi) - z_b over the inliers: beams whose
 * measured range lies within the model's reach (z_b < K ds) and whose model
 * range at the match is within two cells of it (a reading: an unknown or
 * barely observed cell (p near 1/2) ends the model's range early, and such
 * beams would pull the pose toward the map's gaps).  Starting at the match
 * pm, `iters` damped steps
 * xi <- xi - (J^T J + mu I)^-1 J^T e (mu = 1e-6, Cramer's rule), all in
 * fp64.  The correction is abandoned, and pm kept, when an iterate leaves
 * the matcher's search box (|dx|, |dy| <= (n_xy + 1) res, |dth| <=
 * (n_th + 1) dth) or is not finite.  The result is reported on a lattice
 * of 1 mm and 1 mrad: rint(v * 1000) / 1000 in fp64, then fp32 (a reading;
 * far below the 1 cm range noise, and it keeps the downstream integer map
 * independent of the last bits of the arithmetic). */
void orc_slam_correct_pose(const int16_t *belief, int32_t W, int32_t H, int32_t B, float res,
                           double fov, int32_t K, float ds, double logodds_scale, int32_t n_xy,
                           int32_t n_th, float dth, const float *z, const float pm[3], int iters,
                           float out[3])
{
    const int64_t n = (int64_t)W * H;
    float *Lf = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k)
        Lf[k] = (float)((double)belief[k] * logodds_scale);
    orc_soft_cfg sc;
    sc.W = W;
    sc.H = H;
    sc.B = B;
    sc.K = K;
    sc.res = res;
    sc.ds = ds > 0.0f ? (double)ds : (double)res;
    sc.fov = fov;
    const double r_far = (double)sc.K * sc.ds, mu = 1e-6;
    const double box_xy = (double)(n_xy + 1) * (double)res;
    const double box_th = (double)(n_th + 1) * (double)dth;
    double xi[3] = {pm[0], pm[1], pm[2]};
    int ok = 1;
    /* the beams that inform the correction: a measured range within the
     * model's reach (K ds) that the model at the match already explains to
     * within two cells */
    const double gate = 2.0 * (double)res;
    char *use = (char *)malloc((size_t)(B > 0 ? B : 1));
    for (int b = 0; b < B; ++b) {
        const double r0 = orc_soft_range(&sc, Lf, xi[0], xi[1], xi[2], b, 1.0, NULL, NULL);
        use[b] = (double)z[b] < r_far && fabs(r0 - (double)z[b]) < gate;
    }
    for (int it = 0; it < iters && ok; ++it) {
        double A[9] = {0}, g[3] = {0};
        for (int b = 0; b < B; ++b) {
            if (!use[b]) continue;
            double J[3] = {0.0, 0.0, 0.0};
            const double r = orc_soft_range(&sc, Lf, xi[0], xi[1], xi[2], b, 1.0, J, NULL);
            const double eb = r - (double)z[b];
            for (int i = 0; i < 3; ++i) {
                g[i] += J[i] * eb;
                for (int j = 0; j < 3; ++j)
                    A[3 * i + j] += J[i] * J[j];
            }
        }
        for (int i = 0; i < 3; ++i)
            A[4 * i] += mu;
        const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                           A[2] * (A[3] * A[7] - A[4] * A[6]);
        for (int col = 0; col < 3; ++col) {
            double M[9];
            memcpy(M, A, sizeof(M));
            for (int row = 0; row < 3; ++row)
                M[3 * row + col] = -g[row];
            xi[col] += (M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                        M[2] * (M[3] * M[7] - M[4] * M[6])) / det;
        }
        ok = fabs(xi[0] - (double)pm[0]) <= box_xy && fabs(xi[1] - (double)pm[1]) <= box_xy &&
             fabs(xi[2] - (double)pm[2]) <= box_th;     /* false for NaN */
    }
    free(Lf);
    free(use);
    for (int q = 0; q < 3; ++q)
        out[q] = ok ? (float)(rint(xi[q] * 1000.0) / 1000.0) : pm[q];
}

static void orc_slam_correct(const orc_cfg *cfg, const orc_state *st, int e, const float *z,
                             const float pm[3], int iters, float out[3])
{
    orc_slam_correct_pose(st->belief + cfg->map_off[e], cfg->map_w[e], cfg->map_h[e],
                          cfg->n_beams[e], cfg->res, cfg->fov, cfg->uq_samples, cfg->uq_step,
                          cfg->logodds_scale, cfg->csm_n_xy, cfg->csm_n_th, cfg->csm_dth, z, pm,
                          iters, out);
}

/* The SLAM backbone of one env in the step (Sec. III-D), on the map before
 * this scan: the pose predicted from the window's newest estimate and the
 * odometry (v dt, 0, w dt) (the integrated pose when the window is fresh)
 * is matched against the grid by orc_csm, and the match corrected by
 * orc_slam_correct (slam_gn_iters > 0, not on an episode's first scan); the
 * window of at most L poses slides, takes the prediction, the odometry
 * factor and the (corrected) match as a pose factor of information
 * w * meas_info (none for an episode's first scan),
 * anchors its oldest pose at the current estimate with prior_info, and is
 * solved by orc_fixed_lag_gn.  Returns U_t = det(Sigma_last)^(1/3) / scale
 * and writes this scan's map-update weight (the normalised match score, 1
 * for an episode's first scan). */
static double orc_slam_backbone(const orc_cfg *cfg, orc_state *st, int e, float x, float y,
                                float th, float ux, float uth, const float *z, float *upd_w)
{
    const int32_t W = cfg->map_w[e], H = cfg->map_h[e], B = cfg->n_beams[e];
    const int L = cfg->slam_window;
    float *wx = st->win_x + (int64_t)e * L * 3, *wo_ = st->win_odo + (int64_t)e * L * 3;
    float *wm = st->win_meas + (int64_t)e * L * 3, *wi = st->win_minfo + (int64_t)e * L * 3;
    int n = st->win_n[e];
    float pred[3];
    if (n == 0) {
        pred[0] = x; pred[1] = y; pred[2] = th;
    } else {
        const float *last = wx + 3 * (n - 1);
        float s, c;
        orc_sincosf(last[2], &s, &c);
        const float pi_f = (float)3.14159265358979323846;
        const float two_pi_f = (float)(2.0 * 3.14159265358979323846);
        pred[0] = last[0] + c * ux;
        pred[1] = last[1] + s * ux;
        float t = last[2] + uth;
        if (t >= pi_f) t = t - two_pi_f;
        if (t < -pi_f) t = t + two_pi_f;
        pred[2] = t;
    }
    float *pm = st->slam_pose + 3 * (int64_t)e, *mt = st->slam_match + 3 * (int64_t)e;
    orc_csm(st->belief + cfg->map_off[e], W, H, cfg->res, cfg->r_max, B, cfg->fov, z, pred[0],
            pred[1], pred[2], cfg->csm_n_xy, cfg->csm_n_th, cfg->csm_sep, cfg->csm_dth, pm, mt,
            st->slam_scores + 3 * (int64_t)e);
    /* the window's pose measurement: the match, corrected against the map
     * when there is one (an episode's first scan has an empty map) */
    float meas[3] = {pm[0], pm[1], pm[2]};
    if (cfg->slam_gn_iters > 0 && n > 0)
        orc_slam_correct(cfg, st, e, z, pm, cfg->slam_gn_iters, meas);
    if (st->slam_gn_pose)
        for (int q = 0; q < 3; ++q)
            st->slam_gn_pose[3 * (int64_t)e + q] = meas[q];
    if (n == L) {
        for (int i = 0; i + 1 < L; ++i)
            for (int q = 0; q < 3; ++q) {
                wx[3 * i + q] = wx[3 * i + 3 + q];
                wm[3 * i + q] = wm[3 * i + 3 + q];
                wi[3 * i + q] = wi[3 * i + 3 + q];
                if (i + 2 < L) wo_[3 * i + q] = wo_[3 * i + 3 + q];
            }
        n = L - 1;
    }
    const int first = n == 0;
    const float wgt = first ? 0.0f : mt[2];
    *upd_w = first ? 1.0f : mt[0];
    const float odo_step[3] = {ux, 0.0f, uth};
    for (int q = 0; q < 3; ++q) {
        wx[3 * n + q] = pred[q];
        wm[3 * n + q] = meas[q];
        wi[3 * n + q] = wgt * cfg->slam_meas_info[q];
        if (n > 0) wo_[3 * (n - 1) + q] = odo_step[q];
    }
    ++n;
    st->win_n[e] = n;
    double xd[48], od[48], md[48], id[48], prior[3], pinfo[3], wod[3], cov[9];
    for (int k = 0; k < 3 * n; ++k) {
        xd[k] = wx[k];
        md[k] = wm[k];
        id[k] = wi[k];
        od[k] = k < 3 * (n - 1) ? wo_[k] : 0.0;
    }
    for (int q = 0; q < 3; ++q) {
        prior[q] = wx[q];
        pinfo[q] = cfg->slam_prior_info[q];
        wod[q] = 1.0 / ((double)cfg->uq_odo[q] * cfg->uq_odo[q]);
    }
    orc_fixed_lag_gn(n, cfg->slam_iters, xd, od, md, id, prior, pinfo, wod, cov);
    for (int k = 0; k < 3 * n; ++k)
        wx[k] = (float)xd[k];
    double *S = st->sigma + 6 * (int64_t)e;
    S[0] = cov[0];
    S[1] = 0.5 * (cov[1] + cov[3]);
    S[2] = 0.5 * (cov[2] + cov[6]);
    S[3] = cov[4];
    S[4] = 0.5 * (cov[5] + cov[7]);
    S[5] = cov[8];
    double scale = cfg->uq_u_scale;
    if (!(scale > 0.0))
        scale = cbrt((double)cfg->uq_odo[0] * cfg->uq_odo[0] * cfg->uq_odo[1] * cfg->uq_odo[1] *
                     cfg->uq_odo[2] * cfg->uq_odo[2]);
    return cbrt(orc_det3(cov)) / scale;
}

/* Inverse-sensor counts of one beam (Sec. III-D log-odds grid): the ray from
 * the Q16 origin (Px, Py) along the Q30 direction (Dx, Dy) is walked up to
 * its measured range z (r_max for a beam without a return); every cell it
 * crosses gets a miss, except the last, which gets the hit of a returned
 * beam unless the walk left the map before reaching it.  Returns the number
 * of cells counted. */
static int64_t orc_count_beam(const orc_cfg *cfg, int32_t Px, int32_t Py, int32_t Dx, int32_t Dy,
                              float z, int hit, int32_t W, int32_t H, int64_t *cells,
                              int64_t *en, int64_t *ea, int cap, int32_t *hc, int32_t *mc)
{
    const int32_t Tz = orc_q16_of_range(hit ? z : cfg->r_max, cfg->res);
    int left;
    const int nc = orc_walk2d(Px, Py, Dx, Dy, Tz, W, H, cells, en, ea, cap, &left);
    for (int k = 0; k < nc; ++k) {
        if (k == nc - 1 && !left && hit)
            hc[cells[k]] += 1;
        else
            mc[cells[k]] += 1;
    }
    return nc;
}

/* Threads of orc_step2d's loop over environments (1 unless the CPU
 * baseline asks for more; built without OpenMP the loop is serial).  The
 * environments of a step are independent, so the thread count changes no
 * result. */
static int orc_threads = 1;

void orc_set_threads(int n)
{
    orc_threads = n < 1 ? 1 : n;
}

int orc_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

int orc_step2d(const orc_cfg *cfg, orc_state *st, const float *actions, const float *u_in,
               orc_out *out)
{
    const float pi_f = (float)3.14159265358979323846;
    const float two_pi_f = (float)(2.0 * 3.14159265358979323846);
    for (int e = 0; e < cfg->n_envs; ++e)
        if (cfg->n_beams[e] > 4096)
            return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_threads)
#endif
    for (int e = 0; e < cfg->n_envs; ++e) {
        const int32_t W = cfg->map_w[e], H = cfg->map_h[e], B = cfg->n_beams[e];
        const int64_t off = cfg->map_off[e], ncell = (int64_t)W * H;
        if (st->done[e])
            orc_reset_env(cfg, st, e);
        st->t[e] += 1;

        /* Action integration: Euler unicycle with the pre-step heading. */
        float v = fminf(fmaxf(actions[2 * e], 0.0f), cfg->v_max);
        float w = fminf(fmaxf(actions[2 * e + 1], -cfg->w_max), cfg->w_max);
        float s0, c0;
        orc_sincosf(st->th[e], &s0, &c0);
        float x = st->x[e] + (v * c0) * cfg->dt;
        float y = st->y[e] + (v * s0) * cfg->dt;
        float th = st->th[e] + w * cfg->dt;
        if (th >= pi_f)
            th = th - two_pi_f;
        if (th < -pi_f)
            th = th + two_pi_f;
        st->x[e] = x; st->y[e] = y; st->th[e] = th;

        /* Robot cell occupancy (or leaving the map) counts as a collision. */
        int32_t Px0 = (int32_t)lrintf((x / cfg->res) * 65536.0f);
        int32_t Py0 = (int32_t)lrintf((y / cfg->res) * 65536.0f);
        int64_t ri = orc_floordiv(Px0, 65536), rj = orc_floordiv(Py0, 65536);
        int col_cell = (ri < 0 || ri >= W || rj < 0 || rj >= H) ||
                       st->gt[off + rj * W + ri] != 0;

        /* Sensing and per-step hit/miss counts. */
        float cb_tab[4096], sb_tab[4096];
        orc_beam_dirs(B, cfg->fov, cb_tab, sb_tab);
        float s1, c1;
        orc_sincosf(th, &s1, &c1);
        int cap = W + H + 4;
        int64_t *cells = (int64_t *)malloc(sizeof(int64_t) * cap * 3);
        int64_t *en = cells + cap, *ea = cells + 2 * cap;
        int32_t *hc = (int32_t *)calloc((size_t)ncell, sizeof(int32_t));
        int32_t *mc = (int32_t *)calloc((size_t)ncell, sizeof(int32_t));
        const int32_t Tmax = orc_q16_of_range(cfg->r_max, cfg->res);
        int64_t ray_cells = 0, gt_cells = 0;
        float dmin_meas = cfg->r_max, dmin_true = cfg->r_max;
        for (int b = 0; b < B; ++b) {
            int32_t Px, Py, Dx, Dy;
            orc_ray_setup(x, y, c1, s1, cb_tab[b], sb_tab[b], cfg->res, &Px, &Py, &Dx, &Dy);
            int left;
            int nc = orc_walk2d(Px, Py, Dx, Dy, Tmax, W, H, cells, en, ea, cap, &left);
            int hit = 0;
            float z_true = cfg->r_max, z = cfg->r_max;
            for (int k = 0; k < nc; ++k) {
                if (st->gt[off + cells[k]]) {
                    hit = 1;
                    gt_cells += k + 1;
                    z_true = orc_range_of(en[k], ea[k], cfg->res);
                    break;
                }
            }
            if (!hit)
                gt_cells += nc;
            if (hit) {
                uint32_t eid = cfg->env_id ? (uint32_t)cfg->env_id[e] : (uint32_t)e;
                float g = orc_gauss(cfg->seed, eid, (uint32_t)st->g[e], (uint32_t)b);
                z = orc_measured_range(z_true, g, cfg->sigma, cfg->r_min, cfg->r_max,
                                       cfg->dec_scale);
            }
            /* The scan is integrated where the robot is believed to be: the
             * sensing pose here; with the fixed-lag backbone (u_mode 2) the
             * optimised pose, once it is known (below). */
            if (cfg->u_mode != 2)
                ray_cells += orc_count_beam(cfg, Px, Py, Dx, Dy, z, hit, W, H, cells, en, ea,
                                            cap, hc, mc);
            out->z[(int64_t)e * cfg->b_max + b] = z;
            out->z_true[(int64_t)e * cfg->b_max + b] = z_true;
            out->hit[(int64_t)e * cfg->b_max + b] = (uint8_t)hit;
            if (z < dmin_meas) dmin_meas = z;
            if (z_true < dmin_true) dmin_true = z_true;
        }
        for (int b = B; b < cfg->b_max; ++b) {
            out->z[(int64_t)e * cfg->b_max + b] = cfg->r_max;
            out->z_true[(int64_t)e * cfg->b_max + b] = cfg->r_max;
            out->hit[(int64_t)e * cfg->b_max + b] = 0;
        }

        /* In-step uncertainty from the map before this scan (u_mode 1 and 2). */
        float u_scan = 0.0f, upd_w = -1.0f;
        if (cfg->u_mode == 1)
            u_scan = (float)orc_scan_uncertainty(cfg, st, e, x, y, th);
        if (cfg->u_mode == 2)
            u_scan = (float)orc_slam_backbone(cfg, st, e, x, y, th, v * cfg->dt, w * cfg->dt,
                                              out->z + (int64_t)e * cfg->b_max, &upd_w);
        if (cfg->u_mode == 2 && !cfg->slam_weighted)
            upd_w = -1.0f;
        if (st->slam_upd_w)
            st->slam_upd_w[e] = upd_w;
        if (cfg->u_mode == 2) {
            /* Sec. III-D: the scan enters the occupancy grid once the window
             * optimisation has aligned it: every beam of this scan, with its
             * measured range, walked from the window's newest optimised pose
             * (its heading rotating the beams). */
            const float *xe = st->win_x + ((int64_t)e * cfg->slam_window + st->win_n[e] - 1) * 3;
            float se, ce;
            orc_sincosf(xe[2], &se, &ce);
            for (int b = 0; b < B; ++b) {
                int32_t Px, Py, Dx, Dy;
                orc_ray_setup(xe[0], xe[1], ce, se, cb_tab[b], sb_tab[b], cfg->res, &Px, &Py,
                              &Dx, &Dy);
                const int64_t r = (int64_t)e * cfg->b_max + b;
                ray_cells += orc_count_beam(cfg, Px, Py, Dx, Dy, out->z[r], out->hit[r], W, H,
                                            cells, en, ea, cap, hc, mc);
            }
        }
        free(cells);

        /* Map update: per-step sum of increments, then one clamp per cell. */
        int16_t *L = st->belief + off;
        double h_prev = orc_map_entropy(L, ncell, cfg->logodds_scale);
        for (int64_t k = 0; k < ncell; ++k) {
            if (out->cnt_h) {
                out->cnt_h[off + k] = hc[k];
                out->cnt_m[off + k] = mc[k];
            }
            if (hc[k] == 0 && mc[k] == 0)
                continue;
            int32_t d = hc[k] * cfg->hit_q + mc[k] * cfg->miss_q;
            if (upd_w >= 0.0f)
                d = (int32_t)rintf(upd_w * (float)d);     /* confidence-weighted scan */
            int32_t nl = (int32_t)L[k] + d;
            if (nl > cfg->clamp_q) nl = cfg->clamp_q;
            if (nl < -cfg->clamp_q) nl = -cfg->clamp_q;
            L[k] = (int16_t)nl;
        }
        free(hc);
        free(mc);
        double h_new = orc_map_entropy(L, ncell, cfg->logodds_scale);

        /* Collision (Sec. IV-A: closer than d_crash to an obstacle). */
        int col = col_cell || (dmin_true < cfg->d_crash);

        /* Visit grid at the ground-truth position (Eq. 8-9). */
        int32_t Vw, Vh;
        orc_visit_dims(W, H, cfg->res, cfg->visit_cell, &Vw, &Vh);
        float vx0 = -0.5f * ((float)W * cfg->res), vy0 = -0.5f * ((float)H * cfg->res);
        int32_t vi = (int32_t)floorf((x - vx0) / cfg->visit_cell);
        int32_t vj = (int32_t)floorf((y - vy0) / cfg->visit_cell);
        vi = vi < 0 ? 0 : (vi >= Vw ? Vw - 1 : vi);
        vj = vj < 0 ? 0 : (vj >= Vh ? Vh - 1 : vj);
        int32_t *vcell = st->visit + cfg->visit_off[e] + (int64_t)vj * Vw + vi;
        double dcells;
        if (*vcell < 0)
            dcells = 1.0;
        else
            dcells = orc_clip(0.5 * (double)(st->t[e] - *vcell) / (double)cfg->t_episode, 0.0, 1.0);
        *vcell = st->t[e];

        /* Reward, Eq. 7-17. */
        double Up = st->u_prev[e];
        double U = cfg->u_mode != 0 ? (double)u_scan : (u_in ? (double)u_in[e] : 0.0);
        double cgate = orc_clip((cfg->u_hi - Up) / cfg->u_hi, 0.0, 1.0);
        cgate = cgate * cgate;                                      /* Eq. 11 */
        double iota = orc_clip(fmax(Up - U, 0.0) / cfg->kappa, 0.0, 1.0); /* Eq. 12 */
        double I = cgate + (1.0 - cgate) * iota;                    /* Eq. 10 */
        double r_explore = cfg->lam_explore * dcells * I;           /* Eq. 8 */
        double r_abs = cfg->lam_abs * exp(Up) * Up;                 /* Eq. 13 */
        double r_delta = cfg->lam_delta * exp(Up) * (Up - U);       /* Eq. 14 */
        double alpha = orc_clip(((double)dmin_meas - cfg->d_crash) /
                                ((double)cfg->d_full - cfg->d_crash), 0.0, 1.0); /* Eq. 15 */
        double r_explore_s = r_explore * alpha;                     /* Eq. 16 */
        double r_delta_s = (Up - U > 0.0) ? r_delta * alpha : r_delta; /* Eq. 17 */
        double R = col ? -cfg->lam_col : (r_explore_s - r_abs + r_delta_s); /* Eq. 7 */

        double *tm = out->terms + (int64_t)e * ORC_NT;
        tm[0] = h_prev - h_new;
        tm[1] = dcells;
        tm[2] = I;
        tm[3] = alpha;
        tm[4] = r_explore_s;
        tm[5] = r_abs;
        tm[6] = r_delta_s;
        tm[7] = R;
        tm[8] = (double)col;
        tm[9] = (double)dmin_meas;
        tm[10] = (double)dmin_true;
        tm[11] = h_new;
        out->reward_ent[e] = (float)(h_prev - h_new);
        out->reward_comp[e] = (float)R;
        out->ray_cells[e] = ray_cells;
        out->gt_cells[e] = gt_cells;

        /* Observation, Eq. 3: ranges, yaw, U_t. */
        float *o = out->obs + (int64_t)e * (cfg->b_max + 2);
        for (int b = 0; b < cfg->b_max; ++b)
            o[b] = out->z[(int64_t)e * cfg->b_max + b];
        o[cfg->b_max] = th;
        o[cfg->b_max + 1] = (float)U;

        st->done[e] = (uint8_t)(col || st->t[e] >= cfg->t_episode);
        st->u_prev[e] = (float)U;
        st->g[e] += 1;
    }
    return 0;
}
