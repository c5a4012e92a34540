/*
 * raycast3d_oracle.c -- plain CPU oracle of the 3-D voxel variant of the
 * environment step (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA
 * path).
 *
 * The robot moves in the plane exactly as in the 2-D step (Euler unicycle);
 * a multi-ring LiDAR mounted at height z_s casts R rings x A azimuths of
 * beams (elevations evenly spaced over [el_min, el_max], both ends included;
 * azimuths b*2*pi/A rotated by the heading) into a W x H x D voxel world.
 * Traversal, ranges, noise, the per-scan sum-then-clamp log-odds update,
 * the entropy (now over voxels) and the Eq. 7-17 reward follow the 2-D
 * definitions; the traversal visits voxels in the order of the exact ray
 * parameter at which it crosses voxel faces, ties taken Z first, then Y,
 * then X.  Voxel (i, j, k) has flat index (k*H + j)*W + i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* from aslam_oracle.c (same oracle library) */
void orc_sincosf(float x, float *s, float *c);
float orc_gauss(uint64_t seed, uint32_t env, uint32_t step, uint32_t beam);
double orc_cell_entropy(double l);
void orc_visit_dims(int32_t W, int32_t H, float res, float vc, int32_t *Vw, int32_t *Vh);
float orc_measured_range(float z_true, float g, float sigma, float r_min, float r_max,
                         float dec_scale);

static int64_t o3_floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0)))
        q -= 1;
    return q;
}

static int64_t o3_first_gap(int32_t P, int32_t D)
{
    int64_t cell = o3_floordiv(P, 65536);
    if (D > 0)
        return (cell + 1) * 65536 - (int64_t)P;
    return (int64_t)P - cell * 65536;
}

static int o3_within(int64_t n, int64_t ad, int64_t T)
{
    return (i128)n * ((i128)1 << 30) <= (i128)T * (i128)ad;
}

/* Visits the voxels of one ray (origin Q16 voxel units, direction Q30) for
 * crossings with parameter <= T (Q16 voxels); at equal parameter the Z face
 * is crossed first, then Y, then X.  Stops at the first crossing that leaves
 * the W x H x D volume (*left = 1).  Returns the voxels written. */
int orc_walk3d(int32_t Px, int32_t Py, int32_t Pz, int32_t Dx, int32_t Dy, int32_t Dz,
               int64_t T, int32_t W, int32_t H, int32_t Dd, int64_t *cells, int64_t *enter_n,
               int64_t *enter_ad, int cap, int *left)
{
    int64_t p[3] = {o3_floordiv(Px, 65536), o3_floordiv(Py, 65536), o3_floordiv(Pz, 65536)};
    const int64_t lim[3] = {W, H, Dd};
    const int32_t P[3] = {Px, Py, Pz}, D[3] = {Dx, Dy, Dz};
    int64_t n[3], ad[3];
    int sgn[3];
    int n_out = 0;
    *left = 0;
    for (int a = 0; a < 3; ++a)
        if (p[a] < 0 || p[a] >= lim[a]) {
            *left = 1;
            return 0;
        }
    for (int a = 0; a < 3; ++a) {
        sgn[a] = (D[a] > 0) - (D[a] < 0);
        ad[a] = D[a] < 0 ? -(int64_t)D[a] : D[a];
        n[a] = o3_first_gap(P[a], D[a]);
    }
    if (n_out < cap) {
        cells[n_out] = (p[2] * H + p[1]) * W + p[0];
        enter_n[n_out] = 0;
        enter_ad[n_out] = 0;
    }
    n_out++;
    for (;;) {
        /* candidate crossings within range; pick the earliest, ties Z > Y > X */
        int best = -1;
        for (int a = 2; a >= 0; --a) {          /* Z, Y, X: earlier axis wins ties */
            if (sgn[a] == 0 || !o3_within(n[a], ad[a], T))
                continue;
            if (best < 0 || (i128)n[a] * ad[best] < (i128)n[best] * ad[a])
                best = a;
        }
        if (best < 0)
            break;
        int64_t en = n[best], ea = ad[best];
        p[best] += sgn[best];
        n[best] += 65536;
        if (p[best] < 0 || p[best] >= lim[best]) {
            *left = 1;
            break;
        }
        if (n_out < cap) {
            cells[n_out] = (p[2] * H + p[1]) * W + p[0];
            enter_n[n_out] = en;
            enter_ad[n_out] = ea;
        }
        n_out++;
    }
    return n_out;
}

typedef struct {
    int32_t n_envs, n_rings, n_az, n_spawn;
    int32_t hit_q, miss_q, clamp_q, t_episode;
    uint64_t seed;
    float res, r_max, sigma, dt, v_max, w_max, d_crash, d_full, visit_cell, sensor_z;
    float r_min, dec_scale;    /* as in the 2-D sensor */
    double el_min, el_max, logodds_scale;
    double lam_col, lam_explore, lam_abs, lam_delta, kappa, u_hi;
    const int32_t *map_w, *map_h, *map_d;
    const int64_t *map_off, *visit_off;
    const int32_t *env_id;     /* [E] index of each env in the noise stream, or NULL */
} orc_cfg3d;

typedef struct {
    const uint8_t *gt;
    int16_t *belief;
    float *x, *y, *th, *u_prev;
    int32_t *t, *g, *ep;
    uint8_t *done;
    int32_t *visit;
    const float *spawn;
} orc_state3d;

typedef struct {
    float *z, *z_true;         /* [E, B] */
    uint8_t *hit;
    int32_t *cnt_h, *cnt_m;    /* [sum cells] or NULL */
    double *terms;             /* [E, 12] */
    float *obs;                /* [E, B + 2] */
    int64_t *ray_cells, *gt_cells;
} orc_out3d;

static double o3_clip(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Beam directions: per ring (cos el, sin el), per azimuth (cos b, sin b). */
void orc_beams3d(int R, int A, double el_min, double el_max, float *ce, float *se, float *cb,
                 float *sb)
{
    const double two_pi = 2.0 * 3.14159265358979323846;
    for (int r = 0; r < R; ++r) {
        double el = R == 1 ? el_min : el_min + ((double)r * (el_max - el_min)) / (double)(R - 1);
        ce[r] = (float)cos(el);
        se[r] = (float)sin(el);
    }
    for (int a = 0; a < A; ++a) {
        double b = (two_pi * (double)a) / (double)A;
        cb[a] = (float)cos(b);
        sb[a] = (float)sin(b);
    }
}

int orc_step3d(const orc_cfg3d *cfg, orc_state3d *st, const float *actions, const float *u_in,
               orc_out3d *out)
{
    const float pi_f = (float)3.14159265358979323846;
    const float two_pi_f = (float)(2.0 * 3.14159265358979323846);
    const int R = cfg->n_rings, A = cfg->n_az, B = R * A;
    float *ce = malloc(sizeof(float) * (R + A) * 2);
    float *se = ce + R, *cb = se + R, *sb = cb + A;
    orc_beams3d(R, A, cfg->el_min, cfg->el_max, ce, se, cb, sb);
    for (int e = 0; e < cfg->n_envs; ++e) {
        const int32_t W = cfg->map_w[e], H = cfg->map_h[e], Dd = cfg->map_d[e];
        const int64_t off = cfg->map_off[e], ncell = (int64_t)W * H * Dd;
        if (st->done[e]) {
            st->ep[e] += 1;
            const float *sp = st->spawn + ((int64_t)e * cfg->n_spawn + st->ep[e] % cfg->n_spawn) * 3;
            st->x[e] = sp[0]; st->y[e] = sp[1]; st->th[e] = sp[2];
            st->t[e] = 0; st->u_prev[e] = 0.0f; st->done[e] = 0;
            memset(st->belief + off, 0, (size_t)ncell * sizeof(int16_t));
            for (int64_t v = cfg->visit_off[e]; v < cfg->visit_off[e + 1]; ++v)
                st->visit[v] = -1;
        }
        st->t[e] += 1;
        float v = fminf(fmaxf(actions[2 * e], 0.0f), cfg->v_max);
        float w = fminf(fmaxf(actions[2 * e + 1], -cfg->w_max), cfg->w_max);
        float s0, c0;
        orc_sincosf(st->th[e], &s0, &c0);
        float x = st->x[e] + (v * c0) * cfg->dt;
        float y = st->y[e] + (v * s0) * cfg->dt;
        float th = st->th[e] + w * cfg->dt;
        if (th >= pi_f) th = th - two_pi_f;
        if (th < -pi_f) th = th + two_pi_f;
        st->x[e] = x; st->y[e] = y; st->th[e] = th;
        int32_t Px = (int32_t)lrintf((x / cfg->res) * 65536.0f);
        int32_t Py = (int32_t)lrintf((y / cfg->res) * 65536.0f);
        int32_t Pz = (int32_t)lrintf((cfg->sensor_z / cfg->res) * 65536.0f);
        int64_t ri = o3_floordiv(Px, 65536), rj = o3_floordiv(Py, 65536), rk = o3_floordiv(Pz, 65536);
        int col_cell = (ri < 0 || ri >= W || rj < 0 || rj >= H || rk < 0 || rk >= Dd) ||
                       st->gt[off + (rk * H + rj) * W + ri] != 0;
        float s1, c1;
        orc_sincosf(th, &s1, &c1);
        const int cap = W + H + Dd + 4;
        int64_t *cells = malloc(sizeof(int64_t) * cap * 3);
        int64_t *en = cells + cap, *ea = cells + 2 * cap;
        int32_t *hc = calloc((size_t)ncell, sizeof(int32_t));
        int32_t *mc = calloc((size_t)ncell, sizeof(int32_t));
        const int32_t Tmax = (int32_t)lrintf((cfg->r_max / cfg->res) * 65536.0f);
        int64_t ray_cells = 0, gt_cells = 0;
        float dmin_m = cfg->r_max, dmin_t = cfg->r_max;
        for (int r = 0; r < R; ++r)
            for (int a = 0; a < A; ++a) {
                const int b = r * A + a;
                float hx = c1 * cb[a] - s1 * sb[a];
                float hy = s1 * cb[a] + c1 * sb[a];
                float dx = ce[r] * hx, dy = ce[r] * hy, dz = se[r];
                int32_t Dx = (int32_t)lrintf(dx * 1073741824.0f);
                int32_t Dy = (int32_t)lrintf(dy * 1073741824.0f);
                int32_t Dz = (int32_t)lrintf(dz * 1073741824.0f);
                int left;
                int nc = orc_walk3d(Px, Py, Pz, Dx, Dy, Dz, Tmax, W, H, Dd, cells, en, ea, cap, &left);
                int hit = 0;
                float z_true = cfg->r_max, z = cfg->r_max;
                for (int k = 0; k < nc; ++k)
                    if (st->gt[off + cells[k]]) {
                        hit = 1;
                        gt_cells += k + 1;
                        z_true = ea[k] ? (((float)en[k] / (float)ea[k]) * 16384.0f) * cfg->res : 0.0f;
                        break;
                    }
                if (!hit)
                    gt_cells += nc;
                if (hit) {
                    uint32_t eid = cfg->env_id ? (uint32_t)cfg->env_id[e] : (uint32_t)e;
                    float g = orc_gauss(cfg->seed, eid, (uint32_t)st->g[e], (uint32_t)b);
                    z = orc_measured_range(z_true, g, cfg->sigma, cfg->r_min, cfg->r_max,
                                           cfg->dec_scale);
                }
                int32_t Tz = hit ? (int32_t)lrintf((z / cfg->res) * 65536.0f) : Tmax;
                nc = orc_walk3d(Px, Py, Pz, Dx, Dy, Dz, Tz, W, H, Dd, cells, en, ea, cap, &left);
                for (int k = 0; k < nc; ++k) {
                    if (k == nc - 1 && !left && hit)
                        hc[cells[k]] += 1;
                    else
                        mc[cells[k]] += 1;
                }
                ray_cells += nc;
                out->z[(int64_t)e * B + b] = z;
                out->z_true[(int64_t)e * B + b] = z_true;
                out->hit[(int64_t)e * B + b] = (uint8_t)hit;
                if (z < dmin_m) dmin_m = z;
                if (z_true < dmin_t) dmin_t = z_true;
            }
        free(cells);
        int16_t *L = st->belief + off;
        double h_prev = 0.0, h_new = 0.0;
        for (int64_t k = 0; k < ncell; ++k)
            h_prev += orc_cell_entropy((double)L[k] * cfg->logodds_scale);
        for (int64_t k = 0; k < ncell; ++k) {
            if (out->cnt_h) {
                out->cnt_h[off + k] = hc[k];
                out->cnt_m[off + k] = mc[k];
            }
            if (hc[k] == 0 && mc[k] == 0)
                continue;
            int32_t nl = (int32_t)L[k] + hc[k] * cfg->hit_q + mc[k] * cfg->miss_q;
            if (nl > cfg->clamp_q) nl = cfg->clamp_q;
            if (nl < -cfg->clamp_q) nl = -cfg->clamp_q;
            L[k] = (int16_t)nl;
        }
        free(hc);
        free(mc);
        for (int64_t k = 0; k < ncell; ++k)
            h_new += orc_cell_entropy((double)L[k] * cfg->logodds_scale);
        int col = col_cell || (dmin_t < cfg->d_crash);
        int32_t Vw, Vh;
        orc_visit_dims(W, H, cfg->res, cfg->visit_cell, &Vw, &Vh);
        float vx0 = -0.5f * ((float)W * cfg->res), vy0 = -0.5f * ((float)H * cfg->res);
        int32_t vi = (int32_t)floorf((x - vx0) / cfg->visit_cell);
        int32_t vj = (int32_t)floorf((y - vy0) / cfg->visit_cell);
        vi = vi < 0 ? 0 : (vi >= Vw ? Vw - 1 : vi);
        vj = vj < 0 ? 0 : (vj >= Vh ? Vh - 1 : vj);
        int32_t *vc = st->visit + cfg->visit_off[e] + (int64_t)vj * Vw + vi;
        double dcells = *vc < 0 ? 1.0
                                : o3_clip(0.5 * (double)(st->t[e] - *vc) / (double)cfg->t_episode, 0.0, 1.0);
        *vc = st->t[e];
        double Up = st->u_prev[e], U = u_in ? (double)u_in[e] : 0.0;
        double cg = o3_clip((cfg->u_hi - Up) / cfg->u_hi, 0.0, 1.0);
        cg = cg * cg;
        double iota = o3_clip(fmax(Up - U, 0.0) / cfg->kappa, 0.0, 1.0);
        double I = cg + (1.0 - cg) * iota;
        double r_explore = cfg->lam_explore * dcells * I;
        double r_abs = cfg->lam_abs * exp(Up) * Up;
        double r_delta = cfg->lam_delta * exp(Up) * (Up - U);
        double alpha = o3_clip(((double)dmin_m - cfg->d_crash) / ((double)cfg->d_full - cfg->d_crash), 0.0, 1.0);
        double r_explore_s = r_explore * alpha;
        double r_delta_s = (Up - U > 0.0) ? r_delta * alpha : r_delta;
        double Rw = col ? -cfg->lam_col : (r_explore_s - r_abs + r_delta_s);
        double *tm = out->terms + (int64_t)e * 12;
        tm[0] = h_prev - h_new; tm[1] = dcells; tm[2] = I; tm[3] = alpha;
        tm[4] = r_explore_s; tm[5] = r_abs; tm[6] = r_delta_s; tm[7] = Rw;
        tm[8] = (double)col; tm[9] = (double)dmin_m; tm[10] = (double)dmin_t; tm[11] = h_new;
        out->ray_cells[e] = ray_cells;
        out->gt_cells[e] = gt_cells;
        float *o = out->obs + (int64_t)e * (B + 2);
        for (int b = 0; b < B; ++b)
            o[b] = out->z[(int64_t)e * B + b];
        o[B] = th;
        o[B + 1] = (float)U;
        st->done[e] = (uint8_t)(col || st->t[e] >= cfg->t_episode);
        st->u_prev[e] = (float)U;
        st->g[e] += 1;
    }
    free(ce);
    return 0;
}
