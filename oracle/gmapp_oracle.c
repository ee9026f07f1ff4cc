/*
 * G-MAPP oracle: a plain, slow, obviously correct CPU implementation of the
 * perception -> rollout -> cost hot path, written from the paper's equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file; only the tests, the smoke check and the bench's CPU
 * baseline do.  It shares no source with the CUDA library.
 *
 * Precision: the rollout, force and cost run in binary64.  The perception
 * filter is defined as an exact binary32 operation sequence (the paper fixes no
 * precision for it; the GPU filter must match it bit for bit), so that part is
 * written with `float` operands.  This file is compiled with
 * -ffp-contract=off on x86-64 (SSE2, FLT_EVAL_METHOD == 0), so every float
 * + - * / below is one correctly rounded binary32 operation and no multiply is
 * fused into an add.
 *
 * Section references are to the paper (G-MAPP, arXiv 2606.12579):
 *   Sec. IV-B / Sec. V-A  perception: transform, workspace crop, voxel grid
 *                         at edge 2 r_O, voxel centres -> sphere world S_W
 *   Eq. (mfi)             circular-field (MFI) repulsive force
 *   Eq. (apf)             artificial-potential-field (APF) repulsive force
 *   Alg. 1                per-obstacle clamp max(d - (r_a + r_O), eps),
 *                         detection gate d <= r_d, k_f scaling, sum over S_W
 *   Sec. IV-A             F = f_a + f_r, f_a = K e - D v, vdot = I F,
 *                         v_k = v_{k-1} + 1/2 dt vdot, p_{k+1} = p_k + dt v_k
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#pragma STDC FP_CONTRACT OFF

/* ------------------------------------------------------------------------ */
/* Perception filter (Sec. IV-B, Sec. V-A)                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t key;
    uint32_t idx;
} key_idx;

static int cmp_key_idx(const void *a, const void *b)
{
    const key_idx *x = (const key_idx *)a, *y = (const key_idx *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/*
 * Camera-frame cloud -> sorted occupied voxels and their centres.
 *
 *   world point   w_a = ((T[a][0] x + T[a][1] y) + T[a][2] z) + T[a][3]
 *   kept iff      x, y, z finite and, per axis, 0 <= (w_a - lo_a) / voxel < dims_a
 *   voxel index   i_a = floor((w_a - lo_a) / voxel)
 *   linear key    (i_z dims_y + i_y) dims_x + i_x
 *   centre        lo_a + ((float) i_a + 0.5) voxel          (r_O = voxel / 2)
 *
 * Points are grouped by key (sort by key, then by index); a voxel is kept when
 * it holds at least min_pts points.  Output is in ascending key order, with
 * the number of points and the smallest original point index per voxel.
 * Returns the number of kept voxels; only the first `cap` are written.
 */

/* Append (key, idx0 + i) of every kept point of one cloud to kv; returns the
 * number appended. */
static int64_t collect_keys(const float *xyz, int64_t n_raw, const float *T, const float *lo,
                            float voxel, const int32_t *dims, uint32_t idx0, key_idx *kv)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n_raw; ++i) {
        float x = xyz[3 * i + 0], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) continue;
        int64_t ix[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            float t0 = T[4 * a + 0] * x;
            float t1 = T[4 * a + 1] * y;
            float t2 = T[4 * a + 2] * z;
            float w = ((t0 + t1) + t2) + T[4 * a + 3];
            float q = (w - lo[a]) / voxel;
            if (!(q >= 0.0f && q < (float)dims[a])) { inside = 0; break; }
            ix[a] = (int64_t)floorf(q);
        }
        if (!inside) continue;
        uint64_t key = ((uint64_t)ix[2] * (uint64_t)dims[1] + (uint64_t)ix[1]) * (uint64_t)dims[0]
                       + (uint64_t)ix[0];
        kv[m].key = (uint32_t)key;
        kv[m].idx = idx0 + (uint32_t)i;
        ++m;
    }
    return m;
}

/* Sort the m (key, index) pairs and emit the voxels with >= min_pts points. */
static int64_t group_voxels(key_idx *kv, int64_t m, const float *lo, float voxel,
                            const int32_t *dims, int32_t min_pts, int64_t cap, uint32_t *keys,
                            uint32_t *counts, uint32_t *rep_idx, float *cx, float *cy, float *cz)
{
    qsort(kv, (size_t)m, sizeof(key_idx), cmp_key_idx);
    int64_t n_out = 0;
    int64_t r = 0;
    while (r < m) {
        int64_t e = r;
        while (e < m && kv[e].key == kv[r].key) ++e;
        uint32_t cnt = (uint32_t)(e - r);
        if ((int64_t)cnt >= (int64_t)min_pts) {
            if (n_out < cap) {
                uint32_t key = kv[r].key;
                uint32_t i_x = key % (uint32_t)dims[0];
                uint32_t i_y = (key / (uint32_t)dims[0]) % (uint32_t)dims[1];
                uint32_t i_z = key / ((uint32_t)dims[0] * (uint32_t)dims[1]);
                keys[n_out] = key;
                counts[n_out] = cnt;
                rep_idx[n_out] = kv[r].idx; /* smallest index: sorted by idx within key */
                cx[n_out] = lo[0] + ((float)i_x + 0.5f) * voxel;
                cy[n_out] = lo[1] + ((float)i_y + 0.5f) * voxel;
                cz[n_out] = lo[2] + ((float)i_z + 0.5f) * voxel;
            }
            ++n_out;
        }
        r = e;
    }
    return n_out;
}

int64_t oracle_filter(const float *xyz, int64_t n_raw, const float *T,
                      const float *lo, float voxel, const int32_t *dims,
                      int32_t min_pts, int64_t cap, uint32_t *keys,
                      uint32_t *counts, uint32_t *rep_idx, float *cx,
                      float *cy, float *cz)
{
    key_idx *kv = (key_idx *)malloc((size_t)(n_raw > 0 ? n_raw : 1) * sizeof(key_idx));
    int64_t m = collect_keys(xyz, n_raw, T, lo, voxel, dims, 0u, kv);
    int64_t n_out = group_voxels(kv, m, lo, voxel, dims, min_pts, cap, keys, counts, rep_idx,
                                 cx, cy, cz);
    free(kv);
    return n_out;
}

/*
 * Several sensors into one obstacle set (Sec. IV-B: the clouds of N_S
 * sensors, each with its own camera-to-world transform, fused into one
 * voxel grid).  xyz holds the clouds one after another ([sum n_s][3]); point
 * i of sensor s has the index offset_s + i (offset_s = n_0 + ... + n_{s-1}),
 * so a voxel's smallest index is taken over all sensors.  T holds one 3x4
 * transform per sensor ([n_sensors][12]).  Everything else as oracle_filter.
 */
int64_t oracle_filter_fused(const float *xyz, const int64_t *n_s, const float *T,
                            int32_t n_sensors, const float *lo, float voxel,
                            const int32_t *dims, int32_t min_pts, int64_t cap,
                            uint32_t *keys, uint32_t *counts, uint32_t *rep_idx, float *cx,
                            float *cy, float *cz)
{
    int64_t total = 0;
    for (int32_t s = 0; s < n_sensors; ++s) total += n_s[s];
    key_idx *kv = (key_idx *)malloc((size_t)(total > 0 ? total : 1) * sizeof(key_idx));
    int64_t m = 0, off = 0;
    for (int32_t s = 0; s < n_sensors; ++s) {
        m += collect_keys(xyz + 3 * off, n_s[s], T + 12 * s, lo, voxel, dims, (uint32_t)off,
                          kv + m);
        off += n_s[s];
    }
    int64_t n_out = group_voxels(kv, m, lo, voxel, dims, min_pts, cap, keys, counts, rep_idx,
                                 cx, cy, cz);
    free(kv);
    return n_out;
}

/* ------------------------------------------------------------------------ */
/* Circular-field repulsion (Eq. mfi, Alg. 1)                                */
/* ------------------------------------------------------------------------ */

/*
 * Per-agent obstacle sum of Alg. 1 for the MFI heuristic with a fixed current.
 * For every obstacle j of S_W:
 *   d_j = |p - p_Oj|,  s_j = max(d_j - (r_a + r_O), eps)
 *   contributes 1 / s_j when s_j <= r_d (detection gate), else nothing.
 * W = sum of the contributions.  m = min_j (d_j - r_a - r_O) is the clearance
 * to the nearest obstacle surface, unclamped.
 */
static void cf_weight(const double p[3], int64_t n_obs, const double *ox,
                      const double *oy, const double *oz, double R, double eps,
                      double r_d, double *W, double *m)
{
    double w = 0.0, mn = INFINITY;
    for (int64_t j = 0; j < n_obs; ++j) {
        double dx = p[0] - ox[j], dy = p[1] - oy[j], dz = p[2] - oz[j];
        double d = sqrt(dx * dx + dy * dy + dz * dz);
        double s = d - R;
        if (s < mn) mn = s;
        if (s < eps) s = eps;
        if (s <= r_d) w += 1.0 / s;
    }
    *W = w;
    *m = mn;
}

/*
 * Direction factor of Eq. (mfi) for static obstacles (d-dot = -v):
 *   (d-dot / |d-dot|) x (c x d-dot) = v_hat x (c x v) = (|v|^2 c - v (v . c)) / |v|
 * (the factor is even in d-dot).  Zero when |v|^2 < 1e-30.
 */
static void cf_direction(const double v[3], const double c[3], double g[3])
{
    double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (vv < 1e-30) { g[0] = g[1] = g[2] = 0.0; return; }
    double vc = v[0] * c[0] + v[1] * c[1] + v[2] * c[2];
    double nv = sqrt(vv);
    for (int a = 0; a < 3; ++a) g[a] = (vv * c[a] - v[a] * vc) / nv;
}

/*
 * Repulsive force of each agent at a given state (p, v):
 *   f_r = rho k_r W g      (k_f = rho k_r)
 * Layouts: p, v, c, f_r are [3][n_agents] (row per axis); the rest [n_agents].
 */
void oracle_cf_eval(int64_t n_obs, const double *ox, const double *oy,
                    const double *oz, double r_O, int64_t n_agents,
                    const double *p, const double *v, const double *c,
                    const double *k_r, const double *r_d, const double *r_a,
                    double rho, double eps, double *W, double *m, double *f_r)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < n_agents; ++i) {
        double pi[3] = {p[i], p[n_agents + i], p[2 * n_agents + i]};
        double vi[3] = {v[i], v[n_agents + i], v[2 * n_agents + i]};
        double ci[3] = {c[i], c[n_agents + i], c[2 * n_agents + i]};
        double w, mn, g[3];
        cf_weight(pi, n_obs, ox, oy, oz, r_a[i] + r_O, eps, r_d[i], &w, &mn);
        cf_direction(vi, ci, g);
        W[i] = w;
        m[i] = mn;
        for (int a = 0; a < 3; ++a) f_r[a * n_agents + i] = rho * k_r[i] * w * g[a];
    }
}

/*
 * Per-agent obstacle sum of the APF heuristic, Eq. (apf), in the reading of
 * this implementation: for every obstacle j of S_W, with d_j = p - p_Oj and
 * the surface distance d_O = |d_j| - (r_a + r_O),
 *   gate      d_O < r_d (strict, as printed);
 *   distance  rho_j = max(|d_j|, r_a + r_O + eps) -- the clamp of Alg. 1
 *             applied to the surface distance, so a penetrating pair stays
 *             finite; for d_O >= eps, rho_j = |d_j| exactly as printed;
 *   term      (1/rho_j - 1/r_d) rho_j^-2 d_j / |d_j|   (0 when |d_j| = 0),
 * which for d_O >= eps is (1/|d| - 1/r_d) |d|^-3 d of Eq. (apf).
 * f = sum of the terms (the gain k_f is applied by the caller); m as in
 * cf_weight (clearance to the nearest surface, unclamped); sabs (may be
 * NULL) = sum of the term magnitudes |term_j|, the scale of the rounding
 * error of any evaluation of the sum.
 */
static void apf_force(const double p[3], int64_t n_obs, const double *ox,
                      const double *oy, const double *oz, double R, double eps,
                      double r_d, double f[3], double *m, double *sabs)
{
    double fx = 0.0, fy = 0.0, fz = 0.0, mn = INFINITY, sa = 0.0;
    for (int64_t j = 0; j < n_obs; ++j) {
        double dx = p[0] - ox[j], dy = p[1] - oy[j], dz = p[2] - oz[j];
        double d = sqrt(dx * dx + dy * dy + dz * dz);
        double dO = d - R;
        if (dO < mn) mn = dO;
        if (!(dO < r_d) || d == 0.0) continue;
        double rho = d > R + eps ? d : R + eps;
        double coef = (1.0 / rho - 1.0 / r_d) / (rho * rho) / d;
        fx += coef * dx;
        fy += coef * dy;
        fz += coef * dz;
        sa += fabs(coef) * d;
    }
    f[0] = fx;
    f[1] = fy;
    f[2] = fz;
    *m = mn;
    if (sabs) *sabs = sa;
}

/*
 * MFI with the current projected per obstacle (Eq. (mfi) with the current
 * of the equation that follows it), static obstacles, so the relative
 * velocity is d' = -v.  For every obstacle j, with d_j = p - p_Oj:
 *   n_j   = d_j / |d_j|                      surface normal (the term is even in n_j)
 *   c_j   = d' - n_j (n_j . d')              current projected onto the surface
 *   s_j   = max(|d_j| - (r_a + r_O), eps)    clamp of Alg. 1
 *   term  = (1 / s_j) (d' / |d'|) x (c_j x d')   when s_j <= r_d (gate of Alg. 1)
 * written out with the two cross products.  f = sum of the terms (k_f is
 * applied by the caller); f = 0 when |v|^2 < 1e-30; a pair with d_j = 0 has
 * no normal and adds nothing.  m as in cf_weight.
 */
static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void proj_force(const double p[3], const double v[3], int64_t n_obs, const double *ox,
                       const double *oy, const double *oz, double R, double eps, double r_d,
                       double f[3], double *m)
{
    const double dd[3] = {-v[0], -v[1], -v[2]};
    const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double ndd = sqrt(vv);
    double fx = 0.0, fy = 0.0, fz = 0.0, mn = INFINITY;
    for (int64_t j = 0; j < n_obs; ++j) {
        double d[3] = {p[0] - ox[j], p[1] - oy[j], p[2] - oz[j]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double s = dn - R;
        if (s < mn) mn = s;
        if (s < eps) s = eps;
        if (!(s <= r_d) || dn == 0.0 || vv < 1e-30) continue;
        double n[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
        double nd = n[0] * dd[0] + n[1] * dd[1] + n[2] * dd[2];
        double c[3] = {dd[0] - n[0] * nd, dd[1] - n[1] * nd, dd[2] - n[2] * nd};
        double u[3] = {dd[0] / ndd, dd[1] / ndd, dd[2] / ndd};
        double cxd[3], t[3];
        cross3(c, dd, cxd);
        cross3(u, cxd, t);
        fx += t[0] / s;
        fy += t[1] / s;
        fz += t[2] / s;
    }
    f[0] = fx;
    f[1] = fy;
    f[2] = fz;
    *m = mn;
}

/*
 * Projected-current MFI force of each agent at states (p, v):
 *   f_r = rho k_r f      (k_f = rho k_r)
 * Layouts: p, v, f_r are [3][n_agents]; the rest [n_agents].
 */
void oracle_proj_eval(int64_t n_obs, const double *ox, const double *oy,
                      const double *oz, double r_O, int64_t n_agents,
                      const double *p, const double *v, const double *k_r,
                      const double *r_d, const double *r_a, double rho, double eps,
                      double *m, double *f_r)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < n_agents; ++i) {
        double pi[3] = {p[i], p[n_agents + i], p[2 * n_agents + i]};
        double vi[3] = {v[i], v[n_agents + i], v[2 * n_agents + i]};
        double f[3], mn;
        proj_force(pi, vi, n_obs, ox, oy, oz, r_a[i] + r_O, eps, r_d[i], f, &mn);
        m[i] = mn;
        for (int a = 0; a < 3; ++a) f_r[a * n_agents + i] = rho * k_r[i] * f[a];
    }
}

/*
 * APF repulsive force of each agent at positions p:
 *   f_r = rho k_r f      (k_f = rho k_r)
 * and f_abs = |rho k_r| sum_j |term_j| (f_abs may be NULL).
 * Layouts: p, f_r are [3][n_agents]; the rest [n_agents].
 */
void oracle_apf_eval(int64_t n_obs, const double *ox, const double *oy,
                     const double *oz, double r_O, int64_t n_agents,
                     const double *p, const double *k_r, const double *r_d,
                     const double *r_a, double rho, double eps, double *m, double *f_r,
                     double *f_abs)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < n_agents; ++i) {
        double pi[3] = {p[i], p[n_agents + i], p[2 * n_agents + i]};
        double f[3], mn, sa;
        apf_force(pi, n_obs, ox, oy, oz, r_a[i] + r_O, eps, r_d[i], f, &mn, &sa);
        m[i] = mn;
        if (f_abs) f_abs[i] = fabs(rho * k_r[i]) * sa;
        for (int a = 0; a < 3; ++a) f_r[a * n_agents + i] = rho * k_r[i] * f[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Rollout (Sec. IV-A) with the running cost accumulators                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double goal[3];
    double dt;            /* delta_t */
    int64_t n_steps;      /* N_k */
    double damping;       /* D = damping * I_3 */
    double inv_mass;      /* inertia tensor = inv_mass * I_3 */
    double rho;           /* k_f = rho * k_r */
    double eps;           /* clamp of Alg. 1 */
    double vel_half;      /* the 1/2 of the velocity update */
    double clear_margin;  /* softplus clearance penalty margin */
    double clear_beta;    /* softplus sharpness */
} oracle_params;

/* softplus_beta(x) = log(1 + exp(beta x)) / beta, evaluated without overflow */
static double softplus(double x, double beta)
{
    double bx = beta * x;
    if (bx > 0.0) return (bx + log1p(exp(-bx))) / beta;
    return log1p(exp(bx)) / beta;
}

/*
 * N_a independent point-mass agents, N_k steps each.  Step k (0-based):
 *   W, m  <- Alg. 1 sum at p_k                          (clearance m_k)
 *   F     = k_a (p_goal - p_k) - D v_{k-1} + rho k_r W g(v_{k-1}, c)
 *   v_k   = v_{k-1} + vel_half dt inv_mass F
 *   p_k+1 = p_k + dt v_k
 *   L    += |p_k+1 - p_k|;   pen += softplus(margin - m_k);   mc = min(mc, m_k)
 * The trajectory holds p_0 .. p_N_k (N_k + 1 points).
 * Heterogeneous ensemble: the last n_apf agents use the APF heuristic
 * instead, F = k_a (p_goal - p_k) - D v_{k-1} + rho k_r f_apf(p_k), with
 * |f_apf| in the w trace; the n_proj agents before them use MFI with the
 * projected current, F = ... + rho k_r f_proj(p_k, v_{k-1}), |f_proj| in the
 * w trace.
 * Layouts: agent vectors [3][n_agents]; traj [n_agents][n_steps+1][3];
 * w_trace, m_trace [n_agents][n_steps].  traj / traces may be NULL.
 */
void oracle_rollout(int64_t n_obs, const double *ox, const double *oy,
                    const double *oz, double r_O, int64_t n_agents,
                    const double *p0, const double *v0, const double *c,
                    const double *k_r, const double *k_a, const double *r_d,
                    const double *r_a, const oracle_params *prm, double *traj,
                    double *p_final, double *v_final, double *path_len,
                    double *clear_pen, double *min_clear, double *w_trace,
                    double *m_trace, int64_t n_apf, int64_t n_proj)
{
    const int64_t N = prm->n_steps;
#pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < n_agents; ++i) {
        double p[3] = {p0[i], p0[n_agents + i], p0[2 * n_agents + i]};
        double v[3] = {v0[i], v0[n_agents + i], v0[2 * n_agents + i]};
        double ci[3] = {c[i], c[n_agents + i], c[2 * n_agents + i]};
        double L = 0.0, pen = 0.0, mc = INFINITY;
        if (traj) for (int a = 0; a < 3; ++a) traj[(i * (N + 1)) * 3 + a] = p[a];
        const int apf = i >= n_agents - n_apf;
        const int proj = !apf && i >= n_agents - n_apf - n_proj;
        for (int64_t k = 0; k < N; ++k) {
            double w, mn, g[3], F[3], pn[3];
            if (proj) {
                proj_force(p, v, n_obs, ox, oy, oz, r_a[i] + r_O, prm->eps, r_d[i], g, &mn);
                w = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                for (int a = 0; a < 3; ++a)
                    F[a] = k_a[i] * (prm->goal[a] - p[a]) - prm->damping * v[a]
                           + prm->rho * k_r[i] * g[a];
            } else if (apf) {
                apf_force(p, n_obs, ox, oy, oz, r_a[i] + r_O, prm->eps, r_d[i], g, &mn, NULL);
                w = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                for (int a = 0; a < 3; ++a)
                    F[a] = k_a[i] * (prm->goal[a] - p[a]) - prm->damping * v[a]
                           + prm->rho * k_r[i] * g[a];
            } else {
                cf_weight(p, n_obs, ox, oy, oz, r_a[i] + r_O, prm->eps, r_d[i], &w, &mn);
                cf_direction(v, ci, g);
                for (int a = 0; a < 3; ++a)
                    F[a] = k_a[i] * (prm->goal[a] - p[a]) - prm->damping * v[a]
                           + prm->rho * k_r[i] * w * g[a];
            }
            for (int a = 0; a < 3; ++a) v[a] = v[a] + prm->vel_half * prm->dt * prm->inv_mass * F[a];
            for (int a = 0; a < 3; ++a) pn[a] = p[a] + prm->dt * v[a];
            double dx = pn[0] - p[0], dy = pn[1] - p[1], dz = pn[2] - p[2];
            L += sqrt(dx * dx + dy * dy + dz * dz);
            pen += softplus(prm->clear_margin - mn, prm->clear_beta);
            if (mn < mc) mc = mn;
            if (w_trace) w_trace[i * N + k] = w;
            if (m_trace) m_trace[i * N + k] = mn;
            for (int a = 0; a < 3; ++a) p[a] = pn[a];
            if (traj) for (int a = 0; a < 3; ++a) traj[(i * (N + 1) + k + 1) * 3 + a] = p[a];
        }
        for (int a = 0; a < 3; ++a) {
            p_final[a * n_agents + i] = p[a];
            v_final[a * n_agents + i] = v[a];
        }
        path_len[i] = L;
        clear_pen[i] = pen;
        min_clear[i] = mc;
    }
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the rollout and cost (reverse-mode derivative of the  */
/* step map of Sec. IV-A with the Alg. 1 sum and the cost sums)               */
/* ------------------------------------------------------------------------ */

/*
 * W, its gradient with respect to p, the clearance m and its gradient.
 * A pair contributes to the gradient only when it is gated in and not
 * clamped (the clamp and the gate are flat there); the clearance gradient
 * is the unit vector from the nearest obstacle centre (first index on ties).
 * Also counts clamped and gated-in pairs (the branch signature of the step).
 */
static void cf_weight_grad(const double p[3], int64_t n_obs, const double *ox,
                           const double *oy, const double *oz, double R, double eps,
                           double r_d, double *W, double gW[3], double *m, double gm[3],
                           int64_t *n_clamped, int64_t *n_gated, int64_t *jstar)
{
    double w = 0.0, best = INFINITY;
    int64_t jb = -1, nc = 0, ng = 0;
    gW[0] = gW[1] = gW[2] = 0.0;
    for (int64_t j = 0; j < n_obs; ++j) {
        double dx = p[0] - ox[j], dy = p[1] - oy[j], dz = p[2] - oz[j];
        double d = sqrt(dx * dx + dy * dy + dz * dz);
        double s = d - R;
        if (d < best) { best = d; jb = j; }
        int clamped = s < eps;
        if (clamped) s = eps;
        if (s <= r_d) {
            ++ng;
            w += 1.0 / s;
            if (!clamped) {
                double q = -1.0 / (s * s * d);
                gW[0] += q * dx;
                gW[1] += q * dy;
                gW[2] += q * dz;
            } else {
                ++nc;
            }
        }
    }
    *W = w;
    *m = best - R;
    gm[0] = gm[1] = gm[2] = 0.0;
    if (jb >= 0 && best > 0.0) {
        gm[0] = (p[0] - ox[jb]) / best;
        gm[1] = (p[1] - oy[jb]) / best;
        gm[2] = (p[2] - oz[jb]) / best;
    }
    if (n_clamped) *n_clamped = nc;
    if (n_gated) *n_gated = ng;
    if (jstar) *jstar = jb;
}

typedef struct {
    double w_path, w_goal, w_clear;
} oracle_weights;

/*
 * Cost C_i = w_path sum_k |p_k+1 - p_k| + w_goal |p_N - p_goal|
 *          + w_clear sum_k softplus(margin - m_k)
 * and its gradient with respect to v0 (3), k_r, k_a and c (3) for each
 * agent, by the reverse sweep of the stored forward rollout:
 *   a_p <- w_goal (p_N - g)/|p_N - g|,  a_v <- 0
 *   for k = N-1 .. 0:
 *     a_vk  = a_v + dt (a_p + w_path e_k),   e_k = unit(p_k+1 - p_k)
 *     Fbar  = vel_half dt inv_mass a_vk
 *     a_v   = a_vk - D Fbar + rho k_r W_k J_g^T Fbar
 *     a_p  += -k_a Fbar + rho k_r (g_k . Fbar) grad W_k
 *             - w_clear sigmoid(beta (margin - m_k)) grad m_k
 *     dk_a += Fbar . (g - p_k);  dk_r += rho W_k (g_k . Fbar)
 *     dc   += rho k_r W_k J_gc^T Fbar
 *   dv0 = a_v
 * with g(v, c) = |v| c - (v.c) v/|v|,
 *   J_g^T F  = u (c.F) - c (u.F) - ((v.c)/|v|) (F - u (u.F)),  u = v/|v|
 *   J_gc^T F = |v| F - v (u.F).
 * sig[i] is an order-dependent hash of the per-step branch signature
 * (clamped pairs, gated-in pairs, nearest obstacle): finite differences of
 * the cost are only meaningful between runs with equal signatures.
 * Layouts: [3][n] for vector quantities, [n] for scalars; sig may be NULL.
 */
void oracle_adjoint(int64_t n_obs, const double *ox, const double *oy, const double *oz,
                    double r_O, int64_t n_agents, const double *p0, const double *v0,
                    const double *c, const double *k_r, const double *k_a, const double *r_d,
                    const double *r_a, const oracle_params *prm, const oracle_weights *wt,
                    double *cost, double *g_v0, double *g_kr, double *g_ka, double *g_c,
                    uint64_t *sig)
{
    const int64_t N = prm->n_steps;
    const double h = prm->vel_half * prm->dt * prm->inv_mass;
#pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < n_agents; ++i) {
        double *P = (double *)malloc((size_t)(N + 1) * 3 * sizeof(double));
        double *V = (double *)malloc((size_t)N * 3 * sizeof(double)); /* v_{k-1} */
        double *Wk = (double *)malloc((size_t)N * sizeof(double));
        double *GW = (double *)malloc((size_t)N * 3 * sizeof(double));
        double *Mk = (double *)malloc((size_t)N * sizeof(double));
        double *GM = (double *)malloc((size_t)N * 3 * sizeof(double));
        double p[3] = {p0[i], p0[n_agents + i], p0[2 * n_agents + i]};
        double v[3] = {v0[i], v0[n_agents + i], v0[2 * n_agents + i]};
        double ci[3] = {c[i], c[n_agents + i], c[2 * n_agents + i]};
        const double R = r_a[i] + r_O;
        double L = 0.0, pen = 0.0;
        uint64_t hsh = 1469598103934665603ull;
        for (int64_t k = 0; k < N; ++k) {
            double w, gW[3], mn, gm[3], g[3], F[3];
            int64_t nc, ng, js;
            cf_weight_grad(p, n_obs, ox, oy, oz, R, prm->eps, r_d[i], &w, gW, &mn, gm, &nc, &ng,
                           &js);
            uint64_t ev[3] = {(uint64_t)nc, (uint64_t)ng, (uint64_t)js};
            for (int t = 0; t < 3; ++t) hsh = (hsh ^ ev[t]) * 1099511628211ull;
            for (int a = 0; a < 3; ++a) {
                P[3 * k + a] = p[a];
                V[3 * k + a] = v[a];
                GW[3 * k + a] = gW[a];
                GM[3 * k + a] = gm[a];
            }
            Wk[k] = w;
            Mk[k] = mn;
            cf_direction(v, ci, g);
            for (int a = 0; a < 3; ++a)
                F[a] = k_a[i] * (prm->goal[a] - p[a]) - prm->damping * v[a] + prm->rho * k_r[i] * w * g[a];
            for (int a = 0; a < 3; ++a) v[a] += h * F[a];
            double pn[3];
            for (int a = 0; a < 3; ++a) pn[a] = p[a] + prm->dt * v[a];
            double dx = pn[0] - p[0], dy = pn[1] - p[1], dz = pn[2] - p[2];
            L += sqrt(dx * dx + dy * dy + dz * dz);
            pen += softplus(prm->clear_margin - mn, prm->clear_beta);
            for (int a = 0; a < 3; ++a) p[a] = pn[a];
        }
        for (int a = 0; a < 3; ++a) P[3 * N + a] = p[a];
        double eg[3] = {p[0] - prm->goal[0], p[1] - prm->goal[1], p[2] - prm->goal[2]};
        double dg = sqrt(eg[0] * eg[0] + eg[1] * eg[1] + eg[2] * eg[2]);
        cost[i] = wt->w_path * L + wt->w_goal * dg + wt->w_clear * pen;

        double ap[3], av[3] = {0.0, 0.0, 0.0}, dkr = 0.0, dka = 0.0, dc[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a) ap[a] = dg > 0.0 ? wt->w_goal * eg[a] / dg : 0.0;
        for (int64_t k = N - 1; k >= 0; --k) {
            const double *pk = P + 3 * k, *pk1 = P + 3 * (k + 1), *vk = V + 3 * k;
            double e[3] = {pk1[0] - pk[0], pk1[1] - pk[1], pk1[2] - pk[2]};
            double le = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            double avk[3], Fb[3];
            for (int a = 0; a < 3; ++a) {
                double ea = le > 0.0 ? e[a] / le : 0.0;
                avk[a] = av[a] + prm->dt * (ap[a] + wt->w_path * ea);
                Fb[a] = h * avk[a];
            }
            double g[3];
            cf_direction(vk, ci, g);
            double gF = g[0] * Fb[0] + g[1] * Fb[1] + g[2] * Fb[2];
            double JgF[3] = {0.0, 0.0, 0.0}, JcF[3] = {0.0, 0.0, 0.0};
            double vv = vk[0] * vk[0] + vk[1] * vk[1] + vk[2] * vk[2];
            if (vv >= 1e-30) {
                double n = sqrt(vv);
                double u[3] = {vk[0] / n, vk[1] / n, vk[2] / n};
                double cF = ci[0] * Fb[0] + ci[1] * Fb[1] + ci[2] * Fb[2];
                double uF = u[0] * Fb[0] + u[1] * Fb[1] + u[2] * Fb[2];
                double vc = vk[0] * ci[0] + vk[1] * ci[1] + vk[2] * ci[2];
                for (int a = 0; a < 3; ++a) {
                    JgF[a] = u[a] * cF - ci[a] * uF - (vc / n) * (Fb[a] - u[a] * uF);
                    JcF[a] = n * Fb[a] - vk[a] * uF;
                }
            }
            double sg = 1.0 / (1.0 + exp(-prm->clear_beta * (prm->clear_margin - Mk[k])));
            for (int a = 0; a < 3; ++a) {
                av[a] = avk[a] - prm->damping * Fb[a] + prm->rho * k_r[i] * Wk[k] * JgF[a];
                ap[a] += -k_a[i] * Fb[a] + prm->rho * k_r[i] * gF * GW[3 * k + a]
                         - wt->w_clear * sg * GM[3 * k + a];
                dka += Fb[a] * (prm->goal[a] - pk[a]);
                dc[a] += prm->rho * k_r[i] * Wk[k] * JcF[a];
            }
            dkr += prm->rho * Wk[k] * gF;
        }
        for (int a = 0; a < 3; ++a) {
            g_v0[a * n_agents + i] = av[a];
            g_c[a * n_agents + i] = dc[a];
        }
        g_kr[i] = dkr;
        g_ka[i] = dka;
        if (sig) sig[i] = hsh;
        free(P);
        free(V);
        free(Wk);
        free(GW);
        free(Mk);
        free(GM);
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
