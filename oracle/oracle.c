/*
 * CAPT oracle: a plain, slow, obviously correct CPU reference for the query path of
 * the collision-affording point tree (Ramsey, Kingston, Thomason, Kavraki,
 * "Collision-Affording Point Trees: SIMD-Amenable Nearest Neighbors for Fast Collision
 * Checking", 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the benchmark's CPU
 * baseline load this library; the product library never does.  It shares no source,
 * header, table or constant with the CUDA library.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread
 * (-ffp-contract=off: every float expression below is evaluated one rounded operation
 * at a time, in the order written; no fused multiply-add.)
 *
 * Contents and what pins each part (the tests under tests/ hold the pins):
 *   1. orc_brute_*       FP32 brute force: flag(x, r) = exists p: ((x0-p0)^2 + (x1-p1)^2)
 *                        + (x2-p2)^2 <= fl(r*r).  Lemma 1 (Sec. V-B) says the CAPT reaches
 *                        exactly this.  Pinned by hand-computed cases and by an FP64
 *                        brute force (disagreement only within 1e-6 relative of d^2 = r^2).
 *   2. orc_nearest64,    FP64 nearest neighbour (Sec. III), the hinge clearance cost and
 *      orc_clearance64   its analytic gradient.  Pinned by closed forms on one-point
 *                        clouds, d = 0 and d >= r_max cases, and central differences.
 *   3. orc_capt_*        a plain recursive CAPT following Alg. 1 (Construct, Sec. IV-A/B)
 *                        with explicit sets, queried by Alg. 3 (CollisionCheck,
 *                        Sec. IV-D).  Pinned by brute force (Lemma 1), the affordance
 *                        invariant per leaf, the r_min corner condition, leaf ranges, and
 *                        hand-derived trees.
 *   4. orc_sfc_filter    a plain Alg. 2 (Filter, Sec. IV-C).  Pinned by the 1-D special
 *                        case (greedy spacing along a line), hand-computed Morton keys,
 *                        the per-pass anchor invariant (Lemma 2) and idempotence.
 *   5. orc_fk32,         FP32 edge interpolation and serial-arm kinematics (the edge
 *      orc_edges         workload of the configuration-batch early exit, Sec. IV-D).
 *                        Pinned against an FP64 kinematics and against libm sin/cos.
 *
 * Readings of the paper where it is silent or inconsistent (each one is also taken by
 * the product library, which implements it separately):
 *   R1 Descent: right iff x_d > T_i (Alg. 1 and Alg. 3 put p_d <= T_i on the left).
 *   R2 Median: sort the subtree by (p_d, original index); B1 = first half, B2 = rest;
 *      T_i = p_d of the last element of B1.
 *   R3 Padding: pads are points at +inf in every coordinate, sorted after every real
 *      point; they never enter an affordance set or a bounding box.  A leaf whose
 *      representative is a pad keeps its afforded set z only (possibly empty).
 *   R4 Affordance: include p iff dist^2(c, p) <= (r_max (1 + 1e-5))^2, with the
 *      point-to-closed-box distance in FP64 (a superset of the exact set: always safe).
 *   R5 r_min prune: only if every cell bound is finite and the FP64 squared distance
 *      from t to the farthest corner is <= (r_min (1 - 1e-5))^2.
 *   R6 AABB = exact FP32 min/max of the stored points; empty sets reject by count.
 *   R7 Stored order of an affordance set = ascending original point index.
 *   R8 Filter: 21-bit quantisation per axis over the input cloud's box; permutations in
 *      lexicographic order (xyz, xzy, yxz, yzx, zxy, zyx), the first axis of a
 *      permutation most significant in every bit triple; order by (key, original index);
 *      keep p_j iff its FP32 squared distance to the last kept point exceeds
 *      fl(r_filter^2).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EARG (-1)
#define ORC_ENOMEM (-4)

/* ------------------------------------------------------------------------------------
 * A small parallel-for on pthreads (used by the brute-force loops only).
 * ------------------------------------------------------------------------------------ */
typedef void (*range_fn)(void *ctx, size_t lo, size_t hi);
typedef struct { range_fn fn; void *ctx; size_t lo, hi; } range_job;

static void *run_job(void *a) {
    range_job *j = (range_job *)a;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_for(range_fn fn, void *ctx, size_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if ((size_t)nthreads > n) nthreads = (int)(n ? n : 1);
    if (nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    range_job *jb = (range_job *)malloc(sizeof(range_job) * (size_t)nthreads);
    if (!th || !jb) { free(th); free(jb); fn(ctx, 0, n); return; }
    size_t chunk = (n + (size_t)nthreads - 1) / (size_t)nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        size_t lo = (size_t)t * chunk, hi = lo + chunk;
        if (lo >= n) break;
        if (hi > n) hi = n;
        jb[t].fn = fn; jb[t].ctx = ctx; jb[t].lo = lo; jb[t].hi = hi;
        if (pthread_create(&th[t], NULL, run_job, &jb[t]) != 0) { fn(ctx, lo, hi); jb[t].fn = NULL; }
        started = t + 1;
    }
    for (int t = 0; t < started; t++) if (jb[t].fn) pthread_join(th[t], NULL);
    free(th); free(jb);
}

/* ------------------------------------------------------------------------------------
 * 1. FP32 brute force
 * ------------------------------------------------------------------------------------ */

/* The squared distance of the sphere test, one rounded operation at a time. */
static float d2_f32(const float *x, const float *p) {
    float dx = x[0] - p[0];
    float dy = x[1] - p[1];
    float dz = x[2] - p[2];
    float s = dx * dx + dy * dy;
    s = s + dz * dz;
    return s;
}

typedef struct {
    const float *pts; size_t n;
    const float *centers; const float *radii; size_t S; /* S = 0: one radius per sphere */
    uint8_t *flags;
} brute_ctx;

static int brute_one(const brute_ctx *c, const float *x, float r) {
    float r2 = r * r;
    for (size_t j = 0; j < c->n; j++)
        if (d2_f32(x, c->pts + 3 * j) <= r2) return 1;
    return 0;
}

static void brute_spheres_range(void *vc, size_t lo, size_t hi) {
    brute_ctx *c = (brute_ctx *)vc;
    for (size_t i = lo; i < hi; i++) c->flags[i] = (uint8_t)brute_one(c, c->centers + 3 * i, c->radii[i]);
}

/* One flag per sphere: flags[i] = exists p in pts with the FP32 test <= fl(r_i^2). */
int orc_brute_flags(const float *pts, size_t n, const float *centers, const float *radii,
                    size_t m, uint8_t *flags, int nthreads) {
    if ((n && !pts) || (m && (!centers || !radii || !flags))) return ORC_EARG;
    brute_ctx c = {pts, n, centers, radii, 0, flags};
    parallel_for(brute_spheres_range, &c, m, nthreads);
    return ORC_OK;
}

static void brute_configs_range(void *vc, size_t lo, size_t hi) {
    brute_ctx *c = (brute_ctx *)vc;
    for (size_t k = lo; k < hi; k++) {
        uint8_t f = 0;
        for (size_t s = 0; s < c->S && !f; s++)
            f = (uint8_t)brute_one(c, c->centers + 3 * (k * c->S + s), c->radii[s]);
        c->flags[k] = f;
    }
}

/* One flag per configuration of S spheres: OR of the sphere flags (Sec. IV-D). */
int orc_brute_config_flags(const float *pts, size_t n, const float *centers, const float *radii,
                           size_t C, int S, uint8_t *flags, int nthreads) {
    if (S <= 0 || (n && !pts) || (C && (!centers || !radii || !flags))) return ORC_EARG;
    brute_ctx c = {pts, n, centers, radii, (size_t)S, flags};
    parallel_for(brute_configs_range, &c, C, nthreads);
    return ORC_OK;
}

/* FP64 squared distance d^2 for every (sphere, point)?  No: the minimum over points of
 * d^2 - r^2 in FP64 per sphere, so tests can locate spheres that sit on the boundary. */
typedef struct { const float *pts; size_t n; const float *centers; const float *radii; double *gap; } gap_ctx;
static void gap_range(void *vc, size_t lo, size_t hi) {
    gap_ctx *c = (gap_ctx *)vc;
    for (size_t i = lo; i < hi; i++) {
        const float *x = c->centers + 3 * i;
        double r = c->radii[i], best = INFINITY;
        for (size_t j = 0; j < c->n; j++) {
            const float *p = c->pts + 3 * j;
            double dx = (double)x[0] - p[0], dy = (double)x[1] - p[1], dz = (double)x[2] - p[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            double g = fabs(d2 - r * r);
            if (g < best) best = g;
        }
        c->gap[i] = best;
    }
}
/* gap[i] = min over points of |d^2 - r^2| in FP64. */
int orc_min_gap64(const float *pts, size_t n, const float *centers, const float *radii, size_t m,
                  double *gap, int nthreads) {
    if ((n && !pts) || (m && (!centers || !radii || !gap))) return ORC_EARG;
    gap_ctx c = {pts, n, centers, radii, gap};
    parallel_for(gap_range, &c, m, nthreads);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * 2. FP64 nearest neighbour and the hinge clearance cost
 * ------------------------------------------------------------------------------------ */
typedef struct {
    const float *pts; size_t n; const float *centers;
    double *dist; int64_t *idx; double *second;
} nn_ctx;

static void nn_range(void *vc, size_t lo, size_t hi) {
    nn_ctx *c = (nn_ctx *)vc;
    for (size_t i = lo; i < hi; i++) {
        const float *x = c->centers + 3 * i;
        double b1 = INFINITY, b2 = INFINITY;
        int64_t bi = -1;
        for (size_t j = 0; j < c->n; j++) {
            const float *p = c->pts + 3 * j;
            double dx = (double)x[0] - p[0], dy = (double)x[1] - p[1], dz = (double)x[2] - p[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < b1) { b2 = b1; b1 = d2; bi = (int64_t)j; }
            else if (d2 < b2) b2 = d2;
        }
        c->dist[i] = sqrt(b1);
        if (c->idx) c->idx[i] = bi;
        if (c->second) c->second[i] = sqrt(b2);
    }
}

/* dist[i] = min_p ||x_i - p|| in FP64 (lowest index on ties), second = runner-up. */
int orc_nearest64(const float *pts, size_t n, const float *centers, size_t m, double *dist,
                  int64_t *idx, double *second, int nthreads) {
    if ((n && !pts) || (m && (!centers || !dist))) return ORC_EARG;
    nn_ctx c = {pts, n, centers, dist, idx, second};
    parallel_for(nn_range, &c, m, nthreads);
    return ORC_OK;
}

/* Hinge clearance over T trajectories x W waypoints x S spheres (FP64):
 *   d = min(d*, r_max) with d* the exact nearest-point distance,
 *   h = max(0, r_s + margin - d),  cost_t = sum over (w, s) of h^2,
 *   d cost_t / d c = g_t * (-2 h) * (c - p*) / d*  when h > 0 and d* < r_max and d* > 0,
 *   and 0 otherwise (d clipped to r_max has zero derivative; d* = 0 has no direction).
 * centers [T][W][S][3], radii [S], grad_cost [T] (NULL means all ones).
 * Outputs: cost [T], dist [T*W*S] (clipped d), grad [T*W*S*3] (may be NULL). */
int orc_clearance64(const float *pts, size_t n, const float *centers, const float *radii,
                    size_t T, int W, int S, double r_max, double margin, const double *grad_cost,
                    double *cost, double *dist, double *grad, int nthreads) {
    if (W <= 0 || S <= 0 || (T && (!centers || !radii || !cost || !dist))) return ORC_EARG;
    size_t m = T * (size_t)W * (size_t)S;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (m ? m : 1));
    if (!idx) return ORC_ENOMEM;
    int rc = orc_nearest64(pts, n, centers, m, dist, idx, NULL, nthreads);
    if (rc) { free(idx); return rc; }
    for (size_t t = 0; t < T; t++) {
        double g = grad_cost ? grad_cost[t] : 1.0, acc = 0.0;
        for (size_t k = 0; k < (size_t)W * (size_t)S; k++) {
            size_t i = t * (size_t)W * (size_t)S + k;
            int s = (int)(k % (size_t)S);
            double dstar = dist[i];
            double d = dstar < r_max ? dstar : r_max;
            double h = (double)radii[s] + margin - d;
            if (h < 0.0) h = 0.0;
            acc += h * h;
            dist[i] = d;
            if (grad) {
                for (int a = 0; a < 3; a++) grad[3 * i + a] = 0.0;
                if (h > 0.0 && dstar < r_max && dstar > 0.0 && idx[i] >= 0) {
                    const float *x = centers + 3 * i, *p = pts + 3 * idx[i];
                    for (int a = 0; a < 3; a++)
                        grad[3 * i + a] = g * (-2.0 * h) * (((double)x[a] - (double)p[a]) / dstar);
                }
            }
        }
        cost[t] = acc;
    }
    free(idx);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * 3. Plain CAPT: Alg. 1 (Construct) and Alg. 3 (CollisionCheck)
 * ------------------------------------------------------------------------------------ */
typedef struct orc_capt {
    size_t n, N;          /* real points, leaves (power of two, N >= 1) */
    int L;                /* descent length log2(N) */
    float *pts;           /* owned copy [n][3] */
    float *T;             /* Eytzinger split values, N - 1 */
    size_t *set_begin;    /* N + 1 offsets into set_idx */
    uint32_t *set_idx;    /* afforded point indices per leaf, ascending (R7) */
    float *aabb;          /* [N][6]: lo xyz, hi xyz of the stored points (R6) */
    double *cell;         /* [N][6]: closed cell bounds, for the tests */
    uint8_t *pruned;      /* [N]: 1 where the r_min condition stored {t} only */
    /* construction scratch */
    size_t cap, used, next_leaf;
    double thr_afford, thr_prune;
    int oom;
} orc_capt;

typedef struct { float key; uint32_t idx; } keyed;

static int cmp_keyed(const void *a, const void *b) {
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static float coord(const orc_capt *t, uint32_t i, int d) {
    return i < t->n ? t->pts[3 * (size_t)i + d] : INFINITY;   /* R3: pads sit at +inf */
}

/* "Cell c affords p at radius r" (Sec. IV-A): some q in c with ||p - q|| <= r.  For a
 * closed box the nearest q is the clamp of p; R4 widens r_max by 1e-5 relative. */
static int affords(const orc_capt *t, const double c[6], uint32_t i) {
    double s = 0.0;
    for (int d = 0; d < 3; d++) {
        double v = t->pts[3 * (size_t)i + d], q = v;
        if (q < c[d]) q = c[d];
        if (q > c[3 + d]) q = c[3 + d];
        double e = v - q;
        s = s + e * e;
    }
    return s <= t->thr_afford;
}

/* Alg. 1's leaf test negated: no q in c lies farther than r_min from t (R5). */
static int within_rmin(const orc_capt *t, const double c[6], uint32_t i) {
    double s = 0.0;
    for (int d = 0; d < 3; d++) {
        if (!isfinite(c[d]) || !isfinite(c[3 + d])) return 0;
        double v = t->pts[3 * (size_t)i + d];
        double a = fabs(v - c[d]), b = fabs(c[3 + d] - v);
        double e = a > b ? a : b;
        s = s + e * e;
    }
    return s <= t->thr_prune;
}

static int push_set(orc_capt *t, const uint32_t *p, size_t k) {
    if (t->used + k > t->cap) {
        size_t nc = t->cap ? t->cap : 1024;
        while (nc < t->used + k) nc *= 2;
        uint32_t *ns = (uint32_t *)realloc(t->set_idx, nc * sizeof(uint32_t));
        if (!ns) return 0;
        t->set_idx = ns; t->cap = nc;
    }
    memcpy(t->set_idx + t->used, p, k * sizeof(uint32_t));
    t->used += k;
    return 1;
}

/* Construct(PC = B[0..m), c, z, i, d): Alg. 1 with explicit sets. */
static void construct(orc_capt *t, const uint32_t *B, size_t m, const double c[6],
                      const uint32_t *z, size_t nz, size_t i, int d) {
    if (t->oom) return;
    if (m == 1) {
        size_t leaf = i - (t->N - 1);
        if (leaf != t->next_leaf) { t->oom = 1; return; }   /* leaves arrive in order */
        uint32_t rep = B[0];
        uint32_t *P = (uint32_t *)malloc(sizeof(uint32_t) * (nz + 1));
        if (!P) { t->oom = 1; return; }
        size_t k = 0;
        int pruned = 0;
        if (rep < t->n) {
            P[k++] = rep;
            pruned = within_rmin(t, c, rep);
        }
        if (!pruned) for (size_t j = 0; j < nz; j++) P[k++] = z[j];
        qsort(P, k, sizeof(uint32_t), cmp_u32);
        t->set_begin[leaf] = t->used;
        if (!push_set(t, P, k)) { free(P); t->oom = 1; return; }
        t->set_begin[leaf + 1] = t->used;
        float *a = t->aabb + 6 * leaf;
        for (int e = 0; e < 3; e++) { a[e] = INFINITY; a[3 + e] = -INFINITY; }
        for (size_t j = 0; j < k; j++)
            for (int e = 0; e < 3; e++) {
                float v = t->pts[3 * (size_t)P[j] + e];
                if (v < a[e]) a[e] = v;
                if (v > a[3 + e]) a[3 + e] = v;
            }
        memcpy(t->cell + 6 * leaf, c, 6 * sizeof(double));
        t->pruned[leaf] = (uint8_t)pruned;
        t->next_leaf++;
        free(P);
        return;
    }
    /* T_i = the median of p_d over the subtree (R2: rank split, index tie-break) */
    keyed *kb = (keyed *)malloc(sizeof(keyed) * m);
    uint32_t *sorted = (uint32_t *)malloc(sizeof(uint32_t) * m);
    uint32_t *z1 = (uint32_t *)malloc(sizeof(uint32_t) * (nz + m));
    uint32_t *z2 = (uint32_t *)malloc(sizeof(uint32_t) * (nz + m));
    if (!kb || !sorted || !z1 || !z2) { free(kb); free(sorted); free(z1); free(z2); t->oom = 1; return; }
    for (size_t j = 0; j < m; j++) { kb[j].key = coord(t, B[j], d); kb[j].idx = B[j]; }
    qsort(kb, m, sizeof(keyed), cmp_keyed);
    for (size_t j = 0; j < m; j++) sorted[j] = kb[j].idx;
    size_t h = m / 2;
    float Ti = kb[h - 1].key;
    t->T[i] = Ti;
    const uint32_t *B1 = sorted, *B2 = sorted + h;
    double c1[6], c2[6];
    memcpy(c1, c, sizeof(c1));
    memcpy(c2, c, sizeof(c2));
    c1[3 + d] = Ti;      /* shrink the upper bound of c1 on d to T_i */
    c2[d] = Ti;          /* raise the lower bound of c2 on d to T_i */
    size_t n1 = 0, n2 = 0;
    /* z1 = {p in z u B2 : c1 affords p at r_max},  z2 = {p in z u B1 : c2 affords p} */
    for (size_t j = 0; j < nz; j++) if (affords(t, c1, z[j])) z1[n1++] = z[j];
    for (size_t j = 0; j < h; j++) if (B2[j] < t->n && affords(t, c1, B2[j])) z1[n1++] = B2[j];
    for (size_t j = 0; j < nz; j++) if (affords(t, c2, z[j])) z2[n2++] = z[j];
    for (size_t j = 0; j < h; j++) if (B1[j] < t->n && affords(t, c2, B1[j])) z2[n2++] = B1[j];
    free(kb);
    construct(t, B1, h, c1, z1, n1, 2 * i + 1, (d + 1) % 3);
    construct(t, B2, h, c2, z2, n2, 2 * i + 2, (d + 1) % 3);
    free(z1); free(z2); free(sorted);
}

void orc_capt_free(orc_capt *t) {
    if (!t) return;
    free(t->pts); free(t->T); free(t->set_begin); free(t->set_idx);
    free(t->aabb); free(t->cell); free(t->pruned); free(t);
}

/* Build the plain CAPT of n points (float [n][3]) for radii in [r_min, r_max]. */
int orc_capt_build(const float *pts, size_t n, float r_min, float r_max, orc_capt **out) {
    if (!out || (n && !pts) || !(r_min >= 0.0f) || !(r_max >= r_min) || !isfinite(r_max)) return ORC_EARG;
    *out = NULL;
    orc_capt *t = (orc_capt *)calloc(1, sizeof(orc_capt));
    if (!t) return ORC_ENOMEM;
    size_t N = 1;
    int L = 0;
    while (N < n) { N *= 2; L++; }
    t->n = n; t->N = N; t->L = L;
    double ra = (double)r_max * (1.0 + 1e-5), rp = (double)r_min * (1.0 - 1e-5);
    t->thr_afford = ra * ra;
    t->thr_prune = rp * rp;
    t->pts = (float *)malloc(sizeof(float) * 3 * (n ? n : 1));
    t->T = (float *)malloc(sizeof(float) * (N > 1 ? N - 1 : 1));
    t->set_begin = (size_t *)calloc(N + 1, sizeof(size_t));
    t->aabb = (float *)malloc(sizeof(float) * 6 * N);
    t->cell = (double *)malloc(sizeof(double) * 6 * N);
    t->pruned = (uint8_t *)calloc(N, 1);
    uint32_t *B = (uint32_t *)malloc(sizeof(uint32_t) * N);
    if (!t->pts || !t->T || !t->set_begin || !t->aabb || !t->cell || !t->pruned || !B) {
        free(B); orc_capt_free(t); return ORC_ENOMEM;
    }
    if (n) memcpy(t->pts, pts, sizeof(float) * 3 * n);
    for (size_t j = 0; j < N; j++) B[j] = (uint32_t)j;     /* indices >= n are pads */
    double root[6] = {-INFINITY, -INFINITY, -INFINITY, INFINITY, INFINITY, INFINITY};
    construct(t, B, N, root, NULL, 0, 0, 0);
    free(B);
    if (t->oom || t->next_leaf != N) { orc_capt_free(t); return ORC_ENOMEM; }
    *out = t;
    return ORC_OK;
}

/* info[0] = N, info[1] = L, info[2] = total stored entries, info[3] = max set size,
 * info[4] = pruned leaves */
int orc_capt_info(const orc_capt *t, int64_t *info) {
    if (!t || !info) return ORC_EARG;
    size_t mx = 0, np = 0;
    for (size_t l = 0; l < t->N; l++) {
        size_t k = t->set_begin[l + 1] - t->set_begin[l];
        if (k > mx) mx = k;
        np += t->pruned[l];
    }
    info[0] = (int64_t)t->N; info[1] = t->L; info[2] = (int64_t)t->used;
    info[3] = (int64_t)mx; info[4] = (int64_t)np;
    return ORC_OK;
}

/* Copy out the arrays (any pointer may be NULL). */
int orc_capt_export(const orc_capt *t, float *T, int64_t *set_begin, uint32_t *set_idx,
                    float *aabb, double *cell, uint8_t *pruned) {
    if (!t) return ORC_EARG;
    if (T && t->N > 1) memcpy(T, t->T, sizeof(float) * (t->N - 1));
    if (set_begin) for (size_t l = 0; l <= t->N; l++) set_begin[l] = (int64_t)t->set_begin[l];
    if (set_idx && t->used) memcpy(set_idx, t->set_idx, sizeof(uint32_t) * t->used);
    if (aabb) memcpy(aabb, t->aabb, sizeof(float) * 6 * t->N);
    if (cell) memcpy(cell, t->cell, sizeof(double) * 6 * t->N);
    if (pruned) memcpy(pruned, t->pruned, t->N);
    return ORC_OK;
}

/* Alg. 3 for one sphere.  Returns the flag; *leaf = i - (N - 1); *mscan = points of the
 * affordance set examined (0 when the box test rejects; position of the first hit + 1,
 * else the set size). */
static int capt_check(const orc_capt *t, const float *x, float r, int64_t *leaf, int64_t *mscan) {
    size_t i = 0;
    int d = 0;
    while (i < t->N - 1) {                       /* exactly L steps, N is a power of two */
        if (x[d] > t->T[i]) i = 2 * i + 2;       /* R1 */
        else i = 2 * i + 1;
        d = (d + 1) % 3;
    }
    size_t l = i - (t->N - 1);
    if (leaf) *leaf = (int64_t)l;
    if (mscan) *mscan = 0;
    size_t b = t->set_begin[l], e = t->set_begin[l + 1];
    if (b == e) return 0;                        /* empty set: nothing to hit (R6) */
    float r2 = r * r;
    const float *a = t->aabb + 6 * l;
    float s = 0.0f;
    for (int k = 0; k < 3; k++) {                /* squared distance from x to A_l */
        float q = x[k];
        if (q < a[k]) q = a[k];
        if (q > a[3 + k]) q = a[3 + k];
        float g = x[k] - q;
        s = s + g * g;
    }
    if (!(s <= r2)) return 0;                    /* A_l does not intersect the sphere */
    for (size_t j = b; j < e; j++) {
        if (mscan) *mscan += 1;
        if (d2_f32(x, t->pts + 3 * (size_t)t->set_idx[j]) <= r2) return 1;
    }
    return 0;
}

/* Per-sphere queries. leaves / mscan may be NULL. */
int orc_capt_query(const orc_capt *t, const float *centers, const float *radii, size_t m,
                   uint8_t *flags, int64_t *leaves, int64_t *mscan) {
    if (!t || (m && (!centers || !radii || !flags))) return ORC_EARG;
    for (size_t i = 0; i < m; i++)
        flags[i] = (uint8_t)capt_check(t, centers + 3 * i, radii[i], leaves ? leaves + i : NULL,
                                       mscan ? mscan + i : NULL);
    return ORC_OK;
}

/* Per-configuration queries with the early exit of Sec. IV-D: spheres in order, stop at
 * the first hit.  counts (may be NULL) accumulates [spheres checked, spheres passing
 * the box test, points scanned]. */
int orc_capt_query_configs(const orc_capt *t, const float *centers, const float *radii, size_t C,
                           int S, uint8_t *flags, int64_t *counts) {
    if (!t || S <= 0 || (C && (!centers || !radii || !flags))) return ORC_EARG;
    int64_t nsph = 0, npass = 0, npts = 0;
    for (size_t k = 0; k < C; k++) {
        uint8_t f = 0;
        for (int s = 0; s < S && !f; s++) {
            int64_t ms = 0;
            f = (uint8_t)capt_check(t, centers + 3 * (k * (size_t)S + (size_t)s), radii[s], NULL, &ms);
            nsph++;
            npts += ms;
            if (ms) npass++;
        }
        flags[k] = f;
    }
    if (counts) { counts[0] += nsph; counts[1] += npass; counts[2] += npts; }
    return ORC_OK;
}

/* Clearance through the plain CAPT (exact when d <= r_max by Lemma 1, Case 1): the
 * minimum FP64 distance over the leaf's set, clipped to r_max; idx = -1 when clipped. */
int orc_capt_nearest64(const orc_capt *t, const float *centers, size_t m, double r_max,
                       double *dist, int64_t *idx) {
    if (!t || (m && (!centers || !dist))) return ORC_EARG;
    for (size_t i = 0; i < m; i++) {
        const float *x = centers + 3 * i;
        size_t k = 0;
        int d = 0;
        while (k < t->N - 1) { k = x[d] > t->T[k] ? 2 * k + 2 : 2 * k + 1; d = (d + 1) % 3; }
        size_t l = k - (t->N - 1);
        double best = INFINITY;
        int64_t bi = -1;
        for (size_t j = t->set_begin[l]; j < t->set_begin[l + 1]; j++) {
            const float *p = t->pts + 3 * (size_t)t->set_idx[j];
            double dx = (double)x[0] - p[0], dy = (double)x[1] - p[1], dz = (double)x[2] - p[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best) { best = d2; bi = t->set_idx[j]; }
        }
        double dd = sqrt(best);
        if (!(dd < r_max)) { dd = r_max; bi = -1; }
        dist[i] = dd;
        if (idx) idx[i] = bi;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * 4. Plain Alg. 2 (Filter)
 * ------------------------------------------------------------------------------------ */

/* Morton (Z-order) key of 21-bit coordinates under the axis permutation perm[0..2];
 * the bit of axis perm[0] is the most significant in every triple (R8). */
uint64_t orc_morton_key(uint32_t qx, uint32_t qy, uint32_t qz, const int *perm) {
    uint32_t q[3] = {qx, qy, qz};
    uint64_t key = 0;
    for (int b = 20; b >= 0; b--)
        for (int a = 0; a < 3; a++)
            key = (key << 1) | ((q[perm[a]] >> b) & 1u);
    return key;
}

static const int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

typedef struct { uint64_t key; uint32_t idx; } zkey;
static int cmp_zkey(const void *a, const void *b) {
    const zkey *x = (const zkey *)a, *y = (const zkey *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Filter the cloud with radius r_filter.  out_idx (n entries) receives the kept
 * indices in the last pass's curve order; *n_out their count.  trace (may be NULL,
 * 6*n entries) receives, per pass p and per position j of that pass's sorted input,
 * the original index of the kept point the j-th point was compared against (itself
 * when kept); trace_len (6 entries) the pass input sizes; trace_order (6*n) the sorted
 * input of each pass. */
int orc_sfc_filter(const float *pts, size_t n, float r_filter, uint32_t *out_idx, size_t *n_out,
                   uint32_t *trace_order, uint32_t *trace_anchor, int64_t *trace_len) {
    if (!n_out || (n && (!pts || !out_idx)) || !(r_filter >= 0.0f)) return ORC_EARG;
    *n_out = 0;
    if (n == 0) return ORC_OK;
    float lo[3], hi[3];
    for (int a = 0; a < 3; a++) { lo[a] = pts[a]; hi[a] = pts[a]; }
    for (size_t j = 0; j < n; j++)
        for (int a = 0; a < 3; a++) {
            float v = pts[3 * j + a];
            if (!isfinite(v)) return -3;
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * 3 * n);
    uint32_t *cur = (uint32_t *)malloc(sizeof(uint32_t) * n);
    zkey *zk = (zkey *)malloc(sizeof(zkey) * n);
    if (!q || !cur || !zk) { free(q); free(cur); free(zk); return ORC_ENOMEM; }
    for (size_t j = 0; j < n; j++)
        for (int a = 0; a < 3; a++) {
            double ext = (double)hi[a] - (double)lo[a];
            uint32_t v = 0;
            if (ext > 0.0) {
                double f = floor(((double)pts[3 * j + a] - (double)lo[a]) / ext * 2097152.0);
                v = f >= 2097151.0 ? 2097151u : (uint32_t)f;
            }
            q[3 * j + a] = v;
        }
    size_t m = n;
    for (size_t j = 0; j < n; j++) cur[j] = (uint32_t)j;     /* PC' <- PC */
    float rf2 = r_filter * r_filter;
    for (int p = 0; p < 6; p++) {
        for (size_t j = 0; j < m; j++) {
            uint32_t k = cur[j];
            zk[j].key = orc_morton_key(q[3 * k], q[3 * k + 1], q[3 * k + 2], PERMS[p]);
            zk[j].idx = k;
        }
        qsort(zk, m, sizeof(zkey), cmp_zkey);              /* sort PC' along the curve */
        for (size_t j = 0; j < m; j++) cur[j] = zk[j].idx;
        if (trace_order) memcpy(trace_order + (size_t)p * n, cur, m * sizeof(uint32_t));
        if (trace_len) trace_len[p] = (int64_t)m;
        size_t i = 0;
        if (trace_anchor) trace_anchor[(size_t)p * n] = cur[0];
        for (size_t j = 1; j < m; j++) {
            uint32_t pj = cur[j];
            if (d2_f32(pts + 3 * (size_t)cur[i], pts + 3 * (size_t)pj) > rf2) {
                i = i + 1;
                cur[i] = pj;
                if (trace_anchor) trace_anchor[(size_t)p * n + j] = pj;
            } else if (trace_anchor) {
                trace_anchor[(size_t)p * n + j] = cur[i];
            }
        }
        m = i + 1;                                           /* PC' <- PC'_{0..i} */
    }
    memcpy(out_idx, cur, m * sizeof(uint32_t));
    *n_out = m;
    free(q); free(cur); free(zk);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * 5. FP32 edge interpolation and serial-arm kinematics
 * ------------------------------------------------------------------------------------ */

/* sin and cos in FP32 by Cody-Waite reduction (Cody and Waite, "Software Manual for the
 * Elementary Functions", 1980) modulo pi/2, with pi/2 split into three float pieces of
 * which the first two have 12 significant bits (exact products for |k| < 2^12), then
 * Taylor polynomials on [-pi/4, pi/4] (sin to degree 9, cos to degree 10; truncation
 * below 2e-9) evaluated by Horner's rule.  Valid for |x| < 4000. */
void orc_sincos32(float x, float *s_out, float *c_out) {
    float kf = rintf(x * 0.636619746685f);
    float r = x - kf * 1.5703125f;
    r = r - kf * 4.837512969970703125e-4f;
    r = r - kf * 7.549790126404332e-8f;
    float r2 = r * r;
    float ps = 2.7557318844628753e-6f;
    ps = ps * r2 - 1.9841270113829523e-4f;
    ps = ps * r2 + 8.333333767950535e-3f;
    ps = ps * r2 - 0.1666666716337204f;
    float s = r + (r * r2) * ps;
    float pc = -2.755731998149713e-7f;
    pc = pc * r2 + 2.4801587642286904e-5f;
    pc = pc * r2 - 1.3888889225199819e-3f;
    pc = pc * r2 + 4.16666679084301e-2f;
    pc = pc * r2 - 0.5f;
    float c = 1.0f + r2 * pc;
    int k = ((int)kf) & 3;
    float so, co;
    if (k == 0) { so = s; co = c; }
    else if (k == 1) { so = c; co = -s; }
    else if (k == 2) { so = -s; co = -c; }
    else { so = -c; co = s; }
    *s_out = so;
    *c_out = co;
}

typedef struct {
    int J, S;
    const float *base;         /* [3] */
    const int32_t *axis;       /* [J] 0 = x, 1 = y, 2 = z */
    const float *link;         /* [J][3] translation after joint j, in its rotated frame */
    const int32_t *sph_link;   /* [S] */
    const float *sph_off;      /* [S][3] */
    const float *sph_r;        /* [S] */
} arm_desc;

/* R <- R * Rot(axis, q): only two columns change. */
static void rotate_cols(float R[3][3], int axis, float s, float c) {
    int a, b;                  /* the columns mixed by the rotation, in right-handed order */
    if (axis == 0) { a = 1; b = 2; }
    else if (axis == 1) { a = 2; b = 0; }
    else { a = 0; b = 1; }
    for (int r = 0; r < 3; r++) {
        float ca = R[r][a], cb = R[r][b];
        R[r][a] = c * ca + s * cb;
        R[r][b] = c * cb - s * ca;
    }
}

static void mat_vec(const float R[3][3], const float *v, float *out) {
    for (int r = 0; r < 3; r++) {
        float acc = R[r][0] * v[0] + R[r][1] * v[1];
        out[r] = acc + R[r][2] * v[2];
    }
}

static void fk_one(const arm_desc *arm, const float *q, float *centers /* [S][3] */) {
    float R[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    float p[3] = {arm->base[0], arm->base[1], arm->base[2]};
    float Rj[16][3][3], Oj[16][3];
    for (int j = 0; j < arm->J; j++) {
        float s, c;
        orc_sincos32(q[j], &s, &c);
        rotate_cols(R, arm->axis[j], s, c);
        memcpy(Rj[j], R, sizeof(R));
        memcpy(Oj[j], p, sizeof(p));
        float t[3];
        mat_vec(R, arm->link + 3 * j, t);
        for (int a = 0; a < 3; a++) p[a] = p[a] + t[a];
    }
    for (int s = 0; s < arm->S; s++) {
        int f = arm->sph_link[s];
        float t[3];
        mat_vec((const float (*)[3])Rj[f], arm->sph_off + 3 * s, t);
        for (int a = 0; a < 3; a++) centers[3 * s + a] = Oj[f][a] + t[a];
    }
}

/* Sphere centres for C configurations q [C][J] -> centers [C][S][3]. */
int orc_fk32(int J, const float *base, const int32_t *axis, const float *link, int S,
             const int32_t *sph_link, const float *sph_off, const float *q, size_t C, float *centers) {
    if (J <= 0 || J > 16 || S <= 0 || !base || !axis || !link || !sph_link || !sph_off ||
        (C && (!q || !centers))) return ORC_EARG;
    arm_desc arm = {J, S, base, axis, link, sph_link, sph_off, NULL};
    for (size_t k = 0; k < C; k++) fk_one(&arm, q + k * (size_t)J, centers + k * (size_t)S * 3);
    return ORC_OK;
}

/* The k-th of n interpolated configurations of an edge: q = qa + (k/(n-1)) (qb - qa). */
static void interp(int J, const float *qa, const float *qb, int k, int n, float *q) {
    float t = n > 1 ? (float)k / (float)(n - 1) : 0.0f;
    for (int j = 0; j < J; j++) {
        float dq = qb[j] - qa[j];
        q[j] = qa[j] + t * dq;
    }
}

int orc_interp32(int J, const float *qa, const float *qb, int n, float *q_out) {
    if (J <= 0 || !qa || !qb || !q_out) return ORC_EARG;
    for (int k = 0; k < n; k++) interp(J, qa, qb, k, n, q_out + (size_t)k * J);
    return ORC_OK;
}

typedef struct {
    const orc_capt *tree; const float *pts; size_t n;
    arm_desc arm; const float *qa, *qb; const int32_t *ns; uint8_t *valid;
} edge_ctx;

static void edges_range(void *vc, size_t lo, size_t hi) {
    edge_ctx *c = (edge_ctx *)vc;
    int J = c->arm.J, S = c->arm.S;
    float q[16], cen[64 * 3];
    for (size_t e = lo; e < hi; e++) {
        uint8_t ok = 1;
        for (int k = 0; k < c->ns[e] && ok; k++) {
            interp(J, c->qa + e * (size_t)J, c->qb + e * (size_t)J, k, c->ns[e], q);
            fk_one(&c->arm, q, cen);
            for (int s = 0; s < S && ok; s++) {
                int hit;
                if (c->tree) hit = capt_check(c->tree, cen + 3 * s, c->arm.sph_r[s], NULL, NULL);
                else {
                    brute_ctx b = {c->pts, c->n, NULL, NULL, 0, NULL};
                    hit = brute_one(&b, cen + 3 * s, c->arm.sph_r[s]);
                }
                if (hit) ok = 0;
            }
        }
        c->valid[e] = ok;
    }
}

/* Edge validity: 1 iff none of the n_e interpolated configurations collides.  With a
 * tree the sphere test is Alg. 3 on the plain CAPT; with tree == NULL it is the FP32
 * brute force over pts.  An edge with n_e <= 0 has no configuration and is valid. */
int orc_edges(const orc_capt *tree, const float *pts, size_t n, int J, const float *base,
              const int32_t *axis, const float *link, int S, const int32_t *sph_link,
              const float *sph_off, const float *sph_r, const float *qa, const float *qb,
              const int32_t *nsteps, size_t E, uint8_t *valid, int nthreads) {
    if (J <= 0 || J > 16 || S <= 0 || S > 64 || (E && (!qa || !qb || !nsteps || !valid)) ||
        (!tree && n && !pts)) return ORC_EARG;
    edge_ctx c = {tree, pts, n, {J, S, base, axis, link, sph_link, sph_off, sph_r}, qa, qb, nsteps, valid};
    parallel_for(edges_range, &c, E, nthreads);
    return ORC_OK;
}
