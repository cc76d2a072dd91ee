/*
 * FP64 CPU oracle for the data-driven S_n transport sweep (JSweep, arXiv 1803.09876).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * code, header or table with the GPU library; the two meet only through the
 * input arrays.
 *
 * What it computes, and the passages it follows:
 *   - Dependency graph per direction (Sec. II-C, Sec. V-A): vertices are
 *     (cell, direction); cell v depends on cell u when they share an interior
 *     face f and the flow in direction Omega crosses f from u into v, i.e.
 *     sign(Omega . n_f) > 0 with n_f oriented from u to v.  The sign is taken
 *     in FP64 as ((n_x*O_x) + (n_y*O_y)) + (n_z*O_z), evaluated in that order
 *     with no fused multiply-add (build with -ffp-contract=off).  A face with
 *     Omega . n_f == 0 exactly carries no dependency.
 *   - Cycle breaking: the paper leaves cycles to a pre-processing step
 *     (Sec. VI appendix; Plimpton et al.).  Rule used here: repeat {peel the
 *     acyclic part with Kahn's algorithm; on the cells left over, find the
 *     strongly connected components (Tarjan); in every component with two or
 *     more cells, drop ("lag") the active interior face with the smallest face
 *     id whose two cells both lie in the component} until nothing is left
 *     over.  A lagged face keeps its coefficients in the solve; its upwind
 *     value is the previous sweep's (zero before the first sweep).
 *   - Levels: level(v) = 0 for a cell with no active upwind neighbour, else
 *     1 + max level of its active upwind neighbours (longest path from a
 *     source; the count-based readiness of Listing 1: a vertex is ready when
 *     its count of unfinished upwind vertices reaches zero).
 *   - Order: cells of a direction sorted by (level, cell id).
 *   - Per-cell solve ("solve(vertices)", Listing 1; the discretisation is
 *     not given in the paper, so this is the step / upwind finite-volume
 *     scheme):  with mu_f a_f = (Omega . n_f) a_f taken outward from c,
 *        num = S_c V_c + sum_{f incoming} |mu_f| a_f psi_up(f)
 *        den = sigma_t,c V_c + sum_{f outgoing} mu_f a_f
 *        psi_c = num / den,
 *     faces summed in increasing face id; psi_up is the upwind cell's psi of
 *     this sweep, the lagged value for a lagged face, and the boundary inflow
 *     (0 for vacuum) on a boundary face.
 *   - Scalar flux phi_c = sum_m w_m psi_{c,m}, summed in direction order.
 *   - Source iteration (Alg. "Source iterative Sn solver"): phi^0 = 0;
 *     repeat { S = (c sigma_t phi + q) / (4 pi); sweep all directions;
 *     update lagged values; err = max_c |phi_new - phi| / max_c |phi_new| }
 *     until err < tol for every right-hand side.
 *   - Multigroup source iteration (the appendix's transport equation over
 *     energy groups g, same algorithm): every group's source from the
 *     previous iterate of all groups, S_g = (sum_h sigma_s[h][g] phi_h + q_g)
 *     / (4 pi), then one sweep per group with its own sigma_t and lagged
 *     values; err is the largest over the groups.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OD_OK 0
#define OD_NOT_CONVERGED 1
#define OD_BAD_INPUT -1
#define OD_NO_MEMORY -2

typedef struct {
    int64_t n_cells, n_faces, n_dirs, n_bfaces;
    /* copies of the inputs */
    int64_t *face_cells; /* [F][2] */
    double *normals;     /* [F][3] */
    double *areas;       /* [F] */
    double *volumes;     /* [N] */
    double *dirs;        /* [M][3] */
    /* cell -> faces (increasing face id) */
    int64_t *cf_ptr; /* [N+1] */
    int64_t *cf_face;
    int64_t *bface_index; /* [F]: boundary-face ordinal, -1 on interior faces */
    /* per direction results */
    int32_t *level;      /* [M][N] */
    int32_t *order;      /* [M][N] */
    int64_t *nlevels;    /* [M] */
    int32_t **level_ptr; /* [M] -> [nlevels+1] */
    int64_t *lag_ptr;    /* [M+1] offsets into lag_* */
    int64_t *lag_face, *lag_up, *lag_dn;
    int8_t *lag_flag;    /* [M][F]: 1 where the face is lagged for the direction */
} od_dag;

static double face_dot(const od_dag *g, int64_t f, int64_t m)
{
    const double *n = g->normals + 3 * f;
    const double *o = g->dirs + 3 * m;
    double a = n[0] * o[0];
    double b = n[1] * o[1];
    double c = n[2] * o[2];
    double s = a + b;
    return s + c;
}

void od_free(od_dag *g)
{
    if (!g) return;
    free(g->face_cells); free(g->normals); free(g->areas); free(g->volumes); free(g->dirs);
    free(g->cf_ptr); free(g->cf_face); free(g->bface_index);
    free(g->level); free(g->order); free(g->nlevels);
    if (g->level_ptr) {
        for (int64_t m = 0; m < g->n_dirs; ++m) free(g->level_ptr[m]);
        free(g->level_ptr);
    }
    free(g->lag_ptr); free(g->lag_face); free(g->lag_up); free(g->lag_dn); free(g->lag_flag);
    free(g);
}

/* Iterative Tarjan SCC over the cells with alive[c] != 0 and the active edges
 * up[f] -> dn[f].  Writes comp[c] (component id, -1 where not alive) and
 * returns the number of components. */
static int64_t tarjan(const od_dag *g, const int8_t *alive, const int64_t *up,
                      const int64_t *dn, int64_t *comp)
{
    int64_t N = g->n_cells;
    int64_t *idx = malloc(N * sizeof(int64_t));
    int64_t *low = malloc(N * sizeof(int64_t));
    int8_t *onst = calloc(N, 1);
    int64_t *stk = malloc(N * sizeof(int64_t));
    int64_t *cs_v = malloc(N * sizeof(int64_t));
    int64_t *cs_k = malloc(N * sizeof(int64_t));
    int64_t counter = 0, sp = 0, ncomp = 0;
    for (int64_t c = 0; c < N; ++c) { idx[c] = -1; comp[c] = -1; }
    for (int64_t root = 0; root < N; ++root) {
        if (!alive[root] || idx[root] >= 0) continue;
        int64_t csp = 0;
        idx[root] = low[root] = counter++;
        stk[sp++] = root; onst[root] = 1;
        cs_v[csp] = root; cs_k[csp] = g->cf_ptr[root]; ++csp;
        while (csp > 0) {
            int64_t v = cs_v[csp - 1];
            int64_t k = cs_k[csp - 1];
            if (k < g->cf_ptr[v + 1]) {
                cs_k[csp - 1] = k + 1;
                int64_t f = g->cf_face[k];
                if (up[f] != v) continue;
                int64_t w = dn[f];
                if (w < 0 || !alive[w]) continue;
                if (idx[w] < 0) {
                    idx[w] = low[w] = counter++;
                    stk[sp++] = w; onst[w] = 1;
                    cs_v[csp] = w; cs_k[csp] = g->cf_ptr[w]; ++csp;
                } else if (onst[w] && idx[w] < low[v]) {
                    low[v] = idx[w];
                }
            } else {
                --csp;
                if (low[v] == idx[v]) {
                    int64_t w;
                    do {
                        w = stk[--sp];
                        onst[w] = 0;
                        comp[w] = ncomp;
                    } while (w != v);
                    ++ncomp;
                }
                if (csp > 0) {
                    int64_t p = cs_v[csp - 1];
                    if (low[v] < low[p]) low[p] = low[v];
                }
            }
        }
    }
    free(idx); free(low); free(onst); free(stk); free(cs_v); free(cs_k);
    return ncomp;
}

/* Build the dependency graph of one direction: fills level/order for m and
 * returns the lagged faces (appended to *lag arrays). */
static int build_one(od_dag *g, int64_t m, int64_t **lf, int64_t *nl, int64_t *cap)
{
    int64_t N = g->n_cells, F = g->n_faces;
    int64_t *up = malloc(F * sizeof(int64_t));
    int64_t *dn = malloc(F * sizeof(int64_t));
    int64_t *indeg = malloc(N * sizeof(int64_t));
    int64_t *queue = malloc(N * sizeof(int64_t));
    int8_t *alive = malloc(N);
    int64_t *comp = malloc(N * sizeof(int64_t));
    int64_t *minface = malloc(N * sizeof(int64_t));
    int64_t *csize = malloc(N * sizeof(int64_t));
    int8_t *lagged = g->lag_flag + m * F;
    if (!up || !dn || !indeg || !queue || !alive || !comp || !minface || !csize) return OD_NO_MEMORY;

    /* edges from the FP64 sign of Omega . n_f */
    for (int64_t f = 0; f < F; ++f) {
        up[f] = dn[f] = -1;
        int64_t c0 = g->face_cells[2 * f], c1 = g->face_cells[2 * f + 1];
        if (c1 < 0) continue;
        double d = face_dot(g, f, m);
        if (d > 0.0) { up[f] = c0; dn[f] = c1; }
        else if (d < 0.0) { up[f] = c1; dn[f] = c0; }
    }
    for (;;) {
        /* Kahn peel over the active edges */
        for (int64_t c = 0; c < N; ++c) indeg[c] = 0;
        for (int64_t f = 0; f < F; ++f)
            if (up[f] >= 0) indeg[dn[f]]++;
        int64_t head = 0, tail = 0;
        for (int64_t c = 0; c < N; ++c) {
            alive[c] = 1;
            if (indeg[c] == 0) queue[tail++] = c;
        }
        while (head < tail) {
            int64_t u = queue[head++];
            alive[u] = 0;
            for (int64_t k = g->cf_ptr[u]; k < g->cf_ptr[u + 1]; ++k) {
                int64_t f = g->cf_face[k];
                if (up[f] != u) continue;
                if (--indeg[dn[f]] == 0) queue[tail++] = dn[f];
            }
        }
        if (tail == N) break;
        /* strongly connected components of what is left over */
        int64_t nc = tarjan(g, alive, up, dn, comp);
        for (int64_t s = 0; s < nc; ++s) { minface[s] = -1; csize[s] = 0; }
        for (int64_t c = 0; c < N; ++c)
            if (alive[c]) csize[comp[c]]++;
        for (int64_t f = 0; f < F; ++f) {
            if (up[f] < 0) continue;
            int64_t a = up[f], b = dn[f];
            if (!alive[a] || !alive[b] || comp[a] != comp[b]) continue;
            int64_t s = comp[a];
            if (csize[s] >= 2 && (minface[s] < 0 || f < minface[s])) minface[s] = f;
        }
        int64_t newly = 0;
        for (int64_t s = 0; s < nc; ++s) {
            if (csize[s] < 2) continue;
            int64_t f = minface[s];
            if (f < 0) continue; /* cannot happen: a component of >= 2 cells has an internal edge */
            if (*nl == *cap) {
                *cap = *cap ? 2 * *cap : 64;
                int64_t *t = realloc(*lf, 3 * *cap * sizeof(int64_t));
                if (!t) return OD_NO_MEMORY;
                *lf = t;
            }
            (*lf)[3 * *nl + 0] = f;
            (*lf)[3 * *nl + 1] = up[f];
            (*lf)[3 * *nl + 2] = dn[f];
            ++*nl;
            lagged[f] = 1;
            up[f] = dn[f] = -1;
            ++newly;
        }
        if (newly == 0) return OD_BAD_INPUT;
    }
    /* levels: longest path from a source, in Kahn order */
    int32_t *lev = g->level + m * N;
    for (int64_t c = 0; c < N; ++c) { indeg[c] = 0; lev[c] = 0; }
    for (int64_t f = 0; f < F; ++f)
        if (up[f] >= 0) indeg[dn[f]]++;
    int64_t head = 0, tail = 0;
    for (int64_t c = 0; c < N; ++c)
        if (indeg[c] == 0) queue[tail++] = c;
    while (head < tail) {
        int64_t u = queue[head++];
        for (int64_t k = g->cf_ptr[u]; k < g->cf_ptr[u + 1]; ++k) {
            int64_t f = g->cf_face[k];
            if (up[f] != u) continue;
            int64_t v = dn[f];
            if (lev[u] + 1 > lev[v]) lev[v] = lev[u] + 1;
            if (--indeg[v] == 0) queue[tail++] = v;
        }
    }
    /* order: stable counting sort of cell ids by level */
    int64_t L = 0;
    for (int64_t c = 0; c < N; ++c)
        if (lev[c] + 1 > L) L = lev[c] + 1;
    int32_t *ptr = calloc(L + 1, sizeof(int32_t));
    if (!ptr) return OD_NO_MEMORY;
    for (int64_t c = 0; c < N; ++c) ptr[lev[c] + 1]++;
    for (int64_t l = 0; l < L; ++l) ptr[l + 1] += ptr[l];
    int64_t *fill = malloc((L + 1) * sizeof(int64_t));
    for (int64_t l = 0; l <= L; ++l) fill[l] = ptr[l];
    int32_t *ord = g->order + m * N;
    for (int64_t c = 0; c < N; ++c) ord[fill[lev[c]]++] = (int32_t)c;
    free(fill);
    g->nlevels[m] = L;
    g->level_ptr[m] = ptr;
    free(up); free(dn); free(indeg); free(queue); free(alive); free(comp); free(minface); free(csize);
    return OD_OK;
}

static int cmp3(const void *a, const void *b)
{
    const int64_t *x = a, *y = b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

od_dag *od_build_dags(int64_t N, int64_t F, const int64_t *face_cells, const double *normals,
                      const double *areas, const double *volumes, int64_t M, const double *dirs,
                      int *status)
{
    *status = OD_BAD_INPUT;
    if (N <= 0 || F <= 0 || M <= 0 || N > INT32_MAX) return NULL;
    od_dag *g = calloc(1, sizeof(od_dag));
    if (!g) { *status = OD_NO_MEMORY; return NULL; }
    g->n_cells = N; g->n_faces = F; g->n_dirs = M;
    g->face_cells = malloc(2 * F * sizeof(int64_t));
    g->normals = malloc(3 * F * sizeof(double));
    g->areas = malloc(F * sizeof(double));
    g->volumes = malloc(N * sizeof(double));
    g->dirs = malloc(3 * M * sizeof(double));
    memcpy(g->face_cells, face_cells, 2 * F * sizeof(int64_t));
    memcpy(g->normals, normals, 3 * F * sizeof(double));
    memcpy(g->areas, areas, F * sizeof(double));
    memcpy(g->volumes, volumes, N * sizeof(double));
    memcpy(g->dirs, dirs, 3 * M * sizeof(double));
    for (int64_t f = 0; f < F; ++f) {
        int64_t c0 = face_cells[2 * f], c1 = face_cells[2 * f + 1];
        if (c0 < 0 || c0 >= N || c1 >= N || c1 == c0) { od_free(g); return NULL; }
    }
    /* cell -> face lists in increasing face id */
    g->cf_ptr = calloc(N + 1, sizeof(int64_t));
    for (int64_t f = 0; f < F; ++f) {
        g->cf_ptr[face_cells[2 * f] + 1]++;
        if (face_cells[2 * f + 1] >= 0) g->cf_ptr[face_cells[2 * f + 1] + 1]++;
    }
    for (int64_t c = 0; c < N; ++c) g->cf_ptr[c + 1] += g->cf_ptr[c];
    g->cf_face = malloc(g->cf_ptr[N] * sizeof(int64_t));
    int64_t *fill = malloc(N * sizeof(int64_t));
    for (int64_t c = 0; c < N; ++c) fill[c] = g->cf_ptr[c];
    g->bface_index = malloc(F * sizeof(int64_t));
    for (int64_t f = 0; f < F; ++f) {
        g->cf_face[fill[face_cells[2 * f]]++] = f;
        if (face_cells[2 * f + 1] >= 0) {
            g->cf_face[fill[face_cells[2 * f + 1]]++] = f;
            g->bface_index[f] = -1;
        } else {
            g->bface_index[f] = g->n_bfaces++;
        }
    }
    free(fill);

    g->level = malloc(M * N * sizeof(int32_t));
    g->order = malloc(M * N * sizeof(int32_t));
    g->nlevels = calloc(M, sizeof(int64_t));
    g->level_ptr = calloc(M, sizeof(int32_t *));
    g->lag_flag = calloc(M * F, 1);
    g->lag_ptr = calloc(M + 1, sizeof(int64_t));
    if (!g->level || !g->order || !g->lag_flag) { od_free(g); *status = OD_NO_MEMORY; return NULL; }
    int64_t **per_lf = calloc(M, sizeof(int64_t *));
    int64_t *per_n = calloc(M, sizeof(int64_t));
    int rc_all = OD_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t m = 0; m < M; ++m) {
        int64_t cap = 0;
        int rc = build_one(g, m, &per_lf[m], &per_n[m], &cap);
        if (rc != OD_OK) {
#pragma omp critical
            rc_all = rc;
        }
    }
    if (rc_all != OD_OK) {
        for (int64_t m = 0; m < M; ++m) free(per_lf[m]);
        free(per_lf); free(per_n); od_free(g); *status = rc_all; return NULL;
    }
    for (int64_t m = 0; m < M; ++m) g->lag_ptr[m + 1] = g->lag_ptr[m] + per_n[m];
    int64_t T = g->lag_ptr[M];
    g->lag_face = malloc((T + 1) * sizeof(int64_t));
    g->lag_up = malloc((T + 1) * sizeof(int64_t));
    g->lag_dn = malloc((T + 1) * sizeof(int64_t));
    for (int64_t m = 0; m < M; ++m) {
        if (per_n[m] > 0) qsort(per_lf[m], per_n[m], 3 * sizeof(int64_t), cmp3);
        for (int64_t j = 0; j < per_n[m]; ++j) {
            g->lag_face[g->lag_ptr[m] + j] = per_lf[m][3 * j];
            g->lag_up[g->lag_ptr[m] + j] = per_lf[m][3 * j + 1];
            g->lag_dn[g->lag_ptr[m] + j] = per_lf[m][3 * j + 2];
        }
        free(per_lf[m]);
    }
    free(per_lf); free(per_n);
    *status = OD_OK;
    return g;
}

int64_t od_n_bfaces(const od_dag *g) { return g->n_bfaces; }
int64_t od_nlevels(const od_dag *g, int64_t m) { return g->nlevels[m]; }
int64_t od_nlag_total(const od_dag *g) { return g->lag_ptr[g->n_dirs]; }
int64_t od_nlag(const od_dag *g, int64_t m) { return g->lag_ptr[m + 1] - g->lag_ptr[m]; }

void od_levels(const od_dag *g, int64_t m, int32_t *out)
{
    memcpy(out, g->level + m * g->n_cells, g->n_cells * sizeof(int32_t));
}

void od_order(const od_dag *g, int64_t m, int32_t *order, int32_t *level_ptr)
{
    memcpy(order, g->order + m * g->n_cells, g->n_cells * sizeof(int32_t));
    memcpy(level_ptr, g->level_ptr[m], (g->nlevels[m] + 1) * sizeof(int32_t));
}

/* lagged faces of direction m, sorted by face id: rows (face, upwind, downwind) */
void od_lagged(const od_dag *g, int64_t m, int64_t *out)
{
    for (int64_t j = g->lag_ptr[m]; j < g->lag_ptr[m + 1]; ++j) {
        int64_t i = j - g->lag_ptr[m];
        out[3 * i] = g->lag_face[j];
        out[3 * i + 1] = g->lag_up[j];
        out[3 * i + 2] = g->lag_dn[j];
    }
}

/* index of the lagged face f of direction m in the global lag list, or -1 */
static int64_t lag_slot(const od_dag *g, int64_t m, int64_t f)
{
    int64_t lo = g->lag_ptr[m], hi = g->lag_ptr[m + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (g->lag_face[mid] < f) lo = mid + 1; else hi = mid;
    }
    return (lo < g->lag_ptr[m + 1] && g->lag_face[lo] == f) ? lo : -1;
}

/* Sweep one direction for all right-hand sides.  psi_m: [R][N] output. */
static void sweep_dir(const od_dag *g, int64_t m, int64_t R, const double *sigma_t,
                      const double *src, const double *inflow, const double *psi_lag,
                      double *psi_m)
{
    int64_t N = g->n_cells, T = od_nlag_total(g);
    const int32_t *ord = g->order + m * N;
    const int8_t *lagged = g->lag_flag + m * g->n_faces;
    for (int64_t i = 0; i < N; ++i) {
        int64_t c = ord[i];
        double V = g->volumes[c];
        for (int64_t r = 0; r < R; ++r) {
            double num = src[r * N + c] * V;
            double den = sigma_t[c] * V;
            for (int64_t k = g->cf_ptr[c]; k < g->cf_ptr[c + 1]; ++k) {
                int64_t f = g->cf_face[k];
                int64_t c0 = g->face_cells[2 * f], c1 = g->face_cells[2 * f + 1];
                double mu = face_dot(g, f, m);
                if (c != c0) mu = -mu; /* outward from c */
                double coef = mu * g->areas[f];
                if (mu > 0.0) {
                    den += coef;
                } else if (mu < 0.0) {
                    double up;
                    if (c1 < 0) {
                        up = inflow ? inflow[r * g->n_bfaces + g->bface_index[f]] : 0.0;
                    } else if (lagged[f]) {
                        up = psi_lag[r * T + lag_slot(g, m, f)];
                    } else {
                        int64_t u = (c == c0) ? c1 : c0;
                        up = psi_m[r * N + u];
                    }
                    num += -coef * up;
                }
            }
            psi_m[r * N + c] = num / den;
        }
    }
}

/* One transport sweep of the directions dir_list[0..n_list) (all when
 * dir_list is NULL).  src: angular source [R][N] per steradian.  inflow:
 * [R][n_bfaces] isotropic boundary angular flux, NULL for vacuum.  psi_lag:
 * [R][n_lag_total], read as the lagged upwind values and overwritten with this
 * sweep's values.  phi: [R][N] = sum over the swept directions of w_m psi_m
 * (direction order).  psi: optional [R][n_list][N]. */
int od_sweep(const od_dag *g, int64_t R, const double *sigma_t, const double *src,
             const double *inflow, const double *weights, double *psi_lag, double *phi,
             double *psi, const int64_t *dir_list, int64_t n_list, int nthreads)
{
    int64_t N = g->n_cells, M = g->n_dirs, T = od_nlag_total(g);
    if (!dir_list) n_list = M;
    if (nthreads < 1) nthreads = 1;
    double *lag_new = T ? malloc(R * T * sizeof(double)) : NULL;
    if (T) memcpy(lag_new, psi_lag, R * T * sizeof(double));
    double *buf = malloc((size_t)nthreads * R * N * sizeof(double));
    if (!buf || (T && !lag_new)) { free(buf); free(lag_new); return OD_NO_MEMORY; }
    for (int64_t i = 0; i < R * N; ++i) phi[i] = 0.0;
    for (int64_t base = 0; base < n_list; base += nthreads) {
        int64_t cnt = n_list - base < nthreads ? n_list - base : nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t m = dir_list ? dir_list[base + t] : base + t;
            sweep_dir(g, m, R, sigma_t, src, inflow, psi_lag, buf + t * R * N);
        }
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t m = dir_list ? dir_list[base + t] : base + t;
            const double *pm = buf + t * R * N;
            for (int64_t r = 0; r < R; ++r)
                for (int64_t c = 0; c < N; ++c) phi[r * N + c] += weights[m] * pm[r * N + c];
            if (psi)
                for (int64_t r = 0; r < R; ++r)
                    memcpy(psi + ((size_t)r * n_list + base + t) * N, pm + r * N, N * sizeof(double));
            for (int64_t j = g->lag_ptr[m]; j < g->lag_ptr[m + 1]; ++j)
                for (int64_t r = 0; r < R; ++r)
                    lag_new[r * T + j] = pm[r * N + g->lag_up[j]];
        }
    }
    if (T) memcpy(psi_lag, lag_new, R * T * sizeof(double));
    free(lag_new); free(buf);
    return OD_OK;
}

/* Source iteration for R independent right-hand sides.  q: total isotropic
 * source [R][N]; c_ratio: scattering ratio per cell (sigma_s = c sigma_t).
 * Starts from phi = 0 and zero lagged values; stops when every right-hand
 * side's relative max-norm change is below tol, or after max_iters sweeps.
 * Returns OD_NOT_CONVERGED in the latter case (phi is still filled).
 * resid_hist (optional, [max_iters]) receives the max-over-rhs residual of
 * each iteration. */
int od_source_iterate(const od_dag *g, int64_t R, const double *sigma_t, const double *c_ratio,
                      const double *q, const double *inflow, const double *weights, double tol,
                      int64_t max_iters, double *phi, int64_t *iters_out, double *resid_out,
                      double *resid_hist, int nthreads)
{
    int64_t N = g->n_cells, T = od_nlag_total(g);
    const double four_pi = 4.0 * M_PI;
    double *src = malloc(R * N * sizeof(double));
    double *phi_new = malloc(R * N * sizeof(double));
    double *lag = calloc(R * T + 1, sizeof(double));
    if (!src || !phi_new || !lag) { free(src); free(phi_new); free(lag); return OD_NO_MEMORY; }
    for (int64_t i = 0; i < R * N; ++i) phi[i] = 0.0;
    int64_t it = 0;
    double resid = INFINITY;
    int status = OD_NOT_CONVERGED;
    while (it < max_iters) {
        for (int64_t r = 0; r < R; ++r)
            for (int64_t c = 0; c < N; ++c)
                src[r * N + c] = (c_ratio[c] * sigma_t[c] * phi[r * N + c] + q[r * N + c]) / four_pi;
        int rc = od_sweep(g, R, sigma_t, src, inflow, weights, lag, phi_new, NULL, NULL, 0, nthreads);
        if (rc != OD_OK) { status = rc; break; }
        ++it;
        resid = 0.0;
        for (int64_t r = 0; r < R; ++r) {
            double dmax = 0.0, pmax = 0.0;
            for (int64_t c = 0; c < N; ++c) {
                double d = fabs(phi_new[r * N + c] - phi[r * N + c]);
                double p = fabs(phi_new[r * N + c]);
                if (d > dmax) dmax = d;
                if (p > pmax) pmax = p;
            }
            double rr = (pmax > 0.0) ? dmax / pmax : (dmax > 0.0 ? INFINITY : 0.0);
            if (rr > resid) resid = rr;
        }
        memcpy(phi, phi_new, R * N * sizeof(double));
        if (resid_hist) resid_hist[it - 1] = resid;
        if (resid < tol) { status = OD_OK; break; }
    }
    *iters_out = it;
    *resid_out = resid;
    free(src); free(phi_new); free(lag);
    return status;
}

/* Multigroup source iteration (the appendix's transport equation with the
 * energy groups g and Alg. 1): each iteration first forms every group's
 * isotropic scattering source from the previous iterate of all groups,
 *   S_g = (sum_h sigma_s[h][g] phi_h + q_g) / (4 pi),   h in increasing order
 * (step 2.1; sigma_s[h][g][c] is the rate from group h into group g), then
 * sweeps each group with its own sigma_t[g] and its own lagged values
 * (step 2.2), then takes the largest relative max-norm change over the groups
 * (step 2.3).  All groups use the previous iterate (the paper computes every
 * I_mg of an iteration independently).  Arrays: sigma_t [G][N],
 * sigma_s [G][G][N], q [G][N], inflow [G][n_bfaces] or NULL, phi [G][N].
 * Starts from phi = 0 and zero lagged values. */
int od_source_iterate_mg(const od_dag *g, int64_t G, const double *sigma_t, const double *sigma_s,
                         const double *q, const double *inflow, const double *weights, double tol,
                         int64_t max_iters, double *phi, int64_t *iters_out, double *resid_out,
                         double *resid_hist, int nthreads)
{
    int64_t N = g->n_cells, T = od_nlag_total(g), Fb = g->n_bfaces;
    const double four_pi = 4.0 * M_PI;
    double *src = malloc(G * N * sizeof(double));
    double *phi_new = malloc(G * N * sizeof(double));
    double *lag = calloc(G * T + 1, sizeof(double));
    if (!src || !phi_new || !lag) { free(src); free(phi_new); free(lag); return OD_NO_MEMORY; }
    for (int64_t i = 0; i < G * N; ++i) phi[i] = 0.0;
    int64_t it = 0;
    double resid = INFINITY;
    int status = OD_NOT_CONVERGED;
    while (it < max_iters) {
        for (int64_t gg = 0; gg < G; ++gg)
            for (int64_t c = 0; c < N; ++c) {
                double s = 0.0;
                for (int64_t h = 0; h < G; ++h) s += sigma_s[(h * G + gg) * N + c] * phi[h * N + c];
                src[gg * N + c] = (s + q[gg * N + c]) / four_pi;
            }
        int rc = OD_OK;
        for (int64_t gg = 0; gg < G && rc == OD_OK; ++gg)
            rc = od_sweep(g, 1, sigma_t + gg * N, src + gg * N, inflow ? inflow + gg * Fb : NULL, weights,
                          lag + gg * T, phi_new + gg * N, NULL, NULL, 0, nthreads);
        if (rc != OD_OK) { status = rc; break; }
        ++it;
        resid = 0.0;
        for (int64_t gg = 0; gg < G; ++gg) {
            double dmax = 0.0, pmax = 0.0;
            for (int64_t c = 0; c < N; ++c) {
                double d = fabs(phi_new[gg * N + c] - phi[gg * N + c]);
                double p = fabs(phi_new[gg * N + c]);
                if (d > dmax) dmax = d;
                if (p > pmax) pmax = p;
            }
            double rr = (pmax > 0.0) ? dmax / pmax : (dmax > 0.0 ? INFINITY : 0.0);
            if (rr > resid) resid = rr;
        }
        memcpy(phi, phi_new, G * N * sizeof(double));
        if (resid_hist) resid_hist[it - 1] = resid;
        if (resid < tol) { status = OD_OK; break; }
    }
    *iters_out = it;
    *resid_out = resid;
    free(src); free(phi_new); free(lag);
    return status;
}

int od_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
