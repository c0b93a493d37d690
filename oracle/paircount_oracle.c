/*
 * Pair-counting oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU definition of exact pair counting, used to check the CUDA
 * path.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm may load it.  It shares no code with the CUDA library.
 *
 * Compiled with -O2 -ffp-contract=off (no FMA contraction, no fast-math), so
 * every floating-point expression below is evaluated in IEEE binary64 in the
 * order written.
 *
 * What it computes (paper: Sect. 2.5 for s, pi, sigma, mu and the two lines
 * of sight; Sect. 3.2 for monotone, continuous, zero-based bins compared on
 * squared values; Sect. 3.1 for auto counts visiting each unordered pair once
 * and for periodic wrapping):
 *
 *   periodic canonical form  x <- x - L floor(x/L); if x<0 x+=L; if x>=L x-=L
 *   separation               d = x_j - x_i per axis; periodic: if d > L/2
 *                            d -= L, else if d < -L/2 d += L
 *   s2                       (dx*dx + dy*dy) + dz*dz
 *   s bins                   bin k iff E_k <= s2 < E_{k+1},  E_k = e_k*e_k
 *   pi^2, LOS z              p2 = dz*dz
 *   pi^2, LOS midpoint       l = x_i + x_j, sl = (dx lx + dy ly) + dz lz,
 *                            ll = (lx lx + ly ly) + lz lz,
 *                            p2 = (sl*sl)/ll  (0 if ll == 0)
 *   mu bins (s, mu)          j = largest j < n_mu with p2 >= M_j * s2,
 *                            M_j = m_j*m_j  (m_0 = 0, m_n = 1, so mu = 1
 *                            lands in the last bin); s2 == 0 gives j = 0
 *   sigma^2 (sigma, pi)      q2 = s2 - p2, clamped at 0; sigma bins on q2,
 *                            pi bins on p2, both half-open on squared edges
 *   auto                     unordered pairs i < j, self-pairs excluded
 *   cross                    all (i in D1, j in D2)
 *   weights                  pair weight w_i * w_j, summed per bin with
 *                            Neumaier compensation
 *
 * Three drivers share that pair definition: a brute-force O(N1 N2) loop, a
 * cell list with cells no smaller than the largest separation of interest
 * (Sect. 2.1: three passes -- bounds, per-cell counts, grouping -- then visit
 * each cell and its neighbours), and a k-d tree with the dual-tree traversal
 * (Sect. 2.2, Alg. 1 and Sect. 3.1, Alg. 3).  Threads work on disjoint rows
 * or cells with private histograms that are summed at the end, so integer
 * counts do not depend on the thread count; the tree driver runs on one
 * thread.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { MODE_S = 0, MODE_SMU = 1, MODE_SIGPI = 2 };
enum { LOS_Z = 0, LOS_MID = 1 };

typedef struct {
    int periodic;
    double L[3], hL[3];
    int mode, los;
    int na, nb;          /* number of bins along each histogram axis */
    double *Ea;          /* squared s (or sigma) edges, na + 1 */
    double *Eb;          /* squared mu (or pi) edges, nb + 1 */
    int nbins;
} octx;

/* Index k in [0, n) with E[k] <= v < E[k+1], by bisection on the sorted
 * squared edges; the caller has checked E[0] <= v < E[n]. */
static int locate(double v, const double *E, int n)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (v >= E[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

/* Largest j < n with p2 >= M[j] * s2 (M[0] = 0, so j = 0 always qualifies). */
static int locate_mu(double p2, double s2, const double *M, int n)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        double t = M[mid] * s2;
        if (p2 >= t) lo = mid; else hi = mid;
    }
    return lo;
}

/* Histogram bin of the pair (a, b), or -1 when it falls outside every bin. */
static int pair_bin(const octx *c, const double *a, const double *b)
{
    double d0 = b[0] - a[0];
    double d1 = b[1] - a[1];
    double d2 = b[2] - a[2];
    if (c->periodic) {
        if (d0 > c->hL[0]) d0 -= c->L[0]; else if (d0 < -c->hL[0]) d0 += c->L[0];
        if (d1 > c->hL[1]) d1 -= c->L[1]; else if (d1 < -c->hL[1]) d1 += c->L[1];
        if (d2 > c->hL[2]) d2 -= c->L[2]; else if (d2 < -c->hL[2]) d2 += c->L[2];
    }
    double s2 = (d0 * d0 + d1 * d1) + d2 * d2;
    if (c->mode == MODE_S) {
        if (!(s2 >= c->Ea[0] && s2 < c->Ea[c->na])) return -1;
        return locate(s2, c->Ea, c->na);
    }
    double p2;
    if (c->los == LOS_Z) {
        p2 = d2 * d2;
    } else {
        double l0 = a[0] + b[0], l1 = a[1] + b[1], l2 = a[2] + b[2];
        double sl = (d0 * l0 + d1 * l1) + d2 * l2;
        double ll = (l0 * l0 + l1 * l1) + l2 * l2;
        p2 = (ll > 0.0) ? (sl * sl) / ll : 0.0;
    }
    if (c->mode == MODE_SMU) {
        if (!(s2 >= c->Ea[0] && s2 < c->Ea[c->na])) return -1;
        int k = locate(s2, c->Ea, c->na);
        int j = (s2 > 0.0) ? locate_mu(p2, s2, c->Eb, c->nb) : 0;
        return k * c->nb + j;
    }
    double q2 = s2 - p2;
    if (q2 < 0.0) q2 = 0.0;
    if (!(q2 >= c->Ea[0] && q2 < c->Ea[c->na])) return -1;
    if (!(p2 >= c->Eb[0] && p2 < c->Eb[c->nb])) return -1;
    return locate(q2, c->Ea, c->na) * c->nb + locate(p2, c->Eb, c->nb);
}

static double canon(double x, double L)
{
    double y = x - L * floor(x / L);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    return y;
}

static void neumaier_add(double *sum, double *comp, double v)
{
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
    else *comp += (v - t) + *sum;
    *sum = t;
}

/* ------------------------------------------------------------------------ */

typedef struct {
    const octx *c;
    const double *x1, *w1, *x2, *w2;
    int64_t n1, n2;
    int is_auto;
    /* grid driver */
    int use_grid;
    int ng[3];
    const int64_t *start1, *start2;   /* cell starts, ncell + 1 */
    const int64_t *ord1, *ord2;       /* point indices grouped by cell */
    const double *xs1, *xs2;          /* coordinates in cell order (Sect. 2.1: the grid
                                         stores each cell's points contiguously) */
    const double *ws1, *ws2;          /* weights in cell order (or NULL) */
    int64_t ncell;
    int tid, nthreads;
    int64_t *cnt;                     /* private histogram */
    double *wsum, *wcomp;             /* private Neumaier sums (or NULL) */
} job;

static inline void add_pair(job *jb, int64_t i, int64_t j)
{
    const double *a = jb->x1 + 3 * i;
    const double *b = jb->x2 + 3 * j;
    int bin = pair_bin(jb->c, a, b);
    if (bin < 0) return;
    jb->cnt[bin] += 1;
    if (jb->wsum) neumaier_add(&jb->wsum[bin], &jb->wcomp[bin], jb->w1[i] * jb->w2[j]);
}

/* Pair (p, q) of the cell-ordered copies: the same values as add_pair on
 * the original indices ord1[p], ord2[q]. */
static inline void add_pair_sorted(job *jb, int64_t p, int64_t q)
{
    const double *a = jb->xs1 + 3 * p;
    const double *b = jb->xs2 + 3 * q;
    int bin = pair_bin(jb->c, a, b);
    if (bin < 0) return;
    jb->cnt[bin] += 1;
    if (jb->wsum) neumaier_add(&jb->wsum[bin], &jb->wcomp[bin], jb->ws1[p] * jb->ws2[q]);
}

static void *brute_worker(void *arg)
{
    job *jb = (job *)arg;
    /* rows are dealt out in chunks of up to 64, fewer when the rows are few,
     * so that every thread gets an equal share */
    int64_t CH = jb->n1 / ((int64_t)jb->nthreads * 16);
    if (CH > 64) CH = 64;
    if (CH < 1) CH = 1;
    for (int64_t c0 = (int64_t)jb->tid * CH; c0 < jb->n1; c0 += (int64_t)jb->nthreads * CH) {
        int64_t c1 = c0 + CH < jb->n1 ? c0 + CH : jb->n1;
        for (int64_t i = c0; i < c1; i++) {
            int64_t j0 = jb->is_auto ? i + 1 : 0;
            for (int64_t j = j0; j < jb->n2; j++) add_pair(jb, i, j);
        }
    }
    return NULL;
}

/* Work item k = (cell, run of up to GRID_CHUNK of its points) goes to
 * thread k % nthreads, so the split is fixed by the input alone. */
#define GRID_CHUNK 256

static void *grid_worker(void *arg)
{
    job *jb = (job *)arg;
    const int *ng = jb->ng;
    int64_t item = 0;
    for (int64_t a = 0; a < jb->ncell; a++) {
        int64_t a0 = jb->start1[a], a1 = jb->start1[a + 1];
        if (a0 == a1) continue;
        int ax = (int)(a % ng[0]);
        int ay = (int)((a / ng[0]) % ng[1]);
        int az = (int)(a / ((int64_t)ng[0] * ng[1]));
        for (int64_t p0 = a0; p0 < a1; p0 += GRID_CHUNK, item++) {
            if (item % jb->nthreads != jb->tid) continue;
            int64_t p1 = p0 + GRID_CHUNK < a1 ? p0 + GRID_CHUNK : a1;
            for (int oz = -1; oz <= 1; oz++)
            for (int oy = -1; oy <= 1; oy++)
            for (int ox = -1; ox <= 1; ox++) {
                int bx = ax + ox, by = ay + oy, bz = az + oz;
                if (jb->c->periodic) {
                    bx = (bx + ng[0]) % ng[0];
                    by = (by + ng[1]) % ng[1];
                    bz = (bz + ng[2]) % ng[2];
                } else if (bx < 0 || by < 0 || bz < 0 || bx >= ng[0] || by >= ng[1] || bz >= ng[2]) {
                    continue;
                }
                int64_t b = ((int64_t)bz * ng[1] + by) * ng[0] + bx;
                if (jb->is_auto && b < a) continue;
                int64_t b0 = jb->start2[b], b1 = jb->start2[b + 1];
                for (int64_t p = p0; p < p1; p++) {
                    int64_t q0 = (jb->is_auto && b == a) ? p + 1 : b0;
                    for (int64_t q = q0; q < b1; q++) add_pair_sorted(jb, p, q);
                }
            }
        }
    }
    return NULL;
}

/* Group point indices by cell (counting sort). */
static void bucket(const double *x, int64_t n, const double *lo, const double *w,
                   const int *ng, int64_t ncell, int64_t *start, int64_t *ord)
{
    int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    memset(start, 0, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t i = 0; i < n; i++) {
        int64_t id[3];
        for (int a = 0; a < 3; a++) {
            double f = floor((x[3 * i + a] - lo[a]) / w[a]);
            int64_t k;
            if (!(f >= 0.0)) k = 0;
            else if (f >= (double)(ng[a] - 1)) k = ng[a] - 1;
            else k = (int64_t)f;
            id[a] = k;
        }
        cid[i] = (id[2] * ng[1] + id[1]) * ng[0] + id[0];
        start[cid[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; c++) start[c + 1] += start[c];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    memcpy(cur, start, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t i = 0; i < n; i++) ord[cur[cid[i]]++] = i;
    free(cur);
    free(cid);
}

/* Rows of x (each `width` doubles) in the order ord: the cell-sorted copy. */
static double *gather_rows(const double *x, const int64_t *ord, int64_t n, int width)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)(width * (n > 0 ? n : 1)));
    for (int64_t p = 0; p < n; p++)
        for (int a = 0; a < width; a++) y[width * p + a] = x[width * ord[p] + a];
    return y;
}

static int check_edges(const double *e, int n, int zero_one)
{
    if (n < 1 || !e) return 0;
    for (int k = 0; k <= n; k++)
        if (!(e[k] >= 0.0) || !isfinite(e[k])) return 0;
    for (int k = 0; k < n; k++)
        if (!(e[k + 1] > e[k])) return 0;
    if (zero_one && !(e[0] == 0.0 && e[n] == 1.0)) return 0;
    return 1;
}

/*
 * Count pairs.  x2 == NULL means an auto count of x1.  Weights are optional
 * (w1/w2 NULL): when given, wcounts receives the weighted sums.  counts always
 * receives the plain pair counts.  Returns 0, or -1 on invalid arguments.
 */
int oracle_count(const double *x1, const double *w1, int64_t n1,
                 const double *x2, const double *w2, int64_t n2,
                 int periodic, const double *L,
                 int mode, int los,
                 int na, const double *ea, int nb, const double *eb,
                 int use_grid, int nthreads,
                 int64_t *counts, double *wcounts)
{
    if (mode < 0 || mode > 2 || los < 0 || los > 1) return -1;
    if (!check_edges(ea, na, 0)) return -1;
    if (mode != MODE_S && !check_edges(eb, nb, mode == MODE_SMU)) return -1;
    if (periodic && los == LOS_MID && mode != MODE_S) return -1;
    if (n1 < 0 || n2 < 0) return -1;
    int is_auto = (x2 == NULL);
    if (is_auto) { x2 = x1; w2 = w1; n2 = n1; }
    int weighted = (wcounts != NULL) && w1 && w2;
    if (nthreads < 1) nthreads = 1;

    octx c;
    memset(&c, 0, sizeof(c));
    c.periodic = periodic;
    c.mode = mode;
    c.los = los;
    c.na = na;
    c.nb = (mode == MODE_S) ? 1 : nb;
    c.nbins = na * c.nb;
    for (int a = 0; a < 3; a++) {
        c.L[a] = periodic ? L[a] : 0.0;
        c.hL[a] = 0.5 * c.L[a];
        if (periodic && !(L[a] > 0.0)) return -1;
    }
    c.Ea = (double *)malloc(sizeof(double) * (size_t)(na + 1));
    c.Eb = (double *)malloc(sizeof(double) * (size_t)(c.nb + 1));
    for (int k = 0; k <= na; k++) c.Ea[k] = ea[k] * ea[k];
    if (mode == MODE_S) { c.Eb[0] = 0.0; c.Eb[1] = 1.0; }
    else for (int k = 0; k <= nb; k++) c.Eb[k] = eb[k] * eb[k];

    /* periodic canonical form on private copies */
    double *c1 = NULL, *c2 = NULL;
    if (periodic) {
        c1 = (double *)malloc(sizeof(double) * (size_t)(3 * (n1 > 0 ? n1 : 1)));
        for (int64_t i = 0; i < n1; i++)
            for (int a = 0; a < 3; a++) c1[3 * i + a] = canon(x1[3 * i + a], c.L[a]);
        if (is_auto) c2 = c1;
        else {
            c2 = (double *)malloc(sizeof(double) * (size_t)(3 * (n2 > 0 ? n2 : 1)));
            for (int64_t i = 0; i < n2; i++)
                for (int a = 0; a < 3; a++) c2[3 * i + a] = canon(x2[3 * i + a], c.L[a]);
        }
        x1 = c1;
        x2 = c2;
    }

    /* cell geometry for the grid driver */
    int ng[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, wcell[3] = {1, 1, 1};
    int64_t ncell = 1;
    int64_t *st1 = NULL, *st2 = NULL, *or1 = NULL, *or2 = NULL;
    double *xs1 = NULL, *xs2 = NULL, *ws1 = NULL, *ws2 = NULL;
    if (use_grid && n1 > 0 && n2 > 0) {
        double reff = (mode == MODE_SIGPI) ? sqrt(c.Ea[na] + c.Eb[c.nb]) : ea[na];
        double hi[3];
        for (int a = 0; a < 3; a++) {
            if (periodic) { lo[a] = 0.0; hi[a] = c.L[a]; }
            else {
                lo[a] = INFINITY; hi[a] = -INFINITY;
                for (int64_t i = 0; i < n1; i++) {
                    if (x1[3 * i + a] < lo[a]) lo[a] = x1[3 * i + a];
                    if (x1[3 * i + a] > hi[a]) hi[a] = x1[3 * i + a];
                }
                for (int64_t i = 0; i < n2; i++) {
                    if (x2[3 * i + a] < lo[a]) lo[a] = x2[3 * i + a];
                    if (x2[3 * i + a] > hi[a]) hi[a] = x2[3 * i + a];
                }
            }
            double ext = hi[a] - lo[a];
            double cw = reff * (1.0 + 1e-6) + 1e-9 * fabs(ext) + 1e-300;
            double nf = floor(ext / cw);
            if (nf > 512.0) nf = 512.0;
            ng[a] = nf >= 1.0 ? (int)nf : 1;
            if (periodic && ng[a] < 3) { use_grid = 0; break; }
            wcell[a] = ng[a] > 1 ? ext / ng[a] : (ext > 0 ? ext * 2.0 : 1.0);
        }
        if (use_grid) {
            ncell = (int64_t)ng[0] * ng[1] * ng[2];
            st1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
            or1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)n1);
            bucket(x1, n1, lo, wcell, ng, ncell, st1, or1);
            if (is_auto) { st2 = st1; or2 = or1; }
            else {
                st2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
                or2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)n2);
                bucket(x2, n2, lo, wcell, ng, ncell, st2, or2);
            }
            xs1 = gather_rows(x1, or1, n1, 3);
            ws1 = weighted ? gather_rows(w1, or1, n1, 1) : NULL;
            if (is_auto) { xs2 = xs1; ws2 = ws1; }
            else {
                xs2 = gather_rows(x2, or2, n2, 3);
                ws2 = weighted ? gather_rows(w2, or2, n2, 1) : NULL;
            }
        }
    } else {
        use_grid = 0;
    }

    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; t++) {
        job *jb = &jobs[t];
        jb->c = &c;
        jb->x1 = x1; jb->w1 = w1; jb->x2 = x2; jb->w2 = w2;
        jb->n1 = n1; jb->n2 = n2;
        jb->is_auto = is_auto;
        jb->use_grid = use_grid;
        for (int a = 0; a < 3; a++) jb->ng[a] = ng[a];
        jb->start1 = st1; jb->start2 = st2; jb->ord1 = or1; jb->ord2 = or2;
        jb->xs1 = xs1; jb->xs2 = xs2; jb->ws1 = ws1; jb->ws2 = ws2;
        jb->ncell = ncell;
        jb->tid = t; jb->nthreads = nthreads;
        jb->cnt = (int64_t *)calloc((size_t)c.nbins, sizeof(int64_t));
        if (weighted) {
            jb->wsum = (double *)calloc((size_t)c.nbins, sizeof(double));
            jb->wcomp = (double *)calloc((size_t)c.nbins, sizeof(double));
        }
        pthread_create(&th[t], NULL, use_grid ? grid_worker : brute_worker, jb);
    }
    for (int b = 0; b < c.nbins; b++) counts[b] = 0;
    double *fs = NULL, *fc = NULL;
    if (weighted) {
        fs = (double *)calloc((size_t)c.nbins, sizeof(double));
        fc = (double *)calloc((size_t)c.nbins, sizeof(double));
    }
    for (int t = 0; t < nthreads; t++) {
        pthread_join(th[t], NULL);
        for (int b = 0; b < c.nbins; b++) counts[b] += jobs[t].cnt[b];
        if (weighted)
            for (int b = 0; b < c.nbins; b++) {
                neumaier_add(&fs[b], &fc[b], jobs[t].wsum[b]);
                neumaier_add(&fs[b], &fc[b], jobs[t].wcomp[b]);
            }
        free(jobs[t].cnt);
        free(jobs[t].wsum);
        free(jobs[t].wcomp);
    }
    if (weighted)
        for (int b = 0; b < c.nbins; b++) wcounts[b] = fs[b] + fc[b];
    else if (wcounts)
        for (int b = 0; b < c.nbins; b++) wcounts[b] = (double)counts[b];

    free(fs); free(fc);
    free(jobs); free(th);
    if (st2 != st1) { free(st2); free(or2); }
    free(st1); free(or1);
    if (xs2 != xs1) free(xs2);
    if (ws2 != ws1) free(ws2);
    free(xs1); free(ws1);
    if (c2 != c1) free(c2);
    free(c1);
    free(c.Ea); free(c.Eb);
    return 0;
}

/* Bin of one pair (a, b) under the same definition; -1 outside all bins,
 * -2 on invalid arguments.  Coordinates are canonicalised first when periodic. */
int oracle_pair_bin(const double *a, const double *b, int periodic, const double *L,
                    int mode, int los, int na, const double *ea, int nb, const double *eb)
{
    if (!check_edges(ea, na, 0)) return -2;
    if (mode != MODE_S && !check_edges(eb, nb, mode == MODE_SMU)) return -2;
    octx c;
    memset(&c, 0, sizeof(c));
    c.periodic = periodic; c.mode = mode; c.los = los; c.na = na;
    c.nb = (mode == MODE_S) ? 1 : nb;
    double Ea[4096], Eb[4096];
    if (na + 1 > 4096 || c.nb + 1 > 4096) return -2;
    for (int k = 0; k <= na; k++) Ea[k] = ea[k] * ea[k];
    if (mode == MODE_S) { Eb[0] = 0.0; Eb[1] = 1.0; }
    else for (int k = 0; k <= nb; k++) Eb[k] = eb[k] * eb[k];
    c.Ea = Ea; c.Eb = Eb;
    double pa[3], pb[3];
    for (int q = 0; q < 3; q++) {
        c.L[q] = periodic ? L[q] : 0.0;
        c.hL[q] = 0.5 * c.L[q];
        pa[q] = periodic ? canon(a[q], c.L[q]) : a[q];
        pb[q] = periodic ? canon(b[q], c.L[q]) : b[q];
    }
    return pair_bin(&c, pa, pb);
}

/* ------------------------------------------------------------------------ */
/* k-d tree (Sect. 2.2, Alg. 1) and dual-tree traversal (Sect. 3.1, Alg. 3)  */
/* ------------------------------------------------------------------------ */

/* Nodes are kept in heap order: the root is slot 0 and the children of slot
 * h are 2h + 1 (left) and 2h + 2 (right).  Every split gives the left child
 * floor(n / 2) points, so all nodes of one level hold n_d or n_d + 1 points
 * and the tree is balanced. */
typedef struct {
    int depth;            /* deepest level holding a node */
    int64_t nslots;       /* 2^(depth + 1) - 1 */
    int64_t *start;       /* first position of the node in ord */
    int64_t *count;       /* points of the node; -1 in an empty slot */
    int *axis;            /* split axis, -1 for a leaf or an empty slot */
    double *box;          /* lo[3], hi[3] of the node's points (minimum AABB) */
    int64_t *ord;         /* tree order: position -> point index */
} otree;

typedef struct {
    double v;
    int64_t i;
} keyed;

static int keyed_cmp(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->v < b->v) return -1;
    if (a->v > b->v) return 1;
    return (a->i > b->i) - (a->i < b->i);
}

/* Levels below the root until every node holds at most n_leaf points: the
 * largest node of a level holds ceil(n / 2^d) points. */
static int kd_depth(int64_t n, int n_leaf)
{
    int d = 0;
    int64_t m = n;
    while (m > n_leaf) {
        m = (m + 1) / 2;
        d++;
    }
    return d;
}

static void kd_node(otree *t, const double *x, int64_t h, int64_t start, int64_t count,
                    int n_leaf, keyed *tmp)
{
    t->start[h] = start;
    t->count[h] = count;
    double *bx = t->box + 6 * h;
    for (int a = 0; a < 3; a++) {
        bx[a] = INFINITY;
        bx[3 + a] = -INFINITY;
    }
    for (int64_t p = start; p < start + count; p++)
        for (int a = 0; a < 3; a++) {
            double v = x[3 * t->ord[p] + a];
            if (v < bx[a]) bx[a] = v;
            if (v > bx[3 + a]) bx[3 + a] = v;
        }
    if (count <= n_leaf) {
        t->axis[h] = -1;
        return;
    }
    /* axis of the largest coordinate variance (two passes: mean, then the
     * mean squared deviation); the first such axis on a tie */
    int best = 0;
    double bestvar = -1.0;
    for (int a = 0; a < 3; a++) {
        double m = 0.0;
        for (int64_t p = start; p < start + count; p++) m += x[3 * t->ord[p] + a];
        m /= (double)count;
        double v = 0.0;
        for (int64_t p = start; p < start + count; p++) {
            double d = x[3 * t->ord[p] + a] - m;
            v += d * d;
        }
        v /= (double)count;
        if (v > bestvar) {
            bestvar = v;
            best = a;
        }
    }
    t->axis[h] = best;
    /* median split: the floor(n / 2) points with the smallest coordinate
     * along that axis go left (point index breaks ties) */
    for (int64_t k = 0; k < count; k++) {
        tmp[k].v = x[3 * t->ord[start + k] + best];
        tmp[k].i = t->ord[start + k];
    }
    qsort(tmp, (size_t)count, sizeof(keyed), keyed_cmp);
    for (int64_t k = 0; k < count; k++) t->ord[start + k] = tmp[k].i;
    int64_t nl = count / 2;
    kd_node(t, x, 2 * h + 1, start, nl, n_leaf, tmp);
    kd_node(t, x, 2 * h + 2, start + nl, count - nl, n_leaf, tmp);
}

static int kd_build(otree *t, const double *x, int64_t n, int n_leaf)
{
    memset(t, 0, sizeof(*t));
    if (n < 1 || n_leaf < 1) return -1;
    t->depth = kd_depth(n, n_leaf);
    if (t->depth > 30) return -1;
    t->nslots = ((int64_t)2 << t->depth) - 1;
    t->start = (int64_t *)malloc(sizeof(int64_t) * (size_t)t->nslots);
    t->count = (int64_t *)malloc(sizeof(int64_t) * (size_t)t->nslots);
    t->axis = (int *)malloc(sizeof(int) * (size_t)t->nslots);
    t->box = (double *)malloc(sizeof(double) * 6 * (size_t)t->nslots);
    t->ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    keyed *tmp = (keyed *)malloc(sizeof(keyed) * (size_t)n);
    for (int64_t h = 0; h < t->nslots; h++) {
        t->start[h] = 0;
        t->count[h] = -1;
        t->axis[h] = -1;
    }
    for (int64_t i = 0; i < n; i++) t->ord[i] = i;
    kd_node(t, x, 0, 0, n, n_leaf, tmp);
    free(tmp);
    return 0;
}

static void kd_free(otree *t)
{
    free(t->start);
    free(t->count);
    free(t->axis);
    free(t->box);
    free(t->ord);
}

/* Bounds of the squared separations of the pairs of two nodes, from their
 * boxes: per axis the gap between the intervals and the largest distance
 * between their ends.  Periodic axes take the smallest gap over the images
 * b - L, b, b + L, and the largest distance is at most L / 2 after the wrap. */
static void kd_dist_range(const octx *c, const double *A, const double *B, double *dmin2,
                          double *dmax2)
{
    double lo2 = 0.0, hi2 = 0.0;
    for (int a = 0; a < 3; a++) {
        double gap = INFINITY, far;
        int ns = c->periodic ? 3 : 1;
        for (int k = 0; k < ns; k++) {
            double sh = (k == 0) ? 0.0 : (k == 1 ? c->L[a] : -c->L[a]);
            double g = B[a] + sh - A[3 + a];
            double g2 = A[a] - (B[3 + a] + sh);
            if (g2 > g) g = g2;
            if (g < 0.0) g = 0.0;
            if (g < gap) gap = g;
        }
        far = B[3 + a] - A[a];
        if (A[3 + a] - B[a] > far) far = A[3 + a] - B[a];
        if (c->periodic && far > c->hL[a]) far = c->hL[a];
        lo2 += gap * gap;
        hi2 += far * far;
    }
    *dmin2 = lo2;
    *dmax2 = hi2;
}

typedef struct {
    int64_t a, b;
} npair;

/* Dual-tree count (Alg. 3) with an explicit stack of node pairs.  A pair
 * whose separation range misses the range of interest is dropped; one that
 * lies inside it, or a pair of leaves, has all its point pairs evaluated;
 * otherwise the non-leaf nodes are split.  For an auto count only one of
 * {a, b} and {b, a} is visited: a node paired with itself is split into
 * (left, left), (left, right) and (right, right). */
static void kd_dual(job *jb, const otree *t1, const otree *t2, double s2lo, double s2hi)
{
    const octx *c = jb->c;
    int64_t cap = 1024, top = 0;
    npair *st = (npair *)malloc(sizeof(npair) * (size_t)cap);
    st[top++] = (npair){0, 0};
    while (top > 0) {
        npair q = st[--top];
        const double *A = t1->box + 6 * q.a, *B = t2->box + 6 * q.b;
        double dmin2, dmax2;
        kd_dist_range(c, A, B, &dmin2, &dmax2);
        /* bounds carry rounding: prune and accept with a relative margin */
        if (dmin2 > s2hi * (1.0 + 1e-9) || dmax2 < s2lo * (1.0 - 1e-9)) continue;
        int self = jb->is_auto && q.a == q.b;
        int leaf1 = t1->axis[q.a] < 0, leaf2 = t2->axis[q.b] < 0;
        int inside = dmin2 >= s2lo * (1.0 + 1e-9) && dmax2 < s2hi * (1.0 - 1e-9);
        if (inside || (leaf1 && leaf2)) {
            int64_t a0 = t1->start[q.a], a1 = a0 + t1->count[q.a];
            int64_t b0 = t2->start[q.b], b1 = b0 + t2->count[q.b];
            for (int64_t p = a0; p < a1; p++)
                for (int64_t r = self ? p + 1 : b0; r < b1; r++)
                    add_pair(jb, t1->ord[p], t2->ord[r]);
            continue;
        }
        if (top + 4 > cap) {
            cap *= 2;
            st = (npair *)realloc(st, sizeof(npair) * (size_t)cap);
        }
        if (self) {
            st[top++] = (npair){2 * q.a + 2, 2 * q.a + 2};
            st[top++] = (npair){2 * q.a + 1, 2 * q.a + 2};
            st[top++] = (npair){2 * q.a + 1, 2 * q.a + 1};
        } else if (!leaf1 && !leaf2) {
            st[top++] = (npair){2 * q.a + 2, 2 * q.b + 2};
            st[top++] = (npair){2 * q.a + 2, 2 * q.b + 1};
            st[top++] = (npair){2 * q.a + 1, 2 * q.b + 2};
            st[top++] = (npair){2 * q.a + 1, 2 * q.b + 1};
        } else if (leaf1) {
            st[top++] = (npair){q.a, 2 * q.b + 2};
            st[top++] = (npair){q.a, 2 * q.b + 1};
        } else {
            st[top++] = (npair){2 * q.a + 2, q.b};
            st[top++] = (npair){2 * q.a + 1, q.b};
        }
    }
    free(st);
}

/* Range of squared separations that can fall in a bin: [E_0, E_n) on s for
 * s and (s, mu) bins; below sigma_max^2 + pi_max^2 for (sigma, pi) bins. */
static void kd_s2_range(const octx *c, double *lo, double *hi)
{
    if (c->mode == MODE_SIGPI) {
        *lo = 0.0;
        *hi = c->Ea[c->na] + c->Eb[c->nb];
    } else {
        *lo = c->Ea[0];
        *hi = c->Ea[c->na];
    }
}

/*
 * Pair counts through the k-d tree and the dual-tree traversal; the same
 * arguments and results as oracle_count (one thread).  Returns 0, or -1 on
 * invalid arguments.
 */
int oracle_count_kdtree(const double *x1, const double *w1, int64_t n1,
                        const double *x2, const double *w2, int64_t n2,
                        int periodic, const double *L, int mode, int los,
                        int na, const double *ea, int nb, const double *eb,
                        int n_leaf, int64_t *counts, double *wcounts)
{
    if (mode < 0 || mode > 2 || los < 0 || los > 1 || n_leaf < 1) return -1;
    if (!check_edges(ea, na, 0)) return -1;
    if (mode != MODE_S && !check_edges(eb, nb, mode == MODE_SMU)) return -1;
    if (periodic && los == LOS_MID && mode != MODE_S) return -1;
    if (n1 < 0 || n2 < 0) return -1;
    int is_auto = (x2 == NULL);
    if (is_auto) { x2 = x1; w2 = w1; n2 = n1; }
    int weighted = (wcounts != NULL) && w1 && w2;

    octx c;
    memset(&c, 0, sizeof(c));
    c.periodic = periodic;
    c.mode = mode;
    c.los = los;
    c.na = na;
    c.nb = (mode == MODE_S) ? 1 : nb;
    c.nbins = na * c.nb;
    for (int a = 0; a < 3; a++) {
        c.L[a] = periodic ? L[a] : 0.0;
        c.hL[a] = 0.5 * c.L[a];
        if (periodic && !(L[a] > 0.0)) return -1;
    }
    c.Ea = (double *)malloc(sizeof(double) * (size_t)(na + 1));
    c.Eb = (double *)malloc(sizeof(double) * (size_t)(c.nb + 1));
    for (int k = 0; k <= na; k++) c.Ea[k] = ea[k] * ea[k];
    if (mode == MODE_S) { c.Eb[0] = 0.0; c.Eb[1] = 1.0; }
    else for (int k = 0; k <= nb; k++) c.Eb[k] = eb[k] * eb[k];

    double *c1 = NULL, *c2 = NULL;
    if (periodic) {
        c1 = (double *)malloc(sizeof(double) * (size_t)(3 * (n1 > 0 ? n1 : 1)));
        for (int64_t i = 0; i < n1; i++)
            for (int a = 0; a < 3; a++) c1[3 * i + a] = canon(x1[3 * i + a], c.L[a]);
        if (is_auto) c2 = c1;
        else {
            c2 = (double *)malloc(sizeof(double) * (size_t)(3 * (n2 > 0 ? n2 : 1)));
            for (int64_t i = 0; i < n2; i++)
                for (int a = 0; a < 3; a++) c2[3 * i + a] = canon(x2[3 * i + a], c.L[a]);
        }
        x1 = c1;
        x2 = c2;
    }

    for (int b = 0; b < c.nbins; b++) counts[b] = 0;
    job jb;
    memset(&jb, 0, sizeof(jb));
    jb.c = &c;
    jb.x1 = x1; jb.w1 = w1; jb.x2 = x2; jb.w2 = w2;
    jb.n1 = n1; jb.n2 = n2;
    jb.is_auto = is_auto;
    jb.cnt = counts;
    double *fc = NULL;
    if (weighted) {
        for (int b = 0; b < c.nbins; b++) wcounts[b] = 0.0;
        fc = (double *)calloc((size_t)(na > 0 ? c.nbins : 1), sizeof(double));
        jb.wsum = wcounts;
        jb.wcomp = fc;
    }
    if (n1 > 0 && n2 > 0) {
        otree t1, t2;
        kd_build(&t1, x1, n1, n_leaf);
        if (is_auto) t2 = t1;
        else kd_build(&t2, x2, n2, n_leaf);
        double s2lo, s2hi;
        kd_s2_range(&c, &s2lo, &s2hi);
        kd_dual(&jb, &t1, &t2, s2lo, s2hi);
        kd_free(&t1);
        if (!is_auto) kd_free(&t2);
    }
    if (weighted)
        for (int b = 0; b < c.nbins; b++) wcounts[b] += fc[b];
    else if (wcounts)
        for (int b = 0; b < c.nbins; b++) wcounts[b] = (double)counts[b];
    free(fc);
    if (c2 != c1) free(c2);
    free(c1);
    free(c.Ea); free(c.Eb);
    return 0;
}

/*
 * The k-d tree of Alg. 1 over n points (canonicalised first when periodic),
 * in heap order.  Returns the depth (deepest level), or -1 on invalid
 * arguments or when the tree has more than max_slots slots.  With nslots =
 * 2^(depth + 1) - 1 <= max_slots the arrays receive: start[h], count[h]
 * (-1: empty slot), axis[h] (-1: leaf or empty), box[6 h .. 6 h + 5] (lo,
 * hi), and ord[n] (tree position -> point index).
 */
int oracle_kdtree(const double *x, int64_t n, int periodic, const double *L, int n_leaf,
                  int64_t max_slots, int64_t *start, int64_t *count, int *axis, double *box,
                  int64_t *ord)
{
    if (n < 1 || n_leaf < 1) return -1;
    int d = kd_depth(n, n_leaf);
    if (d > 30 || ((int64_t)2 << d) - 1 > max_slots) return -1;
    double *cx = NULL;
    if (periodic) {
        for (int a = 0; a < 3; a++)
            if (!(L[a] > 0.0)) return -1;
        cx = (double *)malloc(sizeof(double) * 3 * (size_t)n);
        for (int64_t i = 0; i < n; i++)
            for (int a = 0; a < 3; a++) cx[3 * i + a] = canon(x[3 * i + a], L[a]);
        x = cx;
    }
    otree t;
    if (kd_build(&t, x, n, n_leaf) != 0) { free(cx); return -1; }
    memcpy(start, t.start, sizeof(int64_t) * (size_t)t.nslots);
    memcpy(count, t.count, sizeof(int64_t) * (size_t)t.nslots);
    memcpy(axis, t.axis, sizeof(int) * (size_t)t.nslots);
    memcpy(box, t.box, sizeof(double) * 6 * (size_t)t.nslots);
    memcpy(ord, t.ord, sizeof(int64_t) * (size_t)n);
    kd_free(&t);
    free(cx);
    return d;
}
