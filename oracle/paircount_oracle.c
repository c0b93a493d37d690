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
 * Two drivers share that pair definition: a brute-force O(N1 N2) loop, and a
 * cell list with cells no smaller than the largest separation of interest
 * (Sect. 2.1: three passes -- bounds, per-cell counts, grouping -- then visit
 * each cell and its neighbours).  Threads work on disjoint rows or cells with
 * private histograms that are summed at the end, so integer counts do not
 * depend on the thread count.
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

static void *brute_worker(void *arg)
{
    job *jb = (job *)arg;
    const int64_t CH = 64;
    for (int64_t c0 = (int64_t)jb->tid * CH; c0 < jb->n1; c0 += (int64_t)jb->nthreads * CH) {
        int64_t c1 = c0 + CH < jb->n1 ? c0 + CH : jb->n1;
        for (int64_t i = c0; i < c1; i++) {
            int64_t j0 = jb->is_auto ? i + 1 : 0;
            for (int64_t j = j0; j < jb->n2; j++) add_pair(jb, i, j);
        }
    }
    return NULL;
}

static void *grid_worker(void *arg)
{
    job *jb = (job *)arg;
    const int *ng = jb->ng;
    for (int64_t a = jb->tid; a < jb->ncell; a += jb->nthreads) {
        int64_t a0 = jb->start1[a], a1 = jb->start1[a + 1];
        if (a0 == a1) continue;
        int ax = (int)(a % ng[0]);
        int ay = (int)((a / ng[0]) % ng[1]);
        int az = (int)(a / ((int64_t)ng[0] * ng[1]));
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
            for (int64_t p = a0; p < a1; p++) {
                int64_t i = jb->ord1[p];
                int64_t q0 = (jb->is_auto && b == a) ? p + 1 : b0;
                for (int64_t q = q0; q < b1; q++) add_pair(jb, i, jb->ord2[q]);
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
