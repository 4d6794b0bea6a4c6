/*
 * pbsm_parallel.c -- TEST AND BENCHMARK INFRASTRUCTURE, not the oracle: the
 * multi-core CPU evaluation of PBSM that the paper itself proposes
 * (Sec. 3.4, parallel processing), used as a CPU timing baseline on all of
 * the host's cores.  Only the benchmark's CPU leg and the tests load it;
 * the tests check its pairs against the oracle (sj_oracle.c).  It shares
 * no code with the oracle or with the CUDA library.
 *
 * The scheme, with m threads (OpenMP):
 *  Partitioning
 *   1. R and S are each divided into m equal contiguous parts;
 *   2. thread i counts, per tile, the rectangles of its part of R and of
 *      S (every tile a rectangle overlaps);
 *   3. the per-tile totals give each tile one segment per side, and each
 *      segment is divided among the threads by their counts (exclusive
 *      prefix over threads within the tile);
 *   4. thread i writes its parts into its ranges of the segments, so every
 *      tile's rectangles end up contiguous, with no locking.
 *  Joining
 *   5. one sorting task per tile and side (by x_l), spread over the threads;
 *   6. one join task per tile (the forward-scan plane sweep of Algorithm 1
 *      with the y-test, reporting a pair only in the tile that holds its
 *      reference point, Eq. 1), spread over the threads.
 *  Tasks are handed out dynamically, heaviest tiles included, so that the
 *  threads stay balanced.  Each thread appends its pairs to its own buffer.
 *
 * The tile of a coordinate v is clamp(floor((v - x0) * g), 0, n - 1) with
 * g = (float)n / (x1 - x0), the subtraction and the product each rounded to
 * float32 (build with -ffp-contract=off); the reference-point test compares
 * tile indices: the tile column of max(r.x_l, s.x_l) and the tile row of
 * max(r.y_l, s.y_l) must be the tile's own.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { float xl, yl, xu, yu; } pp_rect;
typedef struct { float xl, yl, xu, yu; int32_t id; } pp_ent;
typedef struct { int32_t r, s; } pp_pair;

typedef struct {
    pp_pair *p;
    int64_t n, cap;
    int failed;
} pp_buf;

static void buf_push(pp_buf *b, int32_t r, int32_t s)
{
    if (b->failed) return;
    if (b->n == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 4096;
        pp_pair *q = (pp_pair *)realloc(b->p, (size_t)nc * sizeof(pp_pair));
        if (!q) { b->failed = 1; return; }
        b->p = q;
        b->cap = nc;
    }
    b->p[b->n].r = r;
    b->p[b->n].s = s;
    b->n++;
}

typedef struct {
    int nx, ny;
    float x0, y0, gx, gy;
} pp_grid;

static int tile_of(float v, float v0, float g, int n)
{
    float t = (v - v0) * g;
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)n) return n - 1;
    int c = (int)floorf(t);
    return c > n - 1 ? n - 1 : c;
}

static int by_xl(const void *a, const void *b)
{
    const pp_ent *x = (const pp_ent *)a, *y = (const pp_ent *)b;
    return (x->xl > y->xl) - (x->xl < y->xl);
}

/* Steps 2-4 for one input: per-thread tile counts, per-(tile, thread)
 * write offsets, then the writes.  cnt: m * T counters (scratch), start:
 * T + 1 segment starts (out).  Returns the entries, NULL on allocation
 * failure. */
static pp_ent *partition(const pp_rect *A, int64_t n, const pp_grid *g, int m, int64_t *cnt, int64_t *start)
{
    const int64_t T = (int64_t)g->nx * g->ny;
#pragma omp parallel num_threads(m)
    {
        const int i = omp_get_thread_num();
        const int64_t a = n * i / m, b = n * (i + 1) / m;   /* step 1: equal parts */
        int64_t *c = cnt + (int64_t)i * T;
        memset(c, 0, (size_t)T * sizeof(int64_t));
        for (int64_t k = a; k < b; k++) {                   /* step 2: count */
            const int cx0 = tile_of(A[k].xl, g->x0, g->gx, g->nx), cx1 = tile_of(A[k].xu, g->x0, g->gx, g->nx);
            const int cy0 = tile_of(A[k].yl, g->y0, g->gy, g->ny), cy1 = tile_of(A[k].yu, g->y0, g->gy, g->ny);
            for (int cy = cy0; cy <= cy1; cy++)
                for (int cx = cx0; cx <= cx1; cx++) c[(int64_t)cy * g->nx + cx]++;
        }
    }
    /* step 3: tile totals (in parallel), segment starts (their prefix sum),
     * then each thread's offset inside every segment (cnt becomes offsets) */
#pragma omp parallel for num_threads(m) schedule(static)
    for (int64_t t = 0; t < T; t++) {
        int64_t tot = 0;
        for (int i = 0; i < m; i++) tot += cnt[(int64_t)i * T + t];
        start[t + 1] = tot;
    }
    start[0] = 0;
    for (int64_t t = 0; t < T; t++) start[t + 1] += start[t];
#pragma omp parallel for num_threads(m) schedule(static)
    for (int64_t t = 0; t < T; t++) {
        int64_t run = start[t];
        for (int i = 0; i < m; i++) {
            const int64_t v = cnt[(int64_t)i * T + t];
            cnt[(int64_t)i * T + t] = run;
            run += v;
        }
    }
    pp_ent *e = (pp_ent *)malloc((size_t)(start[T] ? start[T] : 1) * sizeof(pp_ent));
    if (!e) return NULL;
#pragma omp parallel num_threads(m)
    {
        const int i = omp_get_thread_num();
        const int64_t a = n * i / m, b = n * (i + 1) / m;
        int64_t *cur = cnt + (int64_t)i * T;
        for (int64_t k = a; k < b; k++) {                   /* step 4: write */
            const int cx0 = tile_of(A[k].xl, g->x0, g->gx, g->nx), cx1 = tile_of(A[k].xu, g->x0, g->gx, g->nx);
            const int cy0 = tile_of(A[k].yl, g->y0, g->gy, g->ny), cy1 = tile_of(A[k].yu, g->y0, g->gy, g->ny);
            for (int cy = cy0; cy <= cy1; cy++)
                for (int cx = cx0; cx <= cx1; cx++) {
                    pp_ent *d = &e[cur[(int64_t)cy * g->nx + cx]++];
                    d->xl = A[k].xl; d->yl = A[k].yl; d->xu = A[k].xu; d->yu = A[k].yu;
                    d->id = (int32_t)k;
                }
        }
    }
    return e;
}

/* Step 6 for tile (col, row): Algorithm 1 over the sorted segments. */
static void join_tile(const pp_ent *r, int64_t nr, const pp_ent *s, int64_t ns, const pp_grid *g, int col,
                      int row, pp_buf *out)
{
    int64_t i = 0, j = 0;
    while (i < nr && j < ns) {
        if (r[i].xl < s[j].xl) {   /* r first: scan s while s.x_l <= r.x_u */
            for (int64_t k = j; k < ns && s[k].xl <= r[i].xu; k++)
                if (r[i].yl <= s[k].yu && s[k].yl <= r[i].yu) {
                    const float mx = r[i].xl > s[k].xl ? r[i].xl : s[k].xl;
                    const float my = r[i].yl > s[k].yl ? r[i].yl : s[k].yl;
                    if (tile_of(mx, g->x0, g->gx, g->nx) == col && tile_of(my, g->y0, g->gy, g->ny) == row)
                        buf_push(out, r[i].id, s[k].id);
                }
            i++;
        } else {                   /* s first (ties too): scan r while r.x_l <= s.x_u */
            for (int64_t k = i; k < nr && r[k].xl <= s[j].xu; k++)
                if (r[k].yl <= s[j].yu && s[j].yl <= r[k].yu) {
                    const float mx = r[k].xl > s[j].xl ? r[k].xl : s[j].xl;
                    const float my = r[k].yl > s[j].yl ? r[k].yl : s[j].yl;
                    if (tile_of(mx, g->x0, g->gx, g->nx) == col && tile_of(my, g->y0, g->gy, g->ny) == row)
                        buf_push(out, r[k].id, s[j].id);
                }
            j++;
        }
    }
}

/* The whole join on m threads (m <= 0: all of OpenMP's threads).  Returns
 * the number of pairs (-1 on failure); if out is not NULL, *out receives a
 * malloc'ed array of the pairs (unordered), to be released with
 * pp_free. */
int64_t pp_pbsm(const pp_rect *R, int64_t nR, const pp_rect *S, int64_t nS, int nx, int ny, float x0, float y0,
                float x1, float y1, int m, pp_pair **out)
{
    if (nx < 1 || ny < 1 || !(x1 > x0) || !(y1 > y0)) return -1;
    if (m <= 0) m = omp_get_max_threads();
    pp_grid g;
    g.nx = nx; g.ny = ny; g.x0 = x0; g.y0 = y0;
    g.gx = (float)nx / (x1 - x0);
    g.gy = (float)ny / (y1 - y0);
    const int64_t T = (int64_t)nx * ny;
    int64_t *cnt = (int64_t *)malloc((size_t)(m * T) * sizeof(int64_t));
    int64_t *sr = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    int64_t *ss = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    pp_buf *bufs = (pp_buf *)calloc((size_t)m, sizeof(pp_buf));
    pp_ent *er = NULL, *es = NULL;
    int64_t total = -1;
    if (!cnt || !sr || !ss || !bufs) goto done;
    er = partition(R, nR, &g, m, cnt, sr);
    if (!er) goto done;
    es = partition(S, nS, &g, m, cnt, ss);
    if (!es) goto done;
#pragma omp parallel for num_threads(m) schedule(dynamic, 64)
    for (int64_t t = 0; t < 2 * T; t++) {                  /* step 5: sorting tasks */
        const int64_t u = t >> 1;
        pp_ent *e = (t & 1) ? es + ss[u] : er + sr[u];
        const int64_t k = (t & 1) ? ss[u + 1] - ss[u] : sr[u + 1] - sr[u];
        if (k > 1) qsort(e, (size_t)k, sizeof(pp_ent), by_xl);
    }
#pragma omp parallel for num_threads(m) schedule(dynamic, 64)
    for (int64_t t = 0; t < T; t++) {                      /* step 6: join tasks */
        const int64_t nr = sr[t + 1] - sr[t], ns = ss[t + 1] - ss[t];
        if (nr && ns)
            join_tile(er + sr[t], nr, es + ss[t], ns, &g, (int)(t % nx), (int)(t / nx), &bufs[omp_get_thread_num()]);
    }
    total = 0;
    for (int i = 0; i < m; i++) {
        if (bufs[i].failed) { total = -1; goto done; }
        total += bufs[i].n;
    }
    if (out) {
        pp_pair *all = (pp_pair *)malloc((size_t)(total ? total : 1) * sizeof(pp_pair));
        if (!all) { total = -1; goto done; }
        int64_t o = 0;
        for (int i = 0; i < m; i++) {
            if (bufs[i].n) memcpy(all + o, bufs[i].p, (size_t)bufs[i].n * sizeof(pp_pair));
            o += bufs[i].n;
        }
        *out = all;
    }
done:
    if (bufs)
        for (int i = 0; i < m; i++) free(bufs[i].p);
    free(bufs); free(cnt); free(sr); free(ss); free(er); free(es);
    return total;
}

void pp_free(void *p) { free(p); }

int pp_max_threads(void) { return omp_get_max_threads(); }
