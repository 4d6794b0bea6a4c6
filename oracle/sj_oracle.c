/*
 * sj_oracle.c -- TEST INFRASTRUCTURE: the plain, slow, single-threaded CPU
 * oracle for the filter step of the partitioning-based spatial join (PBSM) of
 * "Parallel In-Memory Evaluation of Spatial Joins" (Tsitsigkos, Bouros,
 * Mamoulis, Terrovitis).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no code, header or constant with the CUDA
 * library; neither includes the other.  Build: plain C, -O2
 * -ffp-contract=off, no fast-math (so float compares and the two float
 * operations of the cell function are exactly IEEE single precision).
 *
 * What it computes (Sec. 1): J = {(i,j) : R[i] and S[j] have at least one
 * common point}, i.e. the closed test
 *     R.xl <= S.xu && S.xl <= R.xu && R.yl <= S.yu && S.yl <= R.yu
 * on the float32 values as given.  Three independent routes reach J:
 *   orc_brute  -- the definition, all |R||S| pairs (tiny inputs only);
 *   orc_sweep  -- Algorithm 1 (forward-scan plane sweep, Sec. 2.1) over the
 *                 whole space, no partitioning;
 *   orc_pbsm   -- PBSM on a uniform nx x ny grid (Sec. 1, Sec. 2.2): every
 *                 rectangle is copied into every tile it overlaps (counted
 *                 first, then written, Sec. 3.4 steps 2-4), each tile is
 *                 sorted by x_l and joined with Algorithm 1, and a pair is
 *                 reported only where its reference point lies (Eq. 1).
 * All three return the pairs sorted by (r, s).  orc_pbsm_gbda is PBSM with the
 * grouping-based duplicate avoidance instead of the test of Eq. 1 (class
 * groups per tile, 9 of the 16 group-group joins, no duplicate test).
 * orc_pbsm_digest runs orc_pbsm
 * but folds every reported pair into an order-independent digest (count,
 * sum and xor of a 64-bit mix of the pair) instead of storing it, for
 * result sets too large to hold on the host (1e9 pairs).
 *
 * Readings of the paper used here:
 *  - Tile membership: cell(v) = clamp(floor((v - g0) * ginv), 0, n-1), with
 *    ginv = (float)n / (g1 - g0) and the subtraction and product rounded
 *    to float32.  The function is monotone in v, so it partitions the line;
 *    coordinates outside [g0, g1] fall into the border tiles.
 *  - Eq. 1 ("max{r.xl,s.xl} >= T.xl and max{r.yl,s.yl} >= T.yl") is taken
 *    in tile-index form: cell_x(max xl) >= col and cell_y(max yl) >= row.
 *    With the lower bound of tile col read as "the first value whose cell is
 *    col", this is Eq. 1 exactly, and it avoids a float T.x_l that could
 *    round differently from the assignment.  Both rectangles lie in the tile,
 *    so ">=" can only hold as "==": the pair is reported in exactly one tile.
 *  - The "top-left corner" of the prose is the lower corner of Eq. 1 (y axis
 *    pointing down in the figure); Eq. 1 is followed.
 *  - Ties r.x_l == s.x_l make s the pivot (the strict "<" of Algorithm 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { float xl, yl, xu, yu; } orc_rect;
typedef struct { float xl, yl, xu, yu; int32_t id; } orc_ent;
typedef struct { int32_t r, s; } orc_pair;

typedef struct {
    orc_pair *p;
    int64_t n, cap;
    int failed;
    int digest;        /* 1: pairs are folded into (n, sum, xr), not stored */
    uint64_t sum, xr;
} orc_res;

/* ---- result buffer --------------------------------------------------- */
/* The output function of SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): a bijective 64-bit mixer.
 * The digest of a pair set is (count, sum of mix(key) mod 2^64, xor of
 * mix(key)) with key = (uint32)r << 32 | (uint32)s: it does not depend on the
 * order of the pairs, and a changed, missing or repeated pair changes it. */
static uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static void res_push(orc_res *res, int32_t r, int32_t s)
{
    if (res->failed) return;
    if (res->digest) {
        uint64_t h = mix64(((uint64_t)(uint32_t)r << 32) | (uint64_t)(uint32_t)s);
        res->n++;
        res->sum += h;
        res->xr ^= h;
        return;
    }
    if (res->n == res->cap) {
        int64_t nc = res->cap ? 2 * res->cap : 1024;
        orc_pair *q = (orc_pair *)realloc(res->p, (size_t)nc * sizeof(orc_pair));
        if (!q) { res->failed = 1; return; }
        res->p = q;
        res->cap = nc;
    }
    res->p[res->n].r = r;
    res->p[res->n].s = s;
    res->n++;
}

static int cmp_pair(const void *a, const void *b)
{
    const orc_pair *x = (const orc_pair *)a, *y = (const orc_pair *)b;
    if (x->r != y->r) return x->r < y->r ? -1 : 1;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    return 0;
}

static orc_res *res_new(void) { return (orc_res *)calloc(1, sizeof(orc_res)); }

static orc_res *res_finish(orc_res *res)
{
    if (!res->digest && res->n > 1) qsort(res->p, (size_t)res->n, sizeof(orc_pair), cmp_pair);
    return res;
}

int64_t orc_res_count(const orc_res *res) { return res ? res->n : -1; }
int orc_res_failed(const orc_res *res) { return res ? res->failed : 1; }
void orc_res_copy(const orc_res *res, int32_t *out)
{
    if (res->n) memcpy(out, res->p, (size_t)res->n * sizeof(orc_pair));
}
void orc_res_free(orc_res *res)
{
    if (!res) return;
    free(res->p);
    free(res);
}

/* ---- the intersection test (Sec. 1: at least one common point) ------- */
static int y_intersects(float ryl, float ryu, float syl, float syu)
{
    return ryl <= syu && syl <= ryu;
}

/* Definition, all pairs. */
orc_res *orc_brute(const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS)
{
    orc_res *res = res_new();
    if (!res) return NULL;
    for (int64_t i = 0; i < nR; i++)
        for (int64_t j = 0; j < nS; j++)
            if (R[i].xl <= S[j].xu && S[j].xl <= R[i].xu &&
                R[i].yl <= S[j].yu && S[j].yl <= R[i].yu)
                res_push(res, (int32_t)i, (int32_t)j);
    return res_finish(res);
}

/* ---- Algorithm 1 ----------------------------------------------------- */
static int cmp_ent_xl(const void *a, const void *b)
{
    const orc_ent *x = (const orc_ent *)a, *y = (const orc_ent *)b;
    if (x->xl < y->xl) return -1;
    if (x->xl > y->xl) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Duplicate test context of one tile (Eq. 1 in tile-index form).  When
 * `on` is 0 every candidate that intersects is reported (whole space). */
typedef struct {
    int on;
    int col, row, nx, ny;
    float gx0, gy0, ginvx, ginvy;
} dedup_ctx;

static int cell_of(float v, float g0, float ginv, int n)
{
    float t = (v - g0) * ginv;     /* two float32 roundings, no contraction */
    float f = floorf(t);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(n - 1)) return n - 1;
    return (int)f;
}

static int report_here(const dedup_ctx *d, const orc_ent *r, const orc_ent *s)
{
    if (!d->on) return 1;
    float mx = r->xl > s->xl ? r->xl : s->xl;
    float my = r->yl > s->yl ? r->yl : s->yl;
    return cell_of(mx, d->gx0, d->ginvx, d->nx) >= d->col &&
           cell_of(my, d->gy0, d->ginvy, d->ny) >= d->row;
}

/* Forward-scan plane sweep of R and S, both already sorted by x_l. */
static void alg1(const orc_ent *R, int64_t nr, const orc_ent *S, int64_t ns,
                 const dedup_ctx *d, orc_res *res, int64_t *ncand)
{
    int64_t i = 0, j = 0, cand = 0;
    while (i < nr && j < ns) {
        if (R[i].xl < S[j].xl) {
            /* r = R[i] is the pivot; scan S forward from s = S[j]. */
            for (int64_t k = j; k < ns && R[i].xu >= S[k].xl; k++) {
                cand++;
                if (y_intersects(R[i].yl, R[i].yu, S[k].yl, S[k].yu) &&
                    report_here(d, &R[i], &S[k]))
                    res_push(res, R[i].id, S[k].id);
            }
            i++;
        } else {
            /* s = S[j] is the pivot; scan R forward from r = R[i]. */
            for (int64_t k = i; k < nr && S[j].xu >= R[k].xl; k++) {
                cand++;
                if (y_intersects(R[k].yl, R[k].yu, S[j].yl, S[j].yu) &&
                    report_here(d, &R[k], &S[j]))
                    res_push(res, R[k].id, S[j].id);
            }
            j++;
        }
    }
    if (ncand) *ncand += cand;
}

static orc_ent *to_entries(const orc_rect *A, int64_t n)
{
    orc_ent *e = (orc_ent *)malloc((size_t)(n ? n : 1) * sizeof(orc_ent));
    if (!e) return NULL;
    for (int64_t i = 0; i < n; i++) {
        e[i].xl = A[i].xl; e[i].yl = A[i].yl;
        e[i].xu = A[i].xu; e[i].yu = A[i].yu;
        e[i].id = (int32_t)i;
    }
    return e;
}

/* Algorithm 1 over the whole space (no partitioning, no duplicates). */
orc_res *orc_sweep(const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS,
                   int64_t *ncand)
{
    orc_res *res = res_new();
    orc_ent *er = to_entries(R, nR), *es = to_entries(S, nS);
    if (!res || !er || !es) { free(er); free(es); orc_res_free(res); return NULL; }
    qsort(er, (size_t)nR, sizeof(orc_ent), cmp_ent_xl);   /* Alg. 1, line "sort" */
    qsort(es, (size_t)nS, sizeof(orc_ent), cmp_ent_xl);
    dedup_ctx d;
    memset(&d, 0, sizeof d);
    if (ncand) *ncand = 0;
    alg1(er, nR, es, nS, &d, res, ncand);
    free(er);
    free(es);
    return res_finish(res);
}

/* ---- PBSM on a uniform grid ------------------------------------------ */
typedef struct {
    int nx, ny;
    float gx0, gy0, ginvx, ginvy;
} grid_t;

static grid_t make_grid(int nx, int ny, float x0, float y0, float x1, float y1)
{
    grid_t g;
    g.nx = nx; g.ny = ny;
    g.gx0 = x0; g.gy0 = y0;
    g.ginvx = (float)nx / (x1 - x0);
    g.ginvy = (float)ny / (y1 - y0);
    return g;
}

/* Partitioning phase for one collection (Sec. 3.4 steps 2-4, one thread):
 * count per tile, prefix-sum to segment starts, then write each rectangle
 * into every tile it overlaps.  cnt has nx*ny slots, off nx*ny+1. */
static orc_ent *partition(const orc_rect *A, int64_t n, const grid_t *g,
                          int64_t *cnt, int64_t *off)
{
    int64_t T = (int64_t)g->nx * g->ny;
    memset(cnt, 0, (size_t)T * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int cx0 = cell_of(A[i].xl, g->gx0, g->ginvx, g->nx);
        int cx1 = cell_of(A[i].xu, g->gx0, g->ginvx, g->nx);
        int cy0 = cell_of(A[i].yl, g->gy0, g->ginvy, g->ny);
        int cy1 = cell_of(A[i].yu, g->gy0, g->ginvy, g->ny);
        for (int cy = cy0; cy <= cy1; cy++)
            for (int cx = cx0; cx <= cx1; cx++)
                cnt[(int64_t)cy * g->nx + cx]++;
    }
    off[0] = 0;
    for (int64_t t = 0; t < T; t++) off[t + 1] = off[t] + cnt[t];
    orc_ent *e = (orc_ent *)malloc((size_t)(off[T] ? off[T] : 1) * sizeof(orc_ent));
    int64_t *cur = (int64_t *)malloc((size_t)(T ? T : 1) * sizeof(int64_t));
    if (!e || !cur) { free(e); free(cur); return NULL; }
    memcpy(cur, off, (size_t)T * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int cx0 = cell_of(A[i].xl, g->gx0, g->ginvx, g->nx);
        int cx1 = cell_of(A[i].xu, g->gx0, g->ginvx, g->nx);
        int cy0 = cell_of(A[i].yl, g->gy0, g->ginvy, g->ny);
        int cy1 = cell_of(A[i].yu, g->gy0, g->ginvy, g->ny);
        for (int cy = cy0; cy <= cy1; cy++)
            for (int cx = cx0; cx <= cx1; cx++) {
                orc_ent *d = &e[cur[(int64_t)cy * g->nx + cx]++];
                d->xl = A[i].xl; d->yl = A[i].yl;
                d->xu = A[i].xu; d->yu = A[i].yu;
                d->id = (int32_t)i;
            }
    }
    free(cur);
    return e;
}

/* Optional per-tile outputs: tile_cnt_r/s (|R_T|, |S_T|) and tile_pairs
 * (pairs reported by tile T); each nx*ny long, or NULL. */
static orc_res *pbsm_into(orc_res *res, const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS,
                          int nx, int ny, float x0, float y0, float x1, float y1,
                          int64_t *tile_cnt_r, int64_t *tile_cnt_s, int64_t *tile_pairs,
                          int64_t *ncand)
{
    if (!res) return NULL;
    if (nx < 1 || ny < 1 || !(x1 > x0) || !(y1 > y0)) { orc_res_free(res); return NULL; }
    grid_t g = make_grid(nx, ny, x0, y0, x1, y1);
    int64_t T = (int64_t)nx * ny;
    int64_t *cr = (int64_t *)malloc((size_t)T * sizeof(int64_t));
    int64_t *cs = (int64_t *)malloc((size_t)T * sizeof(int64_t));
    int64_t *orr = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    int64_t *os = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    orc_ent *er = NULL, *es = NULL;
    if (!cr || !cs || !orr || !os) goto fail;
    er = partition(R, nR, &g, cr, orr);
    es = partition(S, nS, &g, cs, os);
    if (!er || !es) goto fail;
    if (ncand) *ncand = 0;
    /* Joining phase (Sec. 3.4 steps 5-6): per tile, sort both sides by x_l,
     * then Algorithm 1 with the duplicate test of Eq. 1. */
    for (int64_t t = 0; t < T; t++) {
        orc_ent *rt = er + orr[t], *st = es + os[t];
        int64_t nr = cr[t], ns = cs[t];
        if (tile_cnt_r) tile_cnt_r[t] = nr;
        if (tile_cnt_s) tile_cnt_s[t] = ns;
        int64_t before = res->n;
        if (nr && ns) {
            qsort(rt, (size_t)nr, sizeof(orc_ent), cmp_ent_xl);
            qsort(st, (size_t)ns, sizeof(orc_ent), cmp_ent_xl);
            dedup_ctx d;
            d.on = 1;
            d.col = (int)(t % nx);
            d.row = (int)(t / nx);
            d.nx = nx; d.ny = ny;
            d.gx0 = g.gx0; d.gy0 = g.gy0;
            d.ginvx = g.ginvx; d.ginvy = g.ginvy;
            alg1(rt, nr, st, ns, &d, res, ncand);
        }
        if (tile_pairs) tile_pairs[t] = res->n - before;
    }
    free(cr); free(cs); free(orr); free(os); free(er); free(es);
    return res_finish(res);
fail:
    free(cr); free(cs); free(orr); free(os); free(er); free(es);
    orc_res_free(res);
    return NULL;
}

orc_res *orc_pbsm_ex(const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS,
                     int nx, int ny, float x0, float y0, float x1, float y1,
                     int64_t *tile_cnt_r, int64_t *tile_cnt_s, int64_t *tile_pairs,
                     int64_t *ncand)
{
    return pbsm_into(res_new(), R, nR, S, nS, nx, ny, x0, y0, x1, y1, tile_cnt_r, tile_cnt_s, tile_pairs,
                     ncand);
}

/* PBSM as above, with the pairs folded into their digest (see mix64) instead
 * of stored: out[0] = pairs, out[1] = sum, out[2] = xor.  For result sets too
 * large to hold (the 1e9-pair joins).  Returns 0, or -1 on bad arguments or
 * allocation failure. */
int orc_pbsm_digest(const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS,
                    int nx, int ny, float x0, float y0, float x1, float y1, uint64_t *out)
{
    orc_res *res = res_new();
    if (!res) return -1;
    res->digest = 1;
    res = pbsm_into(res, R, nR, S, nS, nx, ny, x0, y0, x1, y1, NULL, NULL, NULL, NULL);
    if (!res) return -1;
    out[0] = (uint64_t)res->n;
    out[1] = res->sum;
    out[2] = res->xr;
    orc_res_free(res);
    return 0;
}

orc_res *orc_pbsm(const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS,
                  int nx, int ny, float x0, float y0, float x1, float y1)
{
    return orc_pbsm_ex(R, nR, S, nS, nx, ny, x0, y0, x1, y1, NULL, NULL, NULL, NULL);
}

/* ---- GBDA: duplicate avoidance by mini-joins of rectangle classes --------
 * Each tile's rectangles of R (and of S) are divided into four classes by
 * where their projections begin (the section on grouping-based duplicate
 * avoidance that follows Eq. 1):
 *   A: x_l >= T.x_l and y_l >= T.y_l     B: x_l >= T.x_l and y_l < T.y_l
 *   C: x_l <  T.x_l and y_l >= T.y_l     D: x_l <  T.x_l and y_l < T.y_l
 * ("v >= T.x_l" read as cell(v) >= the tile's column, as for Eq. 1).  Of the
 * 16 group-group joins, the 7 that can only produce pairs reported in an
 * earlier tile are not evaluated; the 9 below are, each with Algorithm 1 on
 * the two groups sorted by x_l, and with no duplicate test. */
enum { CL_A = 0, CL_B = 1, CL_C = 2, CL_D = 3 };
static const int gbda_joins[][2] = {
    {CL_A, CL_A}, {CL_A, CL_B}, {CL_A, CL_C}, {CL_A, CL_D},
    {CL_B, CL_A}, {CL_C, CL_A}, {CL_D, CL_A},
    {CL_B, CL_C}, {CL_C, CL_B},
};

static int gbda_class(const orc_ent *e, int col, int row, const grid_t *g)
{
    int xin = cell_of(e->xl, g->gx0, g->ginvx, g->nx) >= col;
    int yin = cell_of(e->yl, g->gy0, g->ginvy, g->ny) >= row;
    if (xin && yin) return CL_A;
    if (xin) return CL_B;
    if (yin) return CL_C;
    return CL_D;
}

/* Stable split of one tile's entries into the four class groups (written to
 * out, group k at out + start[k], start[4] = n). */
static void gbda_groups(const orc_ent *E, int64_t n, int col, int row, const grid_t *g,
                        orc_ent *out, int64_t *start)
{
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int64_t k = 0; k < n; k++) cnt[gbda_class(&E[k], col, row, g)]++;
    start[0] = 0;
    for (int c = 0; c < 4; c++) start[c + 1] = start[c] + cnt[c];
    int64_t cur[4] = {start[0], start[1], start[2], start[3]};
    for (int64_t k = 0; k < n; k++) out[cur[gbda_class(&E[k], col, row, g)]++] = E[k];
}

orc_res *orc_pbsm_gbda(const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS,
                       int nx, int ny, float x0, float y0, float x1, float y1)
{
    if (nx < 1 || ny < 1 || !(x1 > x0) || !(y1 > y0)) return NULL;
    grid_t g = make_grid(nx, ny, x0, y0, x1, y1);
    int64_t T = (int64_t)nx * ny;
    int64_t *cr = (int64_t *)malloc((size_t)T * sizeof(int64_t));
    int64_t *cs = (int64_t *)malloc((size_t)T * sizeof(int64_t));
    int64_t *orr = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    int64_t *os = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    orc_res *res = res_new();
    orc_ent *er = NULL, *es = NULL, *gr = NULL, *gs = NULL;
    if (!cr || !cs || !orr || !os || !res) goto fail;
    er = partition(R, nR, &g, cr, orr);
    es = partition(S, nS, &g, cs, os);
    if (!er || !es) goto fail;
    gr = (orc_ent *)malloc((size_t)(orr[T] ? orr[T] : 1) * sizeof(orc_ent));
    gs = (orc_ent *)malloc((size_t)(os[T] ? os[T] : 1) * sizeof(orc_ent));
    if (!gr || !gs) goto fail;
    dedup_ctx none;
    memset(&none, 0, sizeof none);   /* no duplicate test */
    for (int64_t t = 0; t < T; t++) {
        int64_t nr = cr[t], ns = cs[t];
        if (!nr || !ns) continue;
        int col = (int)(t % nx), row = (int)(t / nx);
        int64_t sr[5], ss[5];
        orc_ent *rt = gr + orr[t], *st = gs + os[t];
        gbda_groups(er + orr[t], nr, col, row, &g, rt, sr);
        gbda_groups(es + os[t], ns, col, row, &g, st, ss);
        for (int c = 0; c < 4; c++) {
            qsort(rt + sr[c], (size_t)(sr[c + 1] - sr[c]), sizeof(orc_ent), cmp_ent_xl);
            qsort(st + ss[c], (size_t)(ss[c + 1] - ss[c]), sizeof(orc_ent), cmp_ent_xl);
        }
        for (size_t k = 0; k < sizeof gbda_joins / sizeof gbda_joins[0]; k++) {
            int a = gbda_joins[k][0], b = gbda_joins[k][1];
            alg1(rt + sr[a], sr[a + 1] - sr[a], st + ss[b], ss[b + 1] - ss[b], &none, res, NULL);
        }
    }
    free(cr); free(cs); free(orr); free(os); free(er); free(es); free(gr); free(gs);
    return res_finish(res);
fail:
    free(cr); free(cs); free(orr); free(os); free(er); free(es); free(gr); free(gs);
    orc_res_free(res);
    return NULL;
}

/* ---- sweep axis of a tile (Sec. 3.3, Eq. 2) ---------------------------
 * The x-projection of tile T is split into k = 8 equal divisions (and the
 * y-projection alike).  H_R^x[i] counts the rectangles of R_T whose
 * x-projection intersects division i; I^x_T = sum_i H_R^x[i] * H_S^x[i]
 * estimates the x-intersecting pairs of R_T x S_T (Eq. 2, read with i = 0..k-1).
 * The tile is swept along y when I^y_T < I^x_T, else along x (ties and tiles
 * without both sides: x).  All of the tile's rectangles are counted (no
 * sampling).
 * Reading: division i of tile column c is the set of coordinates v whose
 * cell-function value t(v) = (v - g0) * ginv (float32, as in cell_of) lies in
 * [c + i/8, c + (i+1)/8); the projection [xl, xu] intersects it when
 * 8 t(xl) < 8c + i + 1 and 8 t(xu) >= 8c + i (8 t is exact in float32).  A
 * rectangle assigned to the tile always intersects at least one division. */
static void tile_histogram(const orc_ent *E, int64_t n, int col, float g0, float ginv, int axis,
                           int64_t *h)
{
    for (int i = 0; i < 8; i++) h[i] = 0;
    for (int64_t k = 0; k < n; k++) {
        float lo = axis ? E[k].yl : E[k].xl, hi = axis ? E[k].yu : E[k].xu;
        float tl = (lo - g0) * ginv, tu = (hi - g0) * ginv;
        for (int i = 0; i < 8; i++) {
            float a = (float)(8 * col + i);
            if (8.0f * tl < a + 1.0f && 8.0f * tu >= a) h[i]++;
        }
    }
}

/* Per tile (row-major, nx*ny): axis[t] = 1 when tile t is swept along y;
 * ix / iy (optional, int64) receive I^x_T and I^y_T. */
int orc_tile_axes(const orc_rect *R, int64_t nR, const orc_rect *S, int64_t nS,
                  int nx, int ny, float x0, float y0, float x1, float y1,
                  uint8_t *axis, int64_t *ix, int64_t *iy)
{
    if (nx < 1 || ny < 1 || !(x1 > x0) || !(y1 > y0)) return -1;
    grid_t g = make_grid(nx, ny, x0, y0, x1, y1);
    int64_t T = (int64_t)nx * ny;
    int64_t *cr = (int64_t *)malloc((size_t)T * sizeof(int64_t));
    int64_t *cs = (int64_t *)malloc((size_t)T * sizeof(int64_t));
    int64_t *orr = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    int64_t *os = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    orc_ent *er = NULL, *es = NULL;
    int rc = -1;
    if (!cr || !cs || !orr || !os) goto done;
    er = partition(R, nR, &g, cr, orr);
    es = partition(S, nS, &g, cs, os);
    if (!er || !es) goto done;
    for (int64_t t = 0; t < T; t++) {
        int col = (int)(t % nx), row = (int)(t / nx);
        int64_t hrx[8], hsx[8], hry[8], hsy[8], sx = 0, sy = 0;
        tile_histogram(er + orr[t], cr[t], col, g.gx0, g.ginvx, 0, hrx);
        tile_histogram(es + os[t], cs[t], col, g.gx0, g.ginvx, 0, hsx);
        tile_histogram(er + orr[t], cr[t], row, g.gy0, g.ginvy, 1, hry);
        tile_histogram(es + os[t], cs[t], row, g.gy0, g.ginvy, 1, hsy);
        for (int i = 0; i < 8; i++) {
            sx += hrx[i] * hsx[i];
            sy += hry[i] * hsy[i];
        }
        axis[t] = (uint8_t)(cr[t] > 0 && cs[t] > 0 && sy < sx);
        if (ix) ix[t] = sx;
        if (iy) iy[t] = sy;
    }
    rc = 0;
done:
    free(cr); free(cs); free(orr); free(os); free(er); free(es);
    return rc;
}

/* The cell function alone, for tests of the per-tile counts. */
int orc_cell(float v, float g0, float g1, int n)
{
    float ginv = (float)n / (g1 - g0);
    return cell_of(v, g0, ginv, n);
}

/* Per-tile counts of one collection (Sec. 3.4 step 2), int64[nx*ny]. */
void orc_tile_counts(const orc_rect *A, int64_t n, int nx, int ny,
                     float x0, float y0, float x1, float y1, int64_t *cnt)
{
    grid_t g = make_grid(nx, ny, x0, y0, x1, y1);
    int64_t T = (int64_t)nx * ny;
    memset(cnt, 0, (size_t)T * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int cx0 = cell_of(A[i].xl, g.gx0, g.ginvx, nx);
        int cx1 = cell_of(A[i].xu, g.gx0, g.ginvx, nx);
        int cy0 = cell_of(A[i].yl, g.gy0, g.ginvy, ny);
        int cy1 = cell_of(A[i].yu, g.gy0, g.ginvy, ny);
        for (int cy = cy0; cy <= cy1; cy++)
            for (int cx = cx0; cx <= cx1; cx++)
                cnt[(int64_t)cy * nx + cx]++;
    }
}

/* The four cells (cx0, cx1, cy0, cy1) of every rectangle, int32[n][4]. */
void orc_cells(const orc_rect *A, int64_t n, int nx, int ny, float x0, float y0, float x1, float y1,
               int32_t *out)
{
    grid_t g = make_grid(nx, ny, x0, y0, x1, y1);
    for (int64_t i = 0; i < n; i++) {
        out[4 * i + 0] = cell_of(A[i].xl, g.gx0, g.ginvx, nx);
        out[4 * i + 1] = cell_of(A[i].xu, g.gx0, g.ginvx, nx);
        out[4 * i + 2] = cell_of(A[i].yl, g.gy0, g.ginvy, ny);
        out[4 * i + 3] = cell_of(A[i].yu, g.gy0, g.ginvy, ny);
    }
}

/* ---- epsilon-distance join on point sets (Sec. 1) ---------------------
 * What it computes: J_eps = {(i,j) : |P[i] - Q[j]| <= eps}, the Euclidean
 * distance between two float32 points.  The paper notes that an
 * intersection join answers it: every point becomes a square of side eps
 * centred on it, the squares are joined, and each intersecting pair is
 * refined by its distance.
 *
 * Readings:
 *  - The distance test is evaluated in IEEE binary64 in one fixed order:
 *    dx = x_p - x_q, dy = y_p - y_q, d2 = dx*dx + dy*dy (each operation
 *    rounded once, no fused multiply-add), accepted when d2 <= eps*eps
 *    (eps widened to binary64, its square rounded once).  The paper fixes no
 *    precision; with this order the decision is a plain function of the
 *    inputs.
 *  - The square is built so that it holds the exact square of side eps:
 *    half-width h >= eps/2 * (1 + 2^-21), corners rounded outward to float32
 *    (one float32 step beyond the nearest value).
 *    An accepted pair has |dx|, |dy| <= eps * (1 + 2^-50) (binary64 rounding
 *    error), so its squares intersect: the filter loses no pair.  Wider
 *    squares only add candidates, which the test removes. */
typedef struct { float x, y; } orc_point;

static int within_eps(orc_point p, orc_point q, double e2)
{
    double dx = (double)p.x - (double)q.x;
    double dy = (double)p.y - (double)q.y;
    double d2 = dx * dx + dy * dy;
    return d2 <= e2;
}

/* Definition, all pairs. */
orc_res *orc_dist_brute(const orc_point *P, int64_t nP, const orc_point *Q, int64_t nQ, float eps)
{
    orc_res *res = res_new();
    if (!res) return NULL;
    double e2 = (double)eps * (double)eps;
    for (int64_t i = 0; i < nP; i++)
        for (int64_t j = 0; j < nQ; j++)
            if (within_eps(P[i], Q[j], e2)) res_push(res, (int32_t)i, (int32_t)j);
    return res_finish(res);
}

/* The square around every point (see the readings above). */
void orc_dist_squares(const orc_point *P, int64_t n, float eps, orc_rect *out)
{
    float h = (float)((double)eps * 0.5 * (1.0 + 0x1p-20));
    h = nextafterf(h, INFINITY);   /* the cast may have rounded down */
    for (int64_t i = 0; i < n; i++) {
        out[i].xl = nextafterf(P[i].x - h, -INFINITY);
        out[i].xu = nextafterf(P[i].x + h, INFINITY);
        out[i].yl = nextafterf(P[i].y - h, -INFINITY);
        out[i].yu = nextafterf(P[i].y + h, INFINITY);
    }
}

/* The paper's route: squares, PBSM on an nx x ny grid (the filter), then
 * the distance test of every reported pair.  *ncand (if not NULL) receives
 * the number of intersecting square pairs. */
orc_res *orc_dist_pbsm(const orc_point *P, int64_t nP, const orc_point *Q, int64_t nQ, float eps,
                       int nx, int ny, float x0, float y0, float x1, float y1, int64_t *ncand)
{
    orc_rect *sp = (orc_rect *)malloc((size_t)(nP ? nP : 1) * sizeof(orc_rect));
    orc_rect *sq = (orc_rect *)malloc((size_t)(nQ ? nQ : 1) * sizeof(orc_rect));
    orc_res *cand = NULL, *res = res_new();
    if (!sp || !sq || !res) goto fail;
    orc_dist_squares(P, nP, eps, sp);
    orc_dist_squares(Q, nQ, eps, sq);
    cand = orc_pbsm_ex(sp, nP, sq, nQ, nx, ny, x0, y0, x1, y1, NULL, NULL, NULL, NULL);
    if (!cand || cand->failed) goto fail;
    if (ncand) *ncand = cand->n;
    double e2 = (double)eps * (double)eps;
    for (int64_t k = 0; k < cand->n; k++) {
        orc_pair c = cand->p[k];
        if (within_eps(P[c.r], Q[c.s], e2)) res_push(res, c.r, c.s);
    }
    free(sp); free(sq);
    orc_res_free(cand);
    return res_finish(res);
fail:
    free(sp); free(sq);
    orc_res_free(cand);
    orc_res_free(res);
    return NULL;
}
