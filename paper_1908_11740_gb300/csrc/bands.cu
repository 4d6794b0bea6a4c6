// bands.cu -- the share of one band of tile rows in a join.
//
// The tiles of the grid are independent join tasks and every pair is
// reported by exactly one tile, the one holding its reference point (Sec. 1,
// Sec. 3.2, Eq. 1).  So the pair set splits over any partition of the tile
// set, and a contiguous band of tile rows [row0, row1) is a unit that one GPU
// can join on its own: the union of the bands' pairs is the join, with no
// pair in two bands.  The band's pairs are computed from the rectangles that
// overlap its rows alone, on the unchanged grid:
//
//  1. k_band_mark_rects / k_band_write_rects: the rectangles of R (then S)
//     that overlap a tile row of the band (cell rows cy0 < row1 and
//     cy1 >= row0), copied in input order with their input indices (ballot
//     words, a count per chunk of 2048, the chunk offsets, an ordered write).
//     Invalid rectangles (NaN / Inf, xl > xu) are kept, so that the join
//     rejects them as it would the whole input;
//  2. the join of the selected rectangles (any mode), candidates in the
//     workspace.  Tiles outside the band receive only rectangles that cross
//     its border, so the work outside the band is small;
//  3. k_band_mark_pairs / k_band_write_pairs: a pair is kept when the row of
//     its reference tile, max(cy0_r, cy0_s) = cell(max(r.y_l, s.y_l)) (the
//     cell function is monotone), lies in the band; kept pairs are written in
//     candidate order with the input indices of both rectangles.
#define SJ_FILE_CODE 6
#include "sj_internal.h"

namespace sj {

constexpr int kBandThreads = 256;
constexpr int kBandPer = 8;
constexpr int kBandChunk = kBandThreads * kBandPer;   // items per CTA
constexpr int kBandWords = kBandChunk / 32;           // ballot words per chunk

// Item k of chunk c is c * 2048 + u * 256 + threadIdx.x (u < 8): its ballot
// word is c * 64 + u * 8 + warp.
__global__ void __launch_bounds__(kBandThreads) k_band_mark_rects(const float4 *__restrict__ A, long long n,
                                                                  GridDev g, int row0, int row1,
                                                                  unsigned *__restrict__ mask,
                                                                  unsigned *__restrict__ cnt) {
    __shared__ unsigned s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kBandChunk + threadIdx.x;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned mine = 0;
#pragma unroll
    for (int u = 0; u < kBandPer; u++) {
        const long long i = base + u * kBandThreads;
        bool keep = false;
        if (i < n) {
            const float4 m = ld_stream(A + i);
            if (!rect_ok(m)) {
                keep = true;
            } else {
                const int cy0 = cell_of(m.y, g.y0, g.gy, g.ny), cy1 = cell_of(m.w, g.y0, g.gy, g.ny);
                keep = cy0 < row1 && cy1 >= row0;
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) {
            mask[(size_t)blockIdx.x * kBandWords + u * (kBandThreads / 32) + warp] = b;
            mine += __popc(b);
        }
    }
    if (lane == 0 && mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = s_cnt;
}

// Exclusive prefix of the popcounts of a chunk's 64 ballot words (warp 0).
__device__ __forceinline__ void chunk_prefix(const unsigned *m, unsigned *s_pre) {
    const unsigned lane = threadIdx.x & 31;
    if ((threadIdx.x >> 5) == 0) {
        const unsigned a = __popc(m[2 * lane]), b = __popc(m[2 * lane + 1]);
        unsigned x = a + b;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        const unsigned ex = x - a - b;
        s_pre[2 * lane] = ex;
        s_pre[2 * lane + 1] = ex + a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBandThreads) k_band_write_rects(const float4 *__restrict__ A, long long n,
                                                                   const unsigned *__restrict__ mask,
                                                                   const unsigned long long *__restrict__ off,
                                                                   float4 *__restrict__ out,
                                                                   int *__restrict__ idx) {
    __shared__ unsigned s_pre[kBandWords];
    const unsigned *m = mask + (size_t)blockIdx.x * kBandWords;
    chunk_prefix(m, s_pre);
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;
    const unsigned long long o = off[blockIdx.x];
    const long long base = (long long)blockIdx.x * kBandChunk + threadIdx.x;
#pragma unroll
    for (int u = 0; u < kBandPer; u++) {
        const int w = u * (kBandThreads / 32) + warp;
        const unsigned b = m[w];
        const long long i = base + u * kBandThreads;
        if (((b >> lane) & 1u) && i < n) {
            const unsigned long long d = o + s_pre[w] + __popc(b & lt);
            out[d] = A[i];
            idx[d] = (int)i;
        }
    }
}

__global__ void __launch_bounds__(kBandThreads) k_band_mark_pairs(const int2 *__restrict__ cand, long long C,
                                                                  const float4 *__restrict__ R,
                                                                  const float4 *__restrict__ S, GridDev g,
                                                                  int row0, int row1, unsigned *__restrict__ mask,
                                                                  unsigned *__restrict__ cnt) {
    __shared__ unsigned s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kBandChunk + threadIdx.x;
    int2 c[kBandPer];
#pragma unroll
    for (int u = 0; u < kBandPer; u++) {
        const long long k = base + u * kBandThreads;
        c[u] = k < C ? __ldg(cand + k) : make_int2(-1, -1);
    }
    float yr[kBandPer], ys[kBandPer];
#pragma unroll
    for (int u = 0; u < kBandPer; u++)
        if (c[u].x >= 0) {
            yr[u] = __ldg(&R[c[u].x].y);
            ys[u] = __ldg(&S[c[u].y].y);
        }
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned mine = 0;
#pragma unroll
    for (int u = 0; u < kBandPer; u++) {
        bool keep = false;
        if (c[u].x >= 0) {
            const int row = cell_of(fmaxf(yr[u], ys[u]), g.y0, g.gy, g.ny);
            keep = row >= row0 && row < row1;
        }
        const unsigned b = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) {
            mask[(size_t)blockIdx.x * kBandWords + u * (kBandThreads / 32) + warp] = b;
            mine += __popc(b);
        }
    }
    if (lane == 0 && mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = s_cnt;
}

__global__ void __launch_bounds__(kBandThreads) k_band_write_pairs(const int2 *__restrict__ cand, long long C,
                                                                   const unsigned *__restrict__ mask,
                                                                   const unsigned long long *__restrict__ off,
                                                                   const int *__restrict__ ir,
                                                                   const int *__restrict__ is,
                                                                   int2 *__restrict__ out, Stats *st,
                                                                   unsigned long long cap) {
    __shared__ unsigned s_pre[kBandWords];
    const unsigned *m = mask + (size_t)blockIdx.x * kBandWords;
    chunk_prefix(m, s_pre);
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;
    const unsigned long long o = off[blockIdx.x];
    const long long base = (long long)blockIdx.x * kBandChunk + threadIdx.x;
#pragma unroll
    for (int u = 0; u < kBandPer; u++) {
        const int w = u * (kBandThreads / 32) + warp;
        const unsigned b = m[w];
        const long long k = base + u * kBandThreads;
        if (((b >> lane) & 1u) && k < C) {
            const int2 p = cand[k];
            const unsigned long long d = o + s_pre[w] + __popc(b & lt);
            if (SJ_IN(st, d, cap)) out[d] = make_int2(__ldg(ir + p.x), __ldg(is + p.y));
        }
    }
}

}  // namespace sj

using namespace sj;

namespace {

// Scratch of the ballot words, chunk counts and offsets for n items.
int band_scratch(sj_ctx *ctx, Workspace &w, long long n) {
    const long long nch = (n + kBandChunk - 1) / kBandChunk + 1;
    int st;
    if ((st = ensure(ctx, w.dmask, 4ull * kBandWords * nch))) return st;
    if ((st = ensure(ctx, w.dcnt, 4ull * nch + 16))) return st;
    if ((st = ensure(ctx, w.doff, 8ull * nch + 16))) return st;
    if ((st = ensure(ctx, w.dstats, 2 * sizeof(Stats)))) return st;
    return SJ_OK;
}

// Ordered selection of the rectangles of A overlapping rows [row0, row1):
// out / idx of the workspace; the count lands in dst->npairs.
int band_select(sj_ctx *ctx, Workspace &w, const float4 *A, long long n, const GridDev &g, int row0, int row1,
                Buf &out, Buf &idx, Stats *dst) {
    int st;
    if ((st = band_scratch(ctx, w, n))) return st;
    if ((st = ensure(ctx, out, 16ull * n + 16))) return st;
    if ((st = ensure(ctx, idx, 4ull * n + 16))) return st;
    const long long nch = (n + kBandChunk - 1) / kBandChunk;
    cudaError_t e;
    if (nch == 0) {
        if ((e = zero_async(ctx, &dst->npairs, sizeof(unsigned long long)))) return cuda_fail(ctx, e, "memset");
        return SJ_OK;
    }
    PhaseScope ph(ctx, PH_OTHER, 3);
    k_band_mark_rects<<<(unsigned)nch, kBandThreads, 0, ctx->stream>>>(A, n, g, row0, row1, (unsigned *)w.dmask.p,
                                                                       (unsigned *)w.dcnt.p);
    if ((e = launch_scan_pairs((const unsigned *)w.dcnt.p, (unsigned)nch, (unsigned long long *)w.doff.p, dst,
                               ctx->stream)))
        return cuda_fail(ctx, e, "band selection");
    k_band_write_rects<<<(unsigned)nch, kBandThreads, 0, ctx->stream>>>(
        A, n, (const unsigned *)w.dmask.p, (const unsigned long long *)w.doff.p, (float4 *)out.p, (int *)idx.p);
    if ((e = cudaGetLastError())) return cuda_fail(ctx, e, "band selection");
    return SJ_OK;
}

int rows_core(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS, const GridDev &gd,
              int row0, int row1, const sj_opts *o, OutSpec &os, int64_t *npairs) {
    Workspace &w = ctx->ws;
    int st;
    cudaError_t e;
    if ((st = ensure(ctx, w.dstats, 2 * sizeof(Stats)))) return st;
    Stats *dst = (Stats *)w.dstats.p;
    if ((st = band_select(ctx, w, (const float4 *)d_R, nR, gd, row0, row1, w.band_r, w.band_ir, dst))) return st;
    if ((st = band_select(ctx, w, (const float4 *)d_S, nS, gd, row0, row1, w.band_s, w.band_is, dst + 1)))
        return st;
    // the two sizes through the context's page-locked stats copy (two of its
    // 8-byte fields)
    Stats *hs = (Stats *)ctx->h_stats;
    if ((e = copy_async(ctx, &hs->npairs, &dst[0].npairs, 8)) || (e = copy_async(ctx, &hs->e_r, &dst[1].npairs, 8)))
        return cuda_fail(ctx, e, "copy of the band sizes");
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
    const long long mR = (long long)hs->npairs, mS = (long long)hs->e_r;
    // the join of the band's rectangles; candidates in the workspace, unsorted
    sj_opts oc{};
    if (o) {
        oc = *o;
        oc.sort_output = 0;
    }
    OutSpec cs{OutSpec::WS};
    int64_t C = 0;
    if ((st = join_core(ctx, w, (const sj_rect *)w.band_r.p, mR, (const sj_rect *)w.band_s.p, mS, gd, o ? &oc : nullptr,
                        cs, &C)))
        return st;
    const sj_stats inner = ctx->last;
    *npairs = 0;
    if (C == 0) {
        ctx->last.npairs = 0;
        return out_acquire(ctx, w, os, 0);
    }
    if ((st = band_scratch(ctx, w, C))) return st;
    const long long nch = (C + kBandChunk - 1) / kBandChunk;
    {
        PhaseScope ph(ctx, PH_OTHER, 2);
        k_band_mark_pairs<<<(unsigned)nch, kBandThreads, 0, ctx->stream>>>(
            cs.got, C, (const float4 *)w.band_r.p, (const float4 *)w.band_s.p, gd, row0, row1, (unsigned *)w.dmask.p,
            (unsigned *)w.dcnt.p);
        if ((e = launch_scan_pairs((const unsigned *)w.dcnt.p, (unsigned)nch, (unsigned long long *)w.doff.p, dst,
                                   ctx->stream)))
            return cuda_fail(ctx, e, "band pair filter");
    }
    if ((e = copy_async(ctx, &hs->npairs, &dst[0].npairs, 8))) return cuda_fail(ctx, e, "copy of the band count");
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
    const unsigned long long P = hs->npairs;
    *npairs = (int64_t)P;
    ctx->last = inner;
    ctx->last.npairs = (int64_t)P;
    if ((st = out_acquire(ctx, w, os, P))) return st;
    if (P == 0) return SJ_OK;
    {
        PhaseScope ph(ctx, PH_OTHER, 1);
        k_band_write_pairs<<<(unsigned)nch, kBandThreads, 0, ctx->stream>>>(
            cs.got, C, (const unsigned *)w.dmask.p, (const unsigned long long *)w.doff.p, (const int *)w.band_ir.p,
            (const int *)w.band_is.p, os.got, (Stats *)w.stats.p, P);
        if ((e = cudaGetLastError())) {
            out_abandon(ctx, os);
            return cuda_fail(ctx, e, "band pair write");
        }
    }
    if (o && o->sort_output && (st = sort_pairs(ctx, w, os.got, P))) {
        out_abandon(ctx, os);
        return st;
    }
    if ((st = check_tail(ctx, w))) out_abandon(ctx, os);
    return st;
}

int rows_check(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS, const sj_grid *g,
               int32_t row0, int32_t row1, const sj_opts *o, GridDev *gd) {
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, gd);
    if (st) return st;
    if ((st = check_opts(ctx, o))) return st;
    if (!(0 <= row0 && row0 <= row1 && row1 <= gd->ny))
        return fail(ctx, SJ_EINVAL, "row band [%d, %d) outside the grid's %d rows", row0, row1, gd->ny);
    return SJ_OK;
}

}  // namespace

extern "C" int sj_join_rows(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                            const sj_grid *g, int32_t row0, int32_t row1, const sj_opts *o, sj_pair **d_pairs,
                            int64_t *npairs) {
    GridDev gd;
    int st = rows_check(ctx, d_R, nR, d_S, nS, g, row0, row1, o, &gd);
    if (st) return st;
    if (!d_pairs || !npairs) return fail(ctx, SJ_EINVAL, "null output pointer");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    *d_pairs = nullptr;
    OutSpec os{OutSpec::LIB};
    if ((st = rows_core(ctx, d_R, nR, d_S, nS, gd, row0, row1, o, os, npairs))) return st;
    *d_pairs = (sj_pair *)os.got;
    return SJ_OK;
}

extern "C" int sj_join_rows_into(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                                 const sj_grid *g, int32_t row0, int32_t row1, const sj_opts *o, sj_pair *d_buf,
                                 int64_t cap, int64_t *npairs) {
    GridDev gd;
    int st = rows_check(ctx, d_R, nR, d_S, nS, g, row0, row1, o, &gd);
    if (st) return st;
    if (cap < 0 || !npairs) return fail(ctx, SJ_EINVAL, "negative capacity or null npairs");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    OutSpec os{OutSpec::INTO};
    os.into = d_buf;
    os.cap = cap;
    return rows_core(ctx, d_R, nR, d_S, nS, gd, row0, row1, o, os, npairs);
}
