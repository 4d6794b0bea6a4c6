// sortpairs.cu -- the sorted output of sj_opts.sort_output: the pairs of a
// join in ascending (r, s) order, sorted on the device.
//
// Stable least-significant-digit radix sort of the int2 pairs, 8 passes of
// 8-bit digits: s bits 0-7, 8-15, 16-23, 24-31, then r bits 0-7 .. 24-31
// (ids are below 2^30, so the key (r, s) is exactly the order of the digit
// sequence read from r's top digit down).  Each pass:
//   1. k_ps_hist: the digit histogram of every tile of 8192 pairs, stored
//      digit-major (hist[d * nT + tile]);
//   2. k_ps_scan_part / k_ps_scan_top / k_ps_scan_fill: exclusive scan of
//      that table, so hist[d * nT + tile] becomes the first output slot of
//      tile's pairs with digit d;
//   3. k_ps_scatter: every warp of a tile owns 1024 consecutive pairs; it
//      counts its digits, the tile turns those counts into per-warp starts,
//      and the warp walks its pairs 32 at a time in order, placing each pair
//      at its digit's next slot (rank among equal digits by lane), so the
//      pass is stable.
//
// A batch's pairs are sorted join by join with the same sort: the r of every
// pair of join j is shifted by the R rectangles of the joins before it, so
// that the joins' r ranges follow each other; one sort of the whole buffer
// then orders every join's pairs by (r, s) and keeps each join in its own
// range (the joins' pair counts do not change), and the shift is undone.
#define SJ_FILE_CODE 7
#include <algorithm>
#include <vector>

#include "sj_internal.h"

namespace sj {

constexpr int kPsWarps = 8;
constexpr int kPsThreads = kPsWarps * 32;
constexpr int kPsPerWarp = 1024;
constexpr int kPsTile = kPsWarps * kPsPerWarp;   // pairs per tile
constexpr int kPsChunk = kPsThreads * 8;         // scan elements per CTA

__device__ __forceinline__ unsigned pair_digit(int2 p, int pass) {
    const unsigned v = pass < 4 ? (unsigned)p.y : (unsigned)p.x;
    return (v >> (8 * (pass & 3))) & 0xffu;
}

__global__ void __launch_bounds__(kPsThreads) k_ps_hist(const int2 *__restrict__ in, unsigned n, int pass,
                                                        unsigned *__restrict__ hist, unsigned nT) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * kPsTile;
    for (int k = threadIdx.x; k < kPsTile; k += kPsThreads) {
        const size_t i = base + k;
        const bool ok = i < n;
        const unsigned d = ok ? pair_digit(in[i], pass) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[d], (unsigned)__popc(peers));
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nT + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of a uint32 array (sum below 2^32) in chunks of kPsChunk.
__device__ __forceinline__ unsigned cta_exclusive(unsigned v, unsigned *s_w, unsigned *total) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
        if ((int)lane >= d) inc += o;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned x = lane < kPsWarps ? s_w[lane] : 0u;
        unsigned xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(0xffffffffu, xi, d);
            if ((int)lane >= d) xi += o;
        }
        if (lane < kPsWarps) s_w[lane] = xi - x;
        if (lane == kPsWarps - 1) s_w[kPsWarps] = xi;
    }
    __syncthreads();
    *total = s_w[kPsWarps];
    return s_w[warp] + inc - v;
}

__global__ void __launch_bounds__(kPsThreads) k_ps_scan_part(const unsigned *__restrict__ a, size_t m,
                                                             unsigned *__restrict__ part) {
    __shared__ unsigned s_w[kPsWarps + 1];
    const size_t b = (size_t)blockIdx.x * kPsChunk + threadIdx.x * 8;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++)
        if (b + k < m) s += a[b + k];
    unsigned tot;
    cta_exclusive(s, s_w, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_ps_scan_top(unsigned *__restrict__ part, unsigned nc) {
    __shared__ unsigned sh[1024];
    const unsigned per = (nc + 1023) / 1024, i0 = threadIdx.x * per;
    unsigned s = 0;
    for (unsigned k = 0; k < per; k++)
        if (i0 + k < nc) s += part[i0 + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const unsigned x = threadIdx.x >= (unsigned)d ? sh[threadIdx.x - d] : 0u;
        __syncthreads();
        sh[threadIdx.x] += x;
        __syncthreads();
    }
    unsigned run = sh[threadIdx.x] - s;
    for (unsigned k = 0; k < per; k++)
        if (i0 + k < nc) {
            const unsigned v = part[i0 + k];
            part[i0 + k] = run;
            run += v;
        }
}

__global__ void __launch_bounds__(kPsThreads) k_ps_scan_fill(unsigned *__restrict__ a, size_t m,
                                                             const unsigned *__restrict__ part) {
    __shared__ unsigned s_w[kPsWarps + 1];
    const size_t b = (size_t)blockIdx.x * kPsChunk + threadIdx.x * 8;
    unsigned v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        v[k] = b + k < m ? a[b + k] : 0u;
        s += v[k];
    }
    unsigned tot;
    unsigned run = cta_exclusive(s, s_w, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 8; k++)
        if (b + k < m) {
            a[b + k] = run;
            run += v[k];
        }
}

__global__ void __launch_bounds__(kPsThreads) k_ps_scatter(const int2 *__restrict__ in, int2 *__restrict__ out,
                                                           unsigned n, int pass, const unsigned *__restrict__ off,
                                                           unsigned nT, Stats *st) {
    __shared__ unsigned wc[kPsWarps][256];
    for (int k = threadIdx.x; k < kPsWarps * 256; k += kPsThreads) (&wc[0][0])[k] = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const size_t start = (size_t)blockIdx.x * kPsTile + (size_t)warp * kPsPerWarp;
    unsigned *c = wc[warp];
    for (int b = 0; b < kPsPerWarp; b += 32) {   // digits of this warp's pairs
        const size_t i = start + b + lane;
        const bool ok = i < n;
        const unsigned d = ok ? pair_digit(in[i], pass) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && (int)lane == __ffs(peers) - 1) c[d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // per-warp starts of digit threadIdx.x
        const unsigned d = threadIdx.x;
        unsigned run = off[(size_t)d * nT + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kPsWarps; w++) {
            const unsigned t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int b = 0; b < kPsPerWarp; b += 32) {   // stable placement
        const size_t i = start + b + lane;
        const bool ok = i < n;
        const int2 p = ok ? in[i] : make_int2(0, 0);
        const unsigned d = ok ? pair_digit(p, pass) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned pos = 0;
        if (ok) pos = c[d] + __popc(peers & lt);
        __syncwarp();
        if (ok) {
            if (SJ_IN(st, pos, n)) out[pos] = p;
            if ((int)lane == __ffs(peers) - 1) c[d] += __popc(peers);
        }
        __syncwarp();
    }
}

// r of every pair of join j += sign * roff[j] (modulo 2^32), where j is the
// join whose range [joff[j], joff[j + 1]) holds the pair.
__global__ void __launch_bounds__(256) k_join_shift(int2 *__restrict__ pairs, unsigned long long n,
                                                    const unsigned long long *__restrict__ joff,
                                                    const unsigned long long *__restrict__ roff, int nj, int sign) {
    extern __shared__ unsigned long long s_off[];   // nj + 1 pair offsets
    for (int j = threadIdx.x; j <= nj; j += blockDim.x) s_off[j] = joff[j];
    __syncthreads();
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += 256ull * gridDim.x) {
        int lo = 0, hi = nj;   // last j with s_off[j] <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= i) lo = mid;
            else hi = mid;
        }
        const unsigned d = (unsigned)roff[lo];
        int2 p = pairs[i];
        p.x = (int)(sign > 0 ? (unsigned)p.x + d : (unsigned)p.x - d);
        pairs[i] = p;
    }
}

int sort_pairs_by_join(sj_ctx *ctx, Workspace &w, int2 *pairs, const int64_t *h_off, const int64_t *nR, int nj) {
    const unsigned long long n = (unsigned long long)h_off[nj];
    if (n < 2) return SJ_OK;
    std::vector<unsigned long long> tab(2 * (size_t)(nj + 1));
    unsigned long long r = 0;
    for (int j = 0; j <= nj; j++) {
        tab[j] = (unsigned long long)h_off[j];
        tab[nj + 1 + j] = r;
        if (j < nj) r += (unsigned long long)nR[j];
    }
    if (r >= (1ull << 32)) return fail(ctx, SJ_EINVAL, "sort_output of a batch needs fewer than 2^32 R rectangles");
    int st;
    if ((st = ensure(ctx, w.bSortOff, 8ull * tab.size()))) return st;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(w.bSortOff.p, tab.data(), 8ull * tab.size(), cudaMemcpyHostToDevice, ctx->stream)))
        return cuda_fail(ctx, e, "copy of the join offsets");
    const unsigned long long *joff = (const unsigned long long *)w.bSortOff.p, *roff = joff + nj + 1;
    const unsigned grid = (unsigned)std::min<unsigned long long>((n + 255) / 256, 4096ull);
    const size_t sm = 8ull * (nj + 1);
    k_join_shift<<<grid, 256, sm, ctx->stream>>>(pairs, n, joff, roff, nj, 1);
    if ((e = cudaGetLastError())) return cuda_fail(ctx, e, "join shift kernel");
    if ((st = sort_pairs(ctx, w, pairs, n))) return st;
    k_join_shift<<<grid, 256, sm, ctx->stream>>>(pairs, n, joff, roff, nj, -1);
    if ((e = cudaGetLastError())) return cuda_fail(ctx, e, "join shift kernel");
    // the host table must outlive the copy
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
    return SJ_OK;
}

int sort_pairs(sj_ctx *ctx, Workspace &w, int2 *pairs, unsigned long long n) {
    if (n < 2) return SJ_OK;
    if (n >= (1ull << 32)) return fail(ctx, SJ_EINVAL, "sort_output supports fewer than 2^32 pairs");
    const unsigned nT = (unsigned)((n + kPsTile - 1) / kPsTile);
    const size_t m = 256ull * nT;
    const unsigned nc = (unsigned)((m + kPsChunk - 1) / kPsChunk);
    int st;
    if ((st = ensure(ctx, w.sort_tmp, 8ull * n))) return st;
    if ((st = ensure(ctx, w.ps_hist, 4ull * m))) return st;
    if ((st = ensure(ctx, w.ps_part, 4ull * nc + 16))) return st;
    int2 *a = pairs, *b = (int2 *)w.sort_tmp.p;
    unsigned *hist = (unsigned *)w.ps_hist.p, *part = (unsigned *)w.ps_part.p;
    cudaStream_t s = ctx->stream;
    PhaseScope ph(ctx, PH_OTHER, 8 * 5);
    for (int pass = 0; pass < 8; pass++) {   // an even number: the result ends in `pairs`
        k_ps_hist<<<nT, kPsThreads, 0, s>>>(a, (unsigned)n, pass, hist, nT);
        k_ps_scan_part<<<nc, kPsThreads, 0, s>>>(hist, m, part);
        k_ps_scan_top<<<1, 1024, 0, s>>>(part, nc);
        k_ps_scan_fill<<<nc, kPsThreads, 0, s>>>(hist, m, part);
        k_ps_scatter<<<nT, kPsThreads, 0, s>>>(a, b, (unsigned)n, pass, hist, nT, (Stats *)w.stats.p);
        int2 *t = a;
        a = b;
        b = t;
    }
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(ctx, e, "pair sort kernels");
    return SJ_OK;
}

}  // namespace sj
