// distance.cu -- the eps-distance join on point sets (Sec. 1): every point
// becomes a square of side eps centred on it, the squares are joined by the
// intersection join of this library (the filter), and every intersecting
// pair is refined by its Euclidean distance.
//
//  1. squares of half-width h = eps * (1/2 + 2^-21) rounded up, corners
//     rounded outward (__fsub_rd / __fadd_ru), so each holds the exact square
//     of side eps.  An accepted pair has |dx|, |dy| <= eps * (1 + 2^-50)
//     (binary64 rounding of the test below), so its squares intersect: the
//     filter loses no pair.  As in the paper, the squares are built on the
//     fly: the two-level kernels read the points and form each square as
//     they load it (load_input).  Only when the data need the single-level
//     path (a tile beyond shared memory) does k_dist_squares write them out;
//  2. the join of the squares (any mode) writes the candidate pairs to the
//     workspace;
//  3. k_dist_mark: the distance test of every candidate.  The decision is
//     that of IEEE binary64 in one fixed order (dx, dy, dx*dx, dy*dy, their
//     sum, each rounded once: __dsub_rn / __dmul_rn / __dadd_rn, so no
//     contraction), accepted when d2 <= eps*eps.  Binary64 is slow on this
//     GPU, so a float32 evaluation of the same expression decides first
//     wherever its error bound settles the binary64 outcome (see
//     within_eps); one bit per candidate (warp ballot) and the accepted
//     count of every chunk of 2048 candidates;
//  4. k_scan_pairs: chunk offsets and the total;
//  5. k_dist_write: every chunk writes its accepted pairs at its offset, in
//     candidate order (prefix of the ballot words), into an output of the
//     exact size.
#define SJ_FILE_CODE 5
#include "sj_internal.h"

namespace sj {

constexpr int kDistThreads = 256;
constexpr int kDistPer = 8;                                   // candidates per thread
constexpr int kDistChunk = kDistThreads * kDistPer;           // candidates per CTA
constexpr int kDistWords = kDistChunk / 32;                   // ballot words per chunk

__global__ void __launch_bounds__(256) k_dist_squares(const float2 *__restrict__ P, long long n, float h,
                                                      float4 *__restrict__ out) {
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += 256ll * gridDim.x) {
        const float2 p = __ldg(P + i);
        out[i] = make_float4(__fsub_rd(p.x, h), __fsub_rd(p.y, h), __fadd_ru(p.x, h), __fadd_ru(p.y, h));
    }
}

// The binary64 decision d2 <= e2 (see above).  With u = 2^-24, the float32
// value d2f = (dx^2 + dy^2 in float32, three roundings after a rounded
// subtraction each) lies within a factor (1 +- 5u) of the exact d2, up to
// an absolute 2^-148 from underflow; e2f = float32(eps^2) within (1 +- u)
// of eps^2.  Hence d2f < e2f (1 - 2^-18) implies d2 < eps^2 (1 - 2^-19),
// where binary64 (relative error below 2^-50) must accept, and
// d2f > e2f (1 + 2^-18) implies d2 > eps^2 (1 + 2^-19), where it must
// reject.  The bounds need e2f >= 2^-100 (no underflow of eps^2, and 2^-148
// negligible against it); below that, and in the band between, binary64
// decides.  Overflow of d2f (far-apart points) is a reject, as in binary64.
__device__ __forceinline__ bool within_eps(float2 p, float2 q, double e2, float lo, float hi) {
    const float fx = __fsub_rn(p.x, q.x), fy = __fsub_rn(p.y, q.y);
    const float d2f = __fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy));
    if (d2f < lo) return true;
    if (d2f > hi) return false;
    const double dx = __dsub_rn((double)p.x, (double)q.x);
    const double dy = __dsub_rn((double)p.y, (double)q.y);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= e2;
}

// Chunk c = candidates [c * 2048, (c + 1) * 2048); candidate k = c * 2048 +
// u * 256 + threadIdx.x, so ballot word k / 32 = c * 64 + u * 8 + warp.
__global__ void __launch_bounds__(kDistThreads) k_dist_mark(const int2 *__restrict__ cand, long long C,
                                                            const float2 *__restrict__ P,
                                                            const float2 *__restrict__ Q, double e2, float lo,
                                                            float hi, unsigned *__restrict__ mask,
                                                            unsigned *__restrict__ cnt) {
    __shared__ unsigned s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kDistChunk + threadIdx.x;
    int2 c[kDistPer];
#pragma unroll
    for (int u = 0; u < kDistPer; u++) {
        const long long k = base + u * kDistThreads;
        c[u] = k < C ? __ldg(cand + k) : make_int2(-1, -1);
    }
    float2 p[kDistPer], q[kDistPer];
#pragma unroll
    for (int u = 0; u < kDistPer; u++) {
        if (c[u].x >= 0) {
            p[u] = __ldg(P + c[u].x);
            q[u] = __ldg(Q + c[u].y);
        }
    }
    unsigned mine = 0;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < kDistPer; u++) {
        const bool ok = c[u].x >= 0 && within_eps(p[u], q[u], e2, lo, hi);
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) {
            mask[(size_t)blockIdx.x * kDistWords + u * (kDistThreads / 32) + warp] = b;
            mine += __popc(b);
        }
    }
    if (lane == 0 && mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = s_cnt;
}

__global__ void __launch_bounds__(kDistThreads) k_dist_write(const int2 *__restrict__ cand, long long C,
                                                             const unsigned *__restrict__ mask,
                                                             const unsigned long long *__restrict__ off,
                                                             int2 *__restrict__ out, Stats *st,
                                                             unsigned long long cap) {
    __shared__ unsigned s_pre[kDistWords];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned *m = mask + (size_t)blockIdx.x * kDistWords;
    if (warp == 0) {   // exclusive prefix of the popcounts of the chunk's 64 words
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
    const unsigned long long o = off[blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kDistChunk + threadIdx.x;
#pragma unroll
    for (int u = 0; u < kDistPer; u++) {
        const int w = u * (kDistThreads / 32) + warp;
        const unsigned b = m[w];
        const long long k = base + u * kDistThreads;
        const unsigned long long d = o + s_pre[w] + __popc(b & lt);
        if (((b >> lane) & 1u) && k < C && SJ_IN(st, d, cap)) out[d] = cand[k];
    }
}

}  // namespace sj

using namespace sj;

static int dist_check(sj_ctx *ctx, const sj_point *P, int64_t nP, const sj_point *Q, int64_t nQ, float eps) {
    if (!ctx) return SJ_EINVAL;
    if (nP < 0 || nQ < 0 || nP >= SJ_MAX_N || nQ >= SJ_MAX_N)
        return fail(ctx, SJ_EINVAL, "sizes must satisfy 0 <= n < 2^30");
    if ((nP && !P) || (nQ && !Q)) return fail(ctx, SJ_EINVAL, "null point pointer");
    if ((reinterpret_cast<uintptr_t>(P) & 7) || (reinterpret_cast<uintptr_t>(Q) & 7))
        return fail(ctx, SJ_EINVAL, "points must be 8-byte aligned");
    if (!(eps >= 0.0f) || !(eps <= 1e18f)) return fail(ctx, SJ_EINVAL, "eps must lie in [0, 1e18]");
    return SJ_OK;
}

// Half-width of the squares: eps * (1/2 + 2^-21) rounded up to float32 (the
// product of two floats is exact in double, so the comparison is exact).
static float square_half_width(float eps) {
    const float m = 0.5f + 0x1p-21f;
    float h = eps * m;
    if ((double)h < (double)eps * (double)m) h = nextafterf(h, INFINITY);
    return h;
}

// Thresholds of the float32 pre-test of within_eps: d2f below lo accepts,
// above hi rejects; lo = -1, hi = +inf send every candidate to binary64.
static void prefilter_bounds(float eps, float *lo, float *hi) {
    const float e2f = eps * eps;
    if (!(e2f >= 0x1p-100f)) {
        *lo = -1.0f;
        *hi = INFINITY;
        return;
    }
    *lo = e2f * (1.0f - 0x1p-18f);
    *hi = e2f * (1.0f + 0x1p-18f);
}

// Keeps the workspace's point-input mode for the duration of one join.
struct PointInputs {
    Workspace &w;
    PointInputs(Workspace &ws, float h) : w(ws) {
        w.in_pts = 1;
        w.in_h = h;
    }
    ~PointInputs() {
        w.in_pts = 0;
        w.in_h = 0.0f;
    }
};

// Squares, candidate join, refinement into os.
static int dist_core(sj_ctx *ctx, const sj_point *d_P, int64_t nP, const sj_point *d_Q, int64_t nQ, float eps,
                     const sj_grid *g, const sj_opts *o, OutSpec &os, int64_t *npairs, int64_t *ncand) {
    Workspace &w = ctx->ws;
    int st;
    GridDev gd;
    if ((st = check_inputs(ctx, nullptr, 0, nullptr, 0, g, &gd))) return st;   // the grid alone
    const float h = square_half_width(eps);
    // the candidates need no order: only the refined pairs are sorted (sort_output)
    sj_opts oc{};
    if (o) {
        oc = *o;
        oc.sort_output = 0;
    }
    const sj_opts *po = o ? &oc : nullptr;
    OutSpec cs{OutSpec::WS};
    int64_t C = 0;
    {   // squares on the fly (two-level path)
        PointInputs in(w, h);
        st = join_core(ctx, w, (const sj_rect *)d_P, nP, (const sj_rect *)d_Q, nQ, gd, po, cs, &C);
    }
    cudaError_t e;
    if (st == PTS_UNSUITED) {   // the single-level path: write the squares out
        if ((st = ensure(ctx, w.dsq_r, 16ull * nP + 16))) return st;
        if ((st = ensure(ctx, w.dsq_s, 16ull * nQ + 16))) return st;
        {
            PhaseScope ph(ctx, PH_OTHER, (nP > 0) + (nQ > 0));
            const int grid = ctx->num_sms * 8;
            if (nP) k_dist_squares<<<grid, 256, 0, ctx->stream>>>((const float2 *)d_P, nP, h, (float4 *)w.dsq_r.p);
            if (nQ) k_dist_squares<<<grid, 256, 0, ctx->stream>>>((const float2 *)d_Q, nQ, h, (float4 *)w.dsq_s.p);
            if ((e = cudaGetLastError())) return cuda_fail(ctx, e, "square kernel");
        }
        cs = OutSpec{OutSpec::WS};
        st = join_core(ctx, w, (const sj_rect *)w.dsq_r.p, nP, (const sj_rect *)w.dsq_s.p, nQ, gd, po, cs, &C);
    }
    if (st) return st;
    if (ncand) *ncand = C;
    *npairs = 0;
    if (C == 0) {
        ctx->last.npairs = 0;
        return out_acquire(ctx, w, os, 0);
    }
    const int2 *cand = cs.got;
    const long long nch = (C + kDistChunk - 1) / kDistChunk;
    if ((st = ensure(ctx, w.dmask, 4ull * kDistWords * nch))) return st;
    if ((st = ensure(ctx, w.dcnt, 4ull * nch + 16))) return st;
    if ((st = ensure(ctx, w.doff, 8ull * nch + 16))) return st;
    if ((st = ensure(ctx, w.dstats, sizeof(Stats)))) return st;
    Stats *dst = (Stats *)w.dstats.p;
    const double e2 = (double)eps * (double)eps;   // one rounded product
    float lo, hi;
    prefilter_bounds(eps, &lo, &hi);
    {
        PhaseScope ph(ctx, PH_REFINE, 2);
        k_dist_mark<<<(unsigned)nch, kDistThreads, 0, ctx->stream>>>(cand, C, (const float2 *)d_P,
                                                                   (const float2 *)d_Q, e2, lo, hi,
                                                                   (unsigned *)w.dmask.p, (unsigned *)w.dcnt.p);
        if ((e = launch_scan_pairs((const unsigned *)w.dcnt.p, (unsigned)nch, (unsigned long long *)w.doff.p,
                                   dst, ctx->stream)))
            return cuda_fail(ctx, e, "refinement kernels");
    }
    Stats *hs = (Stats *)ctx->h_stats;
    if ((e = copy_async(ctx, &hs->npairs, &dst->npairs, sizeof(unsigned long long))))
        return cuda_fail(ctx, e, "copy of the refined count");
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
    const unsigned long long P = hs->npairs;
    *npairs = (int64_t)P;
    ctx->last.npairs = (int64_t)P;
    if ((st = out_acquire(ctx, w, os, P))) return st;
    if (P == 0) return SJ_OK;
    {
        PhaseScope ph(ctx, PH_REFINE, 1);
        k_dist_write<<<(unsigned)nch, kDistThreads, 0, ctx->stream>>>(
            cand, C, (const unsigned *)w.dmask.p, (const unsigned long long *)w.doff.p, os.got, (Stats *)w.stats.p,
            P);
        if ((e = cudaGetLastError())) {
            out_abandon(ctx, os);
            return cuda_fail(ctx, e, "refinement write kernel");
        }
    }
    if (o && o->sort_output && (st = sort_pairs(ctx, w, os.got, P))) {
        out_abandon(ctx, os);
        return st;
    }
    if ((st = check_tail(ctx, w))) out_abandon(ctx, os);
    return st;
}

extern "C" int sj_distance_join(sj_ctx *ctx, const sj_point *d_P, int64_t nP, const sj_point *d_Q, int64_t nQ,
                                float eps, const sj_grid *g, const sj_opts *o, sj_pair **d_pairs,
                                int64_t *npairs, int64_t *ncand) {
    int st = dist_check(ctx, d_P, nP, d_Q, nQ, eps);
    if (st) return st;
    if ((st = check_opts(ctx, o))) return st;
    if (!d_pairs || !npairs) return fail(ctx, SJ_EINVAL, "null output pointer");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    *d_pairs = nullptr;
    OutSpec os{OutSpec::LIB};
    if ((st = dist_core(ctx, d_P, nP, d_Q, nQ, eps, g, o, os, npairs, ncand))) return st;
    *d_pairs = (sj_pair *)os.got;
    return SJ_OK;
}

extern "C" int sj_distance_join_into(sj_ctx *ctx, const sj_point *d_P, int64_t nP, const sj_point *d_Q,
                                     int64_t nQ, float eps, const sj_grid *g, const sj_opts *o, sj_pair *d_buf,
                                     int64_t cap, int64_t *npairs, int64_t *ncand) {
    int st = dist_check(ctx, d_P, nP, d_Q, nQ, eps);
    if (st) return st;
    if ((st = check_opts(ctx, o))) return st;
    if (cap < 0 || !npairs) return fail(ctx, SJ_EINVAL, "negative capacity or null npairs");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    OutSpec os{OutSpec::INTO};
    os.into = d_buf;
    os.cap = cap;
    return dist_core(ctx, d_P, nP, d_Q, nQ, eps, g, o, os, npairs, ncand);
}
