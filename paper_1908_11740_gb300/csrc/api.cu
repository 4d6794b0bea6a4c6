// api.cu -- the C ABI of include/sj.h: contexts, the allocator, a grow-only
// device workspace, and the host orchestration of the kernels of the
// partitioning-based spatial join (PBSM) filter step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "../../include/sj.h"
#include "sj_common.cuh"
#include "sj_internal.h"
#include "sj_learned.h"
#include "sj_kernels.h"

using namespace sj;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
extern "C" const char *sj_strerror(int status) {
    switch (status) {
        case SJ_OK: return "ok";
        case SJ_EINVAL: return "invalid argument or input";
        case SJ_ENOMEM: return "out of device memory";
        case SJ_EOVERFLOW: return "output buffer too small";
        case SJ_ETIMEOUT: return "device-side wait timed out";
        case SJ_ECUDA: return "CUDA runtime error";
        case SJ_EINTERNAL: return "internal error";
        default: return "unknown status";
    }
}

int sj::fail(sj_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->msg, sizeof(ctx->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

int sj::cuda_fail(sj_ctx *ctx, cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(ctx, SJ_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(ctx, SJ_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

extern "C" const char *sj_last_error(sj_ctx *ctx) { return ctx ? ctx->msg : "no context"; }

// ---------------------------------------------------------------------------
// allocation
// ---------------------------------------------------------------------------
void *sj::dev_alloc(sj_ctx *ctx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (ctx->alloc) return ctx->alloc(bytes, ctx->user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void sj::dev_free(sj_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->alloc) {
        if (ctx->free_fn) ctx->free_fn(p, ctx->user);
        return;
    }
    cudaFreeAsync(p, ctx->stream);
}

// Grow `b` to hold at least `bytes` (contents are not kept).
int sj::ensure(sj_ctx *ctx, Buf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return SJ_OK;
    dev_free(ctx, b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 8 + 256;
    want = (want + 255) & ~(size_t)255;
    void *p = dev_alloc(ctx, want);
    if (!p) return fail(ctx, SJ_ENOMEM, "device allocation of %zu bytes failed", want);
    b.p = p;
    b.bytes = want;
    return SJ_OK;
}

void sj::release(sj_ctx *ctx, Workspace &w) {
    Buf *all[] = {&w.stats, &w.cnt, &w.off, &w.bsum, &w.ts, &w.large, &w.ent_r, &w.id_r,
                  &w.ent_s, &w.id_s, &w.seg_off, &w.seg_src, &w.seg_vb, &w.hist, &w.key_a,
                  &w.key_b, &w.val_a, &w.val_b, &w.lmbr, &w.lid, &w.pc, &w.poff, &w.resv,
                  &w.fail_c, &w.fail_l, &w.sort_tmp, &w.ps_hist, &w.ps_part, &w.in_r, &w.in_s, &w.out, &w.bH,
                  &w.bTot, &w.bBoR, &w.bBoS, &w.bItems, &w.bEntR, &w.bEntS, &w.bPc, &w.bPoff,
                  &w.bResv, &w.bFail, &w.bImeta, &w.bIns, &w.bFeatRaw, &w.bFeat, &w.bPred,
                  &w.bOrder, &w.bCapTot, &w.bCur, &w.bList, &w.bSpill, &w.bJd, &w.bIjoin, &w.bJfirst, &w.bJoff, &w.bScanPart, &w.bSortOff,
                  &w.lstart, &w.lcoff, &w.lvb, &w.ly, &w.st_order, &w.dsq_r, &w.dsq_s, &w.dmask, &w.dcnt, &w.doff, &w.dstats,
                  &w.band_r, &w.band_s, &w.band_ir, &w.band_is, &w.tpairs, &w.item_of, &w.cnt64};
    for (Buf *b : all) {
        dev_free(ctx, b->p);
        b->p = nullptr;
        b->bytes = 0;
    }
    w.cap_r = w.cap_s = 0;
    w.bcap_r = w.bcap_s = 0;
}

// ---------------------------------------------------------------------------
// device-side timing
// ---------------------------------------------------------------------------
static const char *kPhaseNames[PH_N] = {"reset",        "count",       "scan",
                                        "scatter",      "large_sort",  "sweep_count",
                                        "pair_scan",    "sweep_write", "large_sweep_count",
                                        "large_sweep_write", "model",  "other",
                                        "refine"};

static cudaEvent_t take_event(Timer &t) {
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

sj::PhaseScope::PhaseScope(sj_ctx *c, int ph, int kernels) : ctx(c), phase(ph) {
    ctx->launches += kernels;
    if (ctx->timer.on) {
        a = take_event(ctx->timer);
        if (a) cudaEventRecord(a, ctx->stream);
    }
}

sj::PhaseScope::~PhaseScope() {
    if (!a) return;
    cudaEvent_t b = take_event(ctx->timer);
    if (!b) return;
    cudaEventRecord(b, ctx->stream);
    ctx->timer.pending.push_back({phase, a, b});
}

static void timing_resolve(sj_ctx *ctx) {
    Timer &t = ctx->timer;
    if (t.pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &r : t.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            t.ms[r.phase] += ms;
            t.n[r.phase] += 1;
        } else {
            cudaGetLastError();
        }
        t.pool.push_back(r.a);
        t.pool.push_back(r.b);
    }
    t.pending.clear();
}

extern "C" int sj_timing_enable(sj_ctx *ctx, int on) {
    if (!ctx) return SJ_EINVAL;
    DeviceGuard g(ctx->device);
    timing_resolve(ctx);
    ctx->timer.on = on != 0;
    for (int i = 0; i < PH_N; i++) {
        ctx->timer.ms[i] = 0;
        ctx->timer.n[i] = 0;
    }
    ctx->launches = 0;
    return SJ_OK;
}

extern "C" int sj_timing_read(sj_ctx *ctx, sj_timing *out) {
    if (!ctx || !out) return SJ_EINVAL;
    DeviceGuard g(ctx->device);
    timing_resolve(ctx);
    memset(out, 0, sizeof *out);
    out->launches = ctx->launches;
    for (int i = 0; i < PH_N && i < SJ_NPHASE; i++) {
        out->ms[i] = ctx->timer.ms[i];
        out->n[i] = ctx->timer.n[i];
        ctx->timer.ms[i] = 0;
        ctx->timer.n[i] = 0;
    }
    ctx->launches = 0;
    return SJ_OK;
}

extern "C" int sj_last_stats(sj_ctx *ctx, sj_stats *out) {
    if (!ctx || !out) return SJ_EINVAL;
    *out = ctx->last;
    return SJ_OK;
}

extern "C" const char *sj_timing_phase_name(int phase) {
    return (phase >= 0 && phase < PH_N) ? kPhaseNames[phase] : "";
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int sj_create(sj_ctx **out, int device, void *cuda_stream) {
    if (!out) return SJ_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SJ_EINVAL;
    }
    sj_ctx *c = new (std::nothrow) sj_ctx();
    if (!c) return SJ_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return SJ_ECUDA;
    }
    if (sweep_setup() != cudaSuccess) {
        delete c;
        return SJ_ECUDA;
    }
    c->sweep_bps = sweep_blocks_per_sm();
    if (blocked_setup() != cudaSuccess || stripe_setup() != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SJ_ECUDA;
    }
    c->bjoin_bps = bjoin_blocks_per_sm();
    {
        const char *e = getenv("SJ_L1_WRITE");   // "private": per-CTA write ranges (tuning / comparison)
        if (e && strcmp(e, "private") == 0) c->shared_cursors = 0;
        const char *t = getenv("SJ_BLOCK_TARGET");   // entries per block of the two-level plan
        if (t && atoi(t) >= 64) c->block_target = atoi(t);
        const char *st = getenv("SJ_STRIPES");   // "0": 1D grids take the general path (comparison)
        if (st && strcmp(st, "0") == 0) c->use_stripes = 0;
        const char *bg = getenv("SJ_BATCH_GRAPHS");   // "0": batches launch directly (phase timing)
        if (bg && strcmp(bg, "0") == 0) c->batch_graphs = 0;
        const char *bc = getenv("SJ_BATCH_COUNT");   // "global": per-rectangle global atomics (comparison)
        if (bc && strcmp(bc, "global") == 0) c->batch_count_local = 0;
    }
    if (cudaMallocHost(&c->h_stats, sizeof(Stats)) != cudaSuccess ||
        cudaMallocHost(&c->h_aux, 64) != cudaSuccess ||
        cudaMallocHost(&c->h_jd, sizeof(JoinDesc) * kMaxJoins) != cudaSuccess ||
        cudaMallocHost(&c->h_joff, 8ull * (kMaxJoins + 1)) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->h_stats) cudaFreeHost(c->h_stats);
        if (c->h_aux) cudaFreeHost(c->h_aux);
        if (c->h_jd) cudaFreeHost(c->h_jd);
        if (c->h_joff) cudaFreeHost(c->h_joff);
        delete c;
        return SJ_ENOMEM;
    }
    c->msg[0] = 0;
    *out = c;
    return SJ_OK;
}

extern "C" int sj_destroy(sj_ctx *ctx) {
    if (!ctx) return SJ_EINVAL;
    DeviceGuard g(ctx->device);
    batch_release(ctx);
    hoststream_release(ctx);
    release(ctx, ctx->ws);
    mlp_release(ctx);
    cudaStreamSynchronize(ctx->stream);
    timing_resolve(ctx);
    for (cudaEvent_t e : ctx->timer.pool) cudaEventDestroy(e);
    cudaFreeHost(ctx->h_stats);
    cudaFreeHost(ctx->h_aux);
    cudaFreeHost(ctx->h_jd);
    cudaFreeHost(ctx->h_joff);
    cudaEventDestroy(ctx->ev_aux);
    delete ctx;
    return SJ_OK;
}

extern "C" int sj_set_allocator(sj_ctx *ctx, sj_alloc_fn alloc, sj_free_fn free_fn, void *user) {
    if (!ctx) return SJ_EINVAL;
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(ctx, SJ_EINVAL, "allocator needs both alloc and free (or neither)");
    DeviceGuard g(ctx->device);
    batch_release(ctx);   // cached graphs point into the workspace
    hoststream_release(ctx);
    release(ctx, ctx->ws);
    mlp_release(ctx);
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    return SJ_OK;
}

extern "C" void sj_free(sj_ctx *ctx, void *d_ptr) {
    if (!ctx || !d_ptr) return;
    DeviceGuard g(ctx->device);
    dev_free(ctx, d_ptr);
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
int sj::check_inputs(sj_ctx *ctx, const sj_rect *R, int64_t nR, const sj_rect *S, int64_t nS,
                     const sj_grid *g, GridDev *gd) {
    if (!ctx) return SJ_EINVAL;
    if (nR < 0 || nS < 0 || nR >= SJ_MAX_N || nS >= SJ_MAX_N)
        return fail(ctx, SJ_EINVAL, "sizes must satisfy 0 <= n < 2^30 (got %lld, %lld)",
                    (long long)nR, (long long)nS);
    if ((nR && !R) || (nS && !S)) return fail(ctx, SJ_EINVAL, "null rectangle pointer");
    if (((uintptr_t)R & 15) || ((uintptr_t)S & 15))
        return fail(ctx, SJ_EINVAL, "rectangle arrays must be 16-byte aligned");
    if (!g) return fail(ctx, SJ_EINVAL, "null grid");
    if (g->nx < 1 || g->ny < 1 || g->nx > (1 << 24) || g->ny > (1 << 24) ||
        (int64_t)g->nx * g->ny > SJ_MAX_TILES)
        return fail(ctx, SJ_EINVAL, "grid %d x %d out of range", g->nx, g->ny);
    if (!isfinite(g->x0) || !isfinite(g->x1) || !isfinite(g->y0) || !isfinite(g->y1) ||
        !(g->x1 > g->x0) || !(g->y1 > g->y0))
        return fail(ctx, SJ_EINVAL, "grid extent must be finite with x1 > x0, y1 > y0");
    volatile float wx = g->x1 - g->x0, wy = g->y1 - g->y0;
    volatile float gx = (float)g->nx / wx, gy = (float)g->ny / wy;
    if (!isfinite(gx) || !isfinite(gy) || !(gx > 0.0f) || !(gy > 0.0f))
        return fail(ctx, SJ_EINVAL, "grid resolution overflows float32");
    gd->nx = g->nx;
    gd->ny = g->ny;
    gd->x0 = g->x0;
    gd->y0 = g->y0;
    gd->gx = gx;
    gd->gy = gy;
    return SJ_OK;
}

// ---------------------------------------------------------------------------
// the pipeline
// ---------------------------------------------------------------------------
// Size every workspace buffer for T tiles and the current entry capacities.
int sj::size_workspace(sj_ctx *ctx, Workspace &w, long long T) {
    int st;
    const unsigned long long ecap = w.cap_r + w.cap_s;
    w.T = T;
    w.nch_cap = (unsigned)((ecap + T) / kChunk + 2);
    w.nl_cap = (unsigned)((ecap + T) / (kChunk + 1) + 1);
    w.items_cap = ecap;
    w.vb_cap = (unsigned)(ecap / kRadixBlock + 2ull * w.nl_cap + 1);
    const unsigned long long nslots = (unsigned long long)w.nch_cap + w.vb_cap;
    if ((st = ensure(ctx, w.stats, sizeof(Stats)))) return st;
    if ((st = ensure(ctx, w.cnt, 8ull * T))) return st;
    if ((st = ensure(ctx, w.off, 8ull * (T + 1)))) return st;
    if ((st = ensure(ctx, w.bsum, 16ull * (scan_blocks(T) + 1)))) return st;
    if ((st = ensure(ctx, w.ts, 4ull * (w.nch_cap + 1)))) return st;
    if ((st = ensure(ctx, w.large, 4ull * (w.nl_cap + 1)))) return st;
    if ((st = ensure(ctx, w.ent_r, 16ull * (w.cap_r + 1)))) return st;
    if ((st = ensure(ctx, w.id_r, 4ull * (w.cap_r + 1)))) return st;
    if ((st = ensure(ctx, w.ent_s, 16ull * (w.cap_s + 1)))) return st;
    if ((st = ensure(ctx, w.id_s, 4ull * (w.cap_s + 1)))) return st;
    if ((st = ensure(ctx, w.seg_off, 4ull * (2ull * w.nl_cap + 2)))) return st;
    if ((st = ensure(ctx, w.seg_src, 4ull * (2ull * w.nl_cap + 2)))) return st;
    if ((st = ensure(ctx, w.seg_vb, 4ull * (2ull * w.nl_cap + 2)))) return st;
    if ((st = ensure(ctx, w.hist, 1024ull * (w.vb_cap + 1)))) return st;
    if ((st = ensure(ctx, w.key_a, 4ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.key_b, 4ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.val_a, 4ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.val_b, 4ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.lmbr, 16ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.lid, 4ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.lstart, 4ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.lcoff, 8ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.ly, 8ull * (w.items_cap + 1)))) return st;
    if ((st = ensure(ctx, w.lvb, 32ull * (w.vb_cap + 2)))) return st;
    if ((st = ensure(ctx, w.pc, 4ull * nslots))) return st;
    if ((st = ensure(ctx, w.poff, 8ull * nslots))) return st;
    if ((st = ensure(ctx, w.resv, 8ull * nslots))) return st;
    if ((st = ensure(ctx, w.fail_c, 4ull * (w.nch_cap + 1)))) return st;
    if ((st = ensure(ctx, w.fail_l, 4ull * (w.vb_cap + 1)))) return st;
    return SJ_OK;
}

LargeArgs sj::large_args(Workspace &w) {
    LargeArgs a;
    memset(&a, 0, sizeof a);
    a.off = (const uint2 *)w.off.p;
    a.large = (const unsigned *)w.large.p;
    a.ent_r = (const float4 *)w.ent_r.p;
    a.id_r = (const unsigned *)w.id_r.p;
    a.ent_s = (const float4 *)w.ent_s.p;
    a.id_s = (const unsigned *)w.id_s.p;
    a.seg_off = (unsigned *)w.seg_off.p;
    a.seg_src = (unsigned *)w.seg_src.p;
    a.seg_vb = (unsigned *)w.seg_vb.p;
    a.hist = (unsigned *)w.hist.p;
    a.key_in = (unsigned *)w.key_a.p;
    a.val_in = (unsigned *)w.val_a.p;
    a.key_out = (unsigned *)w.key_b.p;
    a.val_out = (unsigned *)w.val_b.p;
    a.lmbr = (float4 *)w.lmbr.p;
    a.lid = (unsigned *)w.lid.p;
    a.items_cap = w.items_cap;
    a.vb_cap = w.vb_cap;
    if (w.lcoff.p && w.lstart.p && w.lvb.p && w.ly.p) {
        a.lstart = (unsigned *)w.lstart.p;
        a.ly = (float2 *)w.ly.p;
        a.lcoff = (unsigned long long *)w.lcoff.p;
        unsigned long long *v = (unsigned long long *)w.lvb.p;
        const size_t n = (size_t)w.vb_cap + 2;
        a.vbc = v;
        a.vbpairs = v + n;
        a.vbcur = v + 2 * n;
        a.vbch = (unsigned *)(v + 3 * n);
    }
    a.st = (Stats *)w.stats.p;
    return a;
}

SweepArgs sj::sweep_args(Workspace &w) {
    SweepArgs a;
    memset(&a, 0, sizeof a);
    a.off = (const uint2 *)w.off.p;
    a.ts = (const unsigned *)w.ts.p;
    a.ent_r = (const float4 *)w.ent_r.p;
    a.id_r = (const unsigned *)w.id_r.p;
    a.ent_s = (const float4 *)w.ent_s.p;
    a.id_s = (const unsigned *)w.id_s.p;
    a.st = (Stats *)w.stats.p;
    a.cnt_out = (unsigned *)w.pc.p;
    a.off_in = (const unsigned long long *)w.poff.p;
    a.resv = (unsigned long long *)w.resv.p;
    a.cnt_base = w.nch_cap;
    return a;
}

// Partitioning (count, scan, scatter) and the sort of the large tiles.
// Enqueued only; errors of the device show up in the stats.
int sj::enqueue_partition(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S,
                          long long nS, const GridDev &g) {
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    Stats *st = (Stats *)w.stats.p;
    {
        PhaseScope ph(ctx, PH_RESET, 0);
        if ((e = zero_async(ctx, w.stats.p, sizeof(Stats)))) return cuda_fail(ctx, e, "memset");
        if ((e = zero_async(ctx, w.cnt.p, 8ull * w.T))) return cuda_fail(ctx, e, "memset");
    }
    const int grid_stream = ctx->num_sms * 8;
    const bool any = nR + nS > 0;
    {
        PhaseScope ph(ctx, PH_COUNT, any ? 1 : 0);
        if ((e = launch_count(R, nR, S, nS, g, (unsigned *)w.cnt.p, st, grid_stream, s)))
            return cuda_fail(ctx, e, "count kernel");
    }
    {
        PhaseScope ph(ctx, PH_SCAN, 3);
        if ((e = launch_scan((const uint2 *)w.cnt.p, w.T, (unsigned long long *)w.bsum.p, (uint2 *)w.off.p,
                             (unsigned *)w.ts.p, w.nch_cap + 1, (unsigned *)w.large.p, w.nl_cap, st, s)))
            return cuda_fail(ctx, e, "scan kernels");
    }
    {
        PhaseScope ph(ctx, PH_SCATTER, any ? 1 : 0);
        if ((e = launch_scatter(R, nR, S, nS, g, (unsigned *)w.cnt.p, (const uint2 *)w.off.p,
                                (float4 *)w.ent_r.p, (unsigned *)w.id_r.p, w.cap_r, (float4 *)w.ent_s.p,
                                (unsigned *)w.id_s.p, w.cap_s, st, grid_stream, s)))
            return cuda_fail(ctx, e, "scatter kernel");
    }
    {
        PhaseScope ph(ctx, PH_LSORT, 14);
        if ((e = launch_large_sort(large_args(w), ctx->num_sms * 4, s)))
            return cuda_fail(ctx, e, "large-tile sort");
    }
    return SJ_OK;
}

// Sweep both paths in `mode`; for MODE_WRITE the offsets come from `off_in`.
int sj::enqueue_sweep(sj_ctx *ctx, Workspace &w, int mode, int2 *out, unsigned long long cap,
                      const unsigned long long *off_in, unsigned *tile_pairs, int slot_base) {
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    SweepArgs a = sweep_args(w);
    a.out = out;
    a.cap = cap;
    a.tile_pairs = tile_pairs;
    if (off_in) a.off_in = off_in;
    a.fail = (unsigned *)w.fail_c.p;
    a.nfail = &((Stats *)w.stats.p)->nfail;
    a.work_slot = slot_base;
    {
        PhaseScope ph(ctx, mode == MODE_WRITE || mode == MODE_RESERVE ? PH_SWEEP_WRITE : PH_SWEEP_COUNT, 1);
        if ((e = launch_sweep_chunks(mode, a, ctx->num_sms * ctx->sweep_bps, s)))
            return cuda_fail(ctx, e, "sweep kernel");
    }
    SweepArgs b = a;
    b.fail = (unsigned *)w.fail_l.p;
    b.nfail = &((Stats *)w.stats.p)->nfail_large;
    b.work_slot = slot_base + 1;
    {
        PhaseScope ph(ctx, mode == MODE_WRITE || mode == MODE_RESERVE ? PH_LSWEEP_WRITE : PH_LSWEEP_COUNT,
                      w.lcoff.p && mode != MODE_RESERVE ? (mode == MODE_COUNT ? 4 : 3) : 1);
        if ((e = launch_sweep_large(mode, large_args(w), b, ctx->num_sms * 4, s)))
            return cuda_fail(ctx, e, "large-tile sweep kernel");
    }
    return SJ_OK;
}

// Debug build: SJ_EINTERNAL naming the site of the first failed bounds check.
int sj::check_failed(sj_ctx *ctx, unsigned site) {
    static const char *const files[] = {"?",          "blocked.cu",   "sweep.cu",   "partition.cu",
                                        "stripes.cu", "distance.cu",  "bands.cu",   "sortpairs.cu",
                                        "learned.cu", "noalloc.cu"};
    const unsigned f = site >> 16;
    return fail(ctx, SJ_EINTERNAL, "bounds check failed at %s:%u",
                f < sizeof files / sizeof files[0] ? files[f] : "?", site & 0xffffu);
}

int sj::read_stats(sj_ctx *ctx, Workspace &w, Stats *out) {
    cudaError_t e;
    if ((e = copy_async(ctx, ctx->h_stats, w.stats.p, sizeof(Stats))))
        return cuda_fail(ctx, e, "stats copy");
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
    memcpy(out, ctx->h_stats, sizeof(Stats));
#if SJ_CHECK
    if (out->err & kErrCheck) return check_failed(ctx, out->check);
#endif
    return SJ_OK;
}

// Debug build: after a call's last kernel, read the counters once more so
// that a check failed after the last read is reported (no-op otherwise).
int sj::check_tail(sj_ctx *ctx, Workspace &w) {
#if SJ_CHECK
    Stats s;
    return read_stats(ctx, w, &s);
#else
    (void)ctx;
    (void)w;
    return SJ_OK;
#endif
}

// Partition + count pass with capacity retry.  On return the workspace
// holds the partition, pc/poff the per-item pair counts / offsets, *stats
// the device counters (npairs = exact total).
int sj::partition_and_count(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR,
                            const float4 *S, long long nS, const GridDev &g, Stats *stats,
                            bool count_pass) {
    const long long T = (long long)g.nx * g.ny;
    w.cap_r = std::max<unsigned long long>(w.cap_r, (unsigned long long)nR + nR / 4 + 1024);
    w.cap_s = std::max<unsigned long long>(w.cap_s, (unsigned long long)nS + nS / 4 + 1024);
    for (int attempt = 0; attempt < 3; attempt++) {
        int st;
        if ((st = size_workspace(ctx, w, T))) return st;
        if ((st = enqueue_partition(ctx, w, R, nR, S, nS, g))) return st;
        if (count_pass) {
            cudaError_t e;
            const unsigned nslots = w.nch_cap + w.vb_cap;
            if ((e = zero_async(ctx, w.pc.p, 4ull * nslots)))
                return cuda_fail(ctx, e, "memset");
            if ((st = enqueue_sweep(ctx, w, MODE_COUNT, nullptr, 0, nullptr, nullptr, 0))) return st;
            PhaseScope ph(ctx, PH_PAIRSCAN, 1);
            if ((e = launch_scan_pairs((const unsigned *)w.pc.p, nslots, (unsigned long long *)w.poff.p,
                                       (Stats *)w.stats.p, ctx->stream)))
                return cuda_fail(ctx, e, "pair-count scan");
        }
        if ((st = read_stats(ctx, w, stats))) return st;
        if (stats->err & kErrBadRect)
            return fail(ctx, SJ_EINVAL, "invalid rectangle: NaN/Inf coordinate or xl > xu / yl > yu");
        if (stats->err & kErrTooMany)
            return fail(ctx, SJ_EINVAL, "more than 2^31 replicated entries on one side");
        if (stats->err & (kErrEntCap | kErrChunkCap | kErrLargeCap)) {
            w.cap_r = std::max<unsigned long long>(w.cap_r, stats->e_r + stats->e_r / 8 + 1024);
            w.cap_s = std::max<unsigned long long>(w.cap_s, stats->e_s + stats->e_s / 8 + 1024);
            continue;   // grow and redo
        }
        if (stats->err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats->err);
        memset(&ctx->last, 0, sizeof ctx->last);
        ctx->last.entries_r = (int64_t)stats->e_r;
        ctx->last.entries_s = (int64_t)stats->e_s;
        ctx->last.npairs = (int64_t)stats->npairs;
        return SJ_OK;
    }
    return fail(ctx, SJ_EINTERNAL, "workspace did not converge");
}

// ---------------------------------------------------------------------------
// public joins
// ---------------------------------------------------------------------------
int sj::out_acquire(sj_ctx *ctx, Workspace &w, OutSpec &os, unsigned long long P) {
    if (os.kind == OutSpec::INTO) {
        if ((unsigned long long)os.cap < P)
            return fail(ctx, SJ_EOVERFLOW, "need %llu pairs, cap %lld", P, (long long)os.cap);
        if (P && !os.into) return fail(ctx, SJ_EINVAL, "null output buffer");
        os.got = (int2 *)os.into;
        return SJ_OK;
    }
    if (P == 0) return SJ_OK;
    if (os.kind == OutSpec::WS) {
        int st = ensure(ctx, w.out, P * sizeof(int2));
        if (st) return st;
        os.got = (int2 *)w.out.p;
        return SJ_OK;
    }
    os.got = (int2 *)dev_alloc(ctx, P * sizeof(int2));
    if (!os.got) return fail(ctx, SJ_ENOMEM, "pair buffer of %llu pairs", P);
    return SJ_OK;
}

void sj::out_abandon(sj_ctx *ctx, OutSpec &os) {
    if (os.kind == OutSpec::LIB && os.got) dev_free(ctx, os.got);
    os.got = nullptr;
}

// The exact two-pass join (count, allocate, write) of a partitioned workspace
// whose count pass has run; stats->npairs is the total.
static int write_pass(sj_ctx *ctx, Workspace &w, const Stats &stats, const sj_opts *o, OutSpec &os,
                      int64_t *npairs) {
    const unsigned long long P = stats.npairs;
    *npairs = (int64_t)P;
    int st = out_acquire(ctx, w, os, P);
    if (st) return st;
    if (P == 0) return SJ_OK;
    if ((st = enqueue_sweep(ctx, w, MODE_WRITE, os.got, P, nullptr, nullptr, 2))) {
        out_abandon(ctx, os);
        return st;
    }
    if (o && o->sort_output && (st = sort_pairs(ctx, w, os.got, P))) {
        out_abandon(ctx, os);
        return st;
    }
    return SJ_OK;
}

// ---------------------------------------------------------------------------
// the two-level (blocked) path
// ---------------------------------------------------------------------------
// Blocks of G x G tiles holding about 1.5k entries each; false when the grid
// does not suit the blocked path (then the single-level path runs).
bool sj::plan_blocked(sj_ctx *ctx, const GridDev &g, long long nR, long long nS, BPlan &p) {
    if (!ctx->use_blocked || g.nx > 65535 || g.ny > 65535) return false;
    const double est = (double)(nR + nS) * 1.1 + 1.0;
    const double tgt = (double)ctx->block_target;
    const double nbt = est / tgt > 1.0 ? est / tgt : 1.0;
    int G = (int)ceil(sqrt((double)g.nx * (double)g.ny / nbt));
    if (G < 1) G = 1;
    if (G > kMaxG) G = kMaxG;
    for (;; G++) {
        if (G > kMaxG) return false;
        p.bx = (g.nx + G - 1) / G;
        p.by = (g.ny + G - 1) / G;
        if ((long long)p.bx * p.by <= kMaxBlocks) break;
    }
    p.G = G;
    p.nb = p.bx * p.by;
    p.nc = ctx->num_sms * l1_blocks_per_sm(p.nb);
    return true;
}

int sj::size_blocked(sj_ctx *ctx, Workspace &w, const BPlan &p) {
    int st;
    if ((st = ensure(ctx, w.stats, sizeof(Stats)))) return st;
    if ((st = ensure(ctx, w.bH, 8ull * p.nb * p.nc))) return st;
    if ((st = ensure(ctx, w.bTot, 8ull * p.nb))) return st;
    if ((st = ensure(ctx, w.bBoR, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bBoS, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bItems, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bImeta, 16ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bIns, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bEntR, sizeof(BEnt) * (w.bcap_r + 1)))) return st;
    if ((st = ensure(ctx, w.bEntS, sizeof(BEnt) * (w.bcap_s + 1)))) return st;
    if ((st = ensure(ctx, w.bPc, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bPoff, 8ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bResv, 8ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bFail, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bCur, 8ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bList, 4ull * list_pool_cap(w)))) return st;
    if ((st = ensure(ctx, w.bSpill, 8ull * kPairSpill * ctx->num_sms * ctx->bjoin_bps))) return st;
    if ((st = ensure(ctx, w.bJd, sizeof(JoinDesc) * 2))) return st;
    if ((st = ensure(ctx, w.bScanPart, 24ull * (bscan_chunks(p.nb) + 1)))) return st;
    return SJ_OK;
}

BArgs sj::blocked_args(Workspace &w, const BPlan &p, const float4 *R, long long nR, const float4 *S,
                          long long nS, const GridDev &g) {
    BArgs a;
    memset(&a, 0, sizeof a);   // optional fields (feature sampling) stay off
    a.R = R;
    a.nR = nR;
    a.S = S;
    a.nS = nS;
    a.g = g;
    a.G = p.G;
    a.gmul = p.G > 1 ? (unsigned)(0xFFFFFFFFull / (unsigned long long)p.G + 1ull) : 0u;
    a.bx = p.bx;
    a.by = p.by;
    a.nb = p.nb;
    a.H = (unsigned *)w.bH.p;
    a.btot = (unsigned *)w.bTot.p;
    a.bo_r = (unsigned *)w.bBoR.p;
    a.bo_s = (unsigned *)w.bBoS.p;
    a.items = (unsigned *)w.bItems.p;
    a.imeta = (uint4 *)w.bImeta.p;
    a.ins = (unsigned *)w.bIns.p;
    a.bent_r = (BEnt *)w.bEntR.p;
    a.bent_s = (BEnt *)w.bEntS.p;
    a.cap_r = w.bcap_r;
    a.cap_s = w.bcap_s;
    a.cur = nullptr;
    a.lpool = (unsigned *)w.bList.p;
    a.lpool_cap = list_pool_cap(w);
    a.scan_part = (unsigned long long *)w.bScanPart.p;
    a.jd = (const JoinDesc *)w.bJd.p;   // filled by enqueue_blocked_partition
    a.nj = 1;
    a.pts = w.in_pts;
    a.h = w.in_h;
    a.nbt = p.nb;
    a.fine_cap = kFineCap;
    a.st = (Stats *)w.stats.p;
    return a;
}

BJoinOut sj::bjoin_out(Workspace &w, int slot) {
    BJoinOut o;
    memset(&o, 0, sizeof o);
    o.work_slot = slot;
    o.cnt_out = (unsigned *)w.bPc.p;
    o.off_in = (const unsigned long long *)w.bPoff.p;
    o.resv = (unsigned long long *)w.bResv.p;
    o.fail = (unsigned *)w.bFail.p;
    o.nfail = &((Stats *)w.stats.p)->nfail;
    o.spill = (int2 *)w.bSpill.p;
    return o;
}

// L1 partition of the blocked path (count, scan, write).
int sj::upload_joins(sj_ctx *ctx, Workspace &w, const JoinDesc *h, int nj) {
    int st = ensure(ctx, w.bJd, sizeof(JoinDesc) * (nj + 1));
    if (st) return st;
    memcpy(ctx->h_jd, h, sizeof(JoinDesc) * nj);
    cudaError_t e = copy_async(ctx, w.bJd.p, ctx->h_jd, sizeof(JoinDesc) * nj);
    return e ? cuda_fail(ctx, e, "join table copy") : SJ_OK;
}

// The descriptor of a single join (the kernels read joins from a table).
int sj::upload_single_join(sj_ctx *ctx, Workspace &w, const BArgs &a) {
    JoinDesc d;
    memset(&d, 0, sizeof d);
    d.R = a.R;
    d.S = a.S;
    d.nR = a.nR;
    d.nS = a.nS;
    d.in_off = 0;
    d.g = a.g;
    d.G = a.G;
    d.gmul = a.gmul;
    d.bx = a.bx;
    d.by = a.by;
    d.boff = 0;
    d.h = a.h;
    return upload_joins(ctx, w, &d, 1);
}

int sj::enqueue_blocked_partition(sj_ctx *ctx, Workspace &w, const BPlan &p, const BArgs &a) {
    cudaError_t e;
    cudaStream_t s = ctx->stream;
    {
        int st = upload_single_join(ctx, w, a);
        if (st) return st;
    }
    {
        PhaseScope ph(ctx, PH_RESET, 0);
        if ((e = zero_async(ctx, w.stats.p, sizeof(Stats)))) return cuda_fail(ctx, e, "memset");
        if ((e = zero_async(ctx, w.bPc.p, 4ull * (p.nb + 1)))) return cuda_fail(ctx, e, "memset");
    }
    {
        PhaseScope ph(ctx, PH_COUNT, 1);
        if ((e = launch_bcount(a, p.nc, s))) return cuda_fail(ctx, e, "block count kernel");
    }
    {
        PhaseScope ph(ctx, PH_SCAN, 2);
        if ((e = launch_bscan(a, p.nc, s))) return cuda_fail(ctx, e, "block scan kernels");
    }
    {
        PhaseScope ph(ctx, PH_SCATTER, 1);
        if ((e = launch_bscatter(a, p.nc, s))) return cuda_fail(ctx, e, "block write kernel");
    }
    return SJ_OK;
}

// Blocked partition + count pass.  *use_direct is set when a tile holds more
// entries than shared memory (the caller then runs the single-level path).
int sj::blocked_partition_count(sj_ctx *ctx, Workspace &w, const BPlan &p, const float4 *R,
                                   long long nR, const float4 *S, long long nS, const GridDev &g,
                                   Stats *stats, bool *use_direct, int flags, unsigned char *tile_axis) {
    const bool adaptive = flags & SJ_SWEEP_ADAPTIVE;
    *use_direct = false;
    w.bcap_r = std::max<unsigned long long>(w.bcap_r, (unsigned long long)nR + nR / 8 + 1024);
    w.bcap_s = std::max<unsigned long long>(w.bcap_s, (unsigned long long)nS + nS / 8 + 1024);
    for (int attempt = 0; attempt < 3; attempt++) {
        int st;
        if ((st = size_blocked(ctx, w, p))) return st;
        BArgs a = blocked_args(w, p, R, nR, S, nS, g);
        if (ctx->shared_cursors) a.cur = (unsigned *)w.bCur.p;
        a.adaptive = adaptive;
        a.gbda = (flags & SJ_DEDUP_GBDA) != 0;
        if ((st = enqueue_blocked_partition(ctx, w, p, a))) return st;
        cudaError_t e;
        {
            PhaseScope ph(ctx, PH_SWEEP_COUNT, 1);
            BJoinOut bo = bjoin_out(w, 0);
            bo.tile_axis = tile_axis;
            if ((e = launch_bjoin(MODE_COUNT, a, bo, ctx->num_sms * ctx->bjoin_bps, ctx->stream)))
                return cuda_fail(ctx, e, "block join kernel");
        }
        {
            PhaseScope ph(ctx, PH_PAIRSCAN, 1);
            if ((e = launch_scan_pairs((const unsigned *)w.bPc.p, (unsigned)p.nb, (unsigned long long *)w.bPoff.p,
                                       (Stats *)w.stats.p, ctx->stream)))
                return cuda_fail(ctx, e, "pair-count scan");
        }
        if ((st = read_stats(ctx, w, stats))) return st;
        if (stats->err & kErrBadRect)
            return fail(ctx, SJ_EINVAL, "invalid rectangle: NaN/Inf coordinate or xl > xu / yl > yu");
        if (stats->err & kErrEntCap) {
            w.bcap_r = std::max<unsigned long long>(w.bcap_r, stats->e_r + stats->e_r / 8 + 1024);
            w.bcap_s = std::max<unsigned long long>(w.bcap_s, stats->e_s + stats->e_s / 8 + 1024);
            continue;
        }
        if (stats->err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats->err);
        if (stats->need_direct) *use_direct = true;
        memset(&ctx->last, 0, sizeof ctx->last);
        ctx->last.path = 1;
        ctx->last.block_side = p.G;
        ctx->last.blocks = p.nb;
        ctx->last.work_items = stats->nchunks;
        ctx->last.l1_entries_r = (int64_t)stats->e_r;
        ctx->last.l1_entries_s = (int64_t)stats->e_s;
        ctx->last.npairs = (int64_t)stats->npairs;
        ctx->last.y_sweep_tiles = adaptive ? (int64_t)stats->naxis_y : 0;
        ctx->last.dedup = (flags & SJ_DEDUP_GBDA) ? 1 : 0;
        return SJ_OK;
    }
    return fail(ctx, SJ_EINTERNAL, "blocked workspace did not converge");
}

// One pass on the single-level path (one-pass modes when a tile exceeds
// shared memory): the small tiles are counted (they are cheap to sweep
// twice) and the large tiles' candidate chunks planned; the output holds the
// small tiles' exact pairs plus, as an upper bound for the large tiles, one
// pair per candidate of their chunks.  Then the small tiles are written at
// their exact offsets and every candidate chunk of the large tiles appends
// its pairs after them with one atomic: each large-tile candidate is
// examined once.  The first P pairs of the output are the result.
// ONE_PASS_UNSUITED when a caller buffer is smaller than the bound (the exact
// two-pass join then runs).
static int single_level_one_pass(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S,
                                 long long nS, const GridDev &g, const sj_opts *o, OutSpec &os, int64_t *npairs) {
    const long long T = (long long)g.nx * g.ny;
    w.cap_r = std::max<unsigned long long>(w.cap_r, (unsigned long long)nR + nR / 4 + 1024);
    w.cap_s = std::max<unsigned long long>(w.cap_s, (unsigned long long)nS + nS / 4 + 1024);
    cudaStream_t s = ctx->stream;
    for (int attempt = 0; attempt < 3; attempt++) {
        int st;
        if ((st = size_workspace(ctx, w, T))) return st;
        if (!w.lcoff.p) return ONE_PASS_UNSUITED;
        if ((st = enqueue_partition(ctx, w, R, nR, S, nS, g))) return st;
        cudaError_t e;
        const unsigned nslots = w.nch_cap + w.vb_cap;
        if ((e = zero_async(ctx, w.pc.p, 4ull * nslots))) return cuda_fail(ctx, e, "memset");
        SweepArgs a = sweep_args(w);
        a.work_slot = 0;
        {
            PhaseScope ph(ctx, PH_SWEEP_COUNT, 1);
            if ((e = launch_sweep_chunks(MODE_COUNT, a, ctx->num_sms * ctx->sweep_bps, s)))
                return cuda_fail(ctx, e, "sweep kernel");
        }
        {
            PhaseScope ph(ctx, PH_LSWEEP_COUNT, 2);
            if ((e = launch_large_plan(large_args(w), ctx->num_sms * 4, s)))
                return cuda_fail(ctx, e, "large-tile plan");
        }
        {
            PhaseScope ph(ctx, PH_PAIRSCAN, 1);
            if ((e = launch_scan_pairs((const unsigned *)w.pc.p, nslots, (unsigned long long *)w.poff.p,
                                       (Stats *)w.stats.p, s)))
                return cuda_fail(ctx, e, "pair-count scan");
        }
        Stats stats;
        if ((st = read_stats(ctx, w, &stats))) return st;
        if (stats.err & kErrBadRect)
            return fail(ctx, SJ_EINVAL, "invalid rectangle: NaN/Inf coordinate or xl > xu / yl > yu");
        if (stats.err & kErrTooMany) return fail(ctx, SJ_EINVAL, "more than 2^31 replicated entries on one side");
        if (stats.err & (kErrEntCap | kErrChunkCap | kErrLargeCap)) {
            w.cap_r = std::max<unsigned long long>(w.cap_r, stats.e_r + stats.e_r / 8 + 1024);
            w.cap_s = std::max<unsigned long long>(w.cap_s, stats.e_s + stats.e_s / 8 + 1024);
            continue;
        }
        if (stats.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
        const unsigned long long P_small = stats.npairs;
        const unsigned long long bound = P_small + (unsigned long long)stats.nlch * kLargeCandChunk;
        if (os.kind == OutSpec::INTO && (unsigned long long)os.cap < bound) return ONE_PASS_UNSUITED;
        if ((st = out_acquire(ctx, w, os, bound))) return st;
        if (bound) {
            SweepArgs wa = sweep_args(w);
            wa.out = os.got;
            wa.cap = bound;
            wa.work_slot = 2;
            PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
            if ((e = launch_sweep_chunks(MODE_WRITE, wa, ctx->num_sms * ctx->sweep_bps, s))) {
                out_abandon(ctx, os);
                return cuda_fail(ctx, e, "sweep kernel");
            }
        }
        if (stats.nlch) {
            SweepArgs la = sweep_args(w);
            la.out = os.got;
            la.cap = bound;
            la.work_slot = 3;
            la.base = P_small;
            la.append = &((Stats *)w.stats.p)->apairs;
            PhaseScope ph(ctx, PH_LSWEEP_WRITE, 1);
            if ((e = launch_large_append(large_args(w), la, ctx->num_sms * 4, s))) {
                out_abandon(ctx, os);
                return cuda_fail(ctx, e, "large-tile sweep kernel");
            }
        }
        if ((st = read_stats(ctx, w, &stats))) {
            out_abandon(ctx, os);
            return st;
        }
        if (stats.err) {
            out_abandon(ctx, os);
            return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
        }
        const unsigned long long P = P_small + stats.apairs;
        *npairs = (int64_t)P;
        memset(&ctx->last, 0, sizeof ctx->last);
        ctx->last.entries_r = (int64_t)stats.e_r;
        ctx->last.entries_s = (int64_t)stats.e_s;
        ctx->last.npairs = (int64_t)P;
        ctx->last.one_pass = 1;
        ctx->last.capacity = (int64_t)bound;
        if (o && o->sort_output && P && (st = sort_pairs(ctx, w, os.got, P))) {
            out_abandon(ctx, os);
            return st;
        }
        return SJ_OK;
    }
    return fail(ctx, SJ_EINTERNAL, "workspace did not converge");
}

static int join_core_body(sj_ctx *ctx, Workspace &w, const sj_rect *d_R, int64_t nR, const sj_rect *d_S,
                          int64_t nS, const GridDev &gd, const sj_opts *o, OutSpec &os, int64_t *npairs) {
    const int mode = o ? o->mode : SJ_TWO_PASS;
    {   // 1D grids (stripes): the stripe kernel, exact two-pass, in any mode
        const int st = join_stripes(ctx, w, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, o, os, npairs);
        if (st != STRIPES_UNSUITED) return st;
        os.got = nullptr;
    }
    const bool one_pass = (mode == SJ_ONE_PASS || mode == SJ_ONE_PASS_HEUR ||
                           (mode == SJ_AUTO && ctx->mlp_loaded));
    bool direct_known = false;   // a tile exceeds shared memory: the single-level path
    if (one_pass) {
        int st = join_one_pass_spec(ctx, w, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, o,
                                    mode == SJ_ONE_PASS_HEUR ? 1 : 0, os, npairs, nullptr);
        if (st != ONE_PASS_UNSUITED && st != ONE_PASS_DIRECT) return st;
        direct_known = st == ONE_PASS_DIRECT;
        os.got = nullptr;   // the grid or the data need another path
    }
    Stats stats;
    int st;
    BPlan bp;
    const int flags = o ? o->flags : 0;
    if (!direct_known && plan_blocked(ctx, gd, nR, nS, bp)) {
        bool direct = false;
        if ((st = blocked_partition_count(ctx, w, bp, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd,
                                          &stats, &direct, flags)))
            return st;
        if (!direct) {
            const unsigned long long P = stats.npairs;
            *npairs = (int64_t)P;
            if ((st = out_acquire(ctx, w, os, P))) return st;
            if (P == 0) return SJ_OK;
            BArgs a = blocked_args(w, bp, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd);
            if (ctx->shared_cursors) a.cur = (unsigned *)w.bCur.p;
            a.adaptive = (flags & SJ_SWEEP_ADAPTIVE) != 0;
            a.gbda = (flags & SJ_DEDUP_GBDA) != 0;
            BJoinOut bo = bjoin_out(w, 1);
            bo.out = os.got;
            bo.cap = P;
#if SJ_CHECK
            // debug build, self-test of the checks: one slot fewer than the
            // pairs, so the bound of the last pair's write fails (the write
            // is skipped, nothing is written out of bounds)
            if (getenv("SJ_CHECK_SELFTEST")) bo.cap = P - 1;
#endif
            cudaError_t e;
            {
                PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
                if ((e = launch_bjoin(MODE_WRITE, a, bo, ctx->num_sms * ctx->bjoin_bps, ctx->stream))) {
                    out_abandon(ctx, os);
                    return cuda_fail(ctx, e, "block join kernel");
                }
            }
            if (o && o->sort_output && (st = sort_pairs(ctx, w, os.got, P))) {
                out_abandon(ctx, os);
                return st;
            }
            return SJ_OK;
        }
    }
    if (w.in_pts) return PTS_UNSUITED;   // the single-level path reads rectangles only
    if (one_pass) {
        st = single_level_one_pass(ctx, w, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, o, os, npairs);
        if (st != ONE_PASS_UNSUITED) return st;
        os.got = nullptr;
    }
    st = partition_and_count(ctx, w, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, &stats, true);
    if (st) return st;
    return write_pass(ctx, w, stats, o, os, npairs);
}

int sj::join_core(sj_ctx *ctx, Workspace &w, const sj_rect *d_R, int64_t nR, const sj_rect *d_S,
                  int64_t nS, const GridDev &gd, const sj_opts *o, OutSpec &os, int64_t *npairs) {
    int st = join_core_body(ctx, w, d_R, nR, d_S, nS, gd, o, os, npairs);
    if (st == SJ_OK && (st = check_tail(ctx, w))) out_abandon(ctx, os);
    return st;
}

int sj::check_opts(sj_ctx *ctx, const sj_opts *o) {
    if (!o) return SJ_OK;
    if (o->flags & ~(SJ_SWEEP_ADAPTIVE | SJ_DEDUP_GBDA))
        return fail(ctx, SJ_EINVAL, "unknown sj_opts.flags bits 0x%x", o->flags);
    if ((o->flags & SJ_SWEEP_ADAPTIVE) && (o->flags & SJ_DEDUP_GBDA))
        return fail(ctx, SJ_EINVAL, "SJ_SWEEP_ADAPTIVE and SJ_DEDUP_GBDA cannot be combined");
    if (o->mode < SJ_TWO_PASS || o->mode > SJ_AUTO) return fail(ctx, SJ_EINVAL, "unknown mode %d", o->mode);
    if (!(o->margin >= 0.0f) || !(o->margin < 1e6f)) return fail(ctx, SJ_EINVAL, "margin out of range");
    return SJ_OK;
}

extern "C" int sj_join(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                       const sj_grid *g, const sj_opts *o, sj_pair **d_pairs, int64_t *npairs) {
    GridDev gd;
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, &gd);
    if (st) return st;
    if ((st = check_opts(ctx, o))) return st;
    if (!d_pairs || !npairs) return fail(ctx, SJ_EINVAL, "null output pointer");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    *d_pairs = nullptr;
    OutSpec os{OutSpec::LIB};
    if ((st = join_core(ctx, ctx->ws, d_R, nR, d_S, nS, gd, o, os, npairs))) return st;
    *d_pairs = (sj_pair *)os.got;
    return SJ_OK;
}

extern "C" int sj_join_into(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S,
                            int64_t nS, const sj_grid *g, const sj_opts *o, sj_pair *d_buf,
                            int64_t cap, int64_t *npairs) {
    GridDev gd;
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, &gd);
    if (st) return st;
    if ((st = check_opts(ctx, o))) return st;
    if (cap < 0 || !npairs) return fail(ctx, SJ_EINVAL, "negative capacity or null npairs");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    OutSpec os{OutSpec::INTO};
    os.into = d_buf;
    os.cap = cap;
    return join_core(ctx, ctx->ws, d_R, nR, d_S, nS, gd, o, os, npairs);
}

extern "C" int sj_join_host(sj_ctx *ctx, const sj_rect *h_R, int64_t nR, const sj_rect *h_S,
                            int64_t nS, const sj_grid *g, const sj_opts *o, sj_pair *h_out,
                            int64_t cap, int64_t *npairs) {
    if (!ctx) return SJ_EINVAL;
    if ((nR && !h_R) || (nS && !h_S)) return fail(ctx, SJ_EINVAL, "null rectangle pointer");
    if (nR < 0 || nS < 0 || nR >= SJ_MAX_N || nS >= SJ_MAX_N)
        return fail(ctx, SJ_EINVAL, "sizes must satisfy 0 <= n < 2^30");
    if (cap < 0 || !npairs) return fail(ctx, SJ_EINVAL, "negative capacity or null npairs");
    int st;
    if ((st = check_opts(ctx, o))) return st;
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    Workspace &w = ctx->ws;
    if ((st = ensure(ctx, w.in_r, 16ull * nR + 16))) return st;
    if ((st = ensure(ctx, w.in_s, 16ull * nS + 16))) return st;
    cudaError_t e;
    {
        PhaseScope ph(ctx, PH_OTHER, 0);
        if (nR && (e = cudaMemcpyAsync(w.in_r.p, h_R, 16ull * nR, cudaMemcpyHostToDevice, ctx->stream)))
            return cuda_fail(ctx, e, "copy of R to the device");
        if (nS && (e = cudaMemcpyAsync(w.in_s.p, h_S, 16ull * nS, cudaMemcpyHostToDevice, ctx->stream)))
            return cuda_fail(ctx, e, "copy of S to the device");
    }
    GridDev gd;
    if ((st = check_inputs(ctx, (const sj_rect *)w.in_r.p, nR, (const sj_rect *)w.in_s.p, nS, g, &gd)))
        return st;
    OutSpec os{OutSpec::WS};
    if ((st = join_core(ctx, w, (const sj_rect *)w.in_r.p, nR, (const sj_rect *)w.in_s.p, nS, gd, o, os,
                        npairs)))
        return st;
    if (*npairs > cap) return fail(ctx, SJ_EOVERFLOW, "need %lld pairs, cap %lld", (long long)*npairs, (long long)cap);
    if (*npairs) {
        if (!h_out) return fail(ctx, SJ_EINVAL, "null output buffer");
        if ((e = cudaMemcpyAsync(h_out, os.got, 8ull * *npairs, cudaMemcpyDeviceToHost, ctx->stream)))
            return cuda_fail(ctx, e, "copy of the pairs to the host");
    }
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
    return SJ_OK;
}

extern "C" int sj_count(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                        const sj_grid *g, int64_t *out_npairs) {
    GridDev gd;
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, &gd);
    if (st) return st;
    if (!out_npairs) return fail(ctx, SJ_EINVAL, "null out_npairs");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    Stats stats;
    BPlan bp;
    if (plan_blocked(ctx, gd, nR, nS, bp)) {
        bool direct = false;
        if ((st = blocked_partition_count(ctx, ctx->ws, bp, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd,
                                          &stats, &direct, 0)))
            return st;
        if (!direct) {
            *out_npairs = (int64_t)stats.npairs;
            return SJ_OK;
        }
    }
    if ((st = partition_and_count(ctx, ctx->ws, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd,
                                  &stats, true)))
        return st;
    *out_npairs = (int64_t)stats.npairs;
    return SJ_OK;
}

// The per-tile sweep axes of SJ_SWEEP_ADAPTIVE (partition + count pass of the
// two-level path with the adaptive kernel, which also writes the axes).
extern "C" int sj_tile_axes(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                            const sj_grid *g, uint8_t *d_axis) {
    GridDev gd;
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, &gd);
    if (st) return st;
    if (!d_axis) return fail(ctx, SJ_EINVAL, "null d_axis");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    BPlan bp;
    if (!plan_blocked(ctx, gd, nR, nS, bp)) return fail(ctx, SJ_EINVAL, "grid does not suit the two-level path");
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_axis, 0, (size_t)gd.nx * (size_t)gd.ny, ctx->stream))) return cuda_fail(ctx, e, "memset");
    Stats stats;
    bool direct = false;
    if ((st = blocked_partition_count(ctx, ctx->ws, bp, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, &stats,
                                      &direct, SJ_SWEEP_ADAPTIVE, (unsigned char *)d_axis)))
        return st;
    if (direct) return fail(ctx, SJ_EINVAL, "a tile exceeds shared memory: the single-level path sweeps along x");
    return SJ_OK;
}

// ---------------------------------------------------------------------------
// per-tile statistics
// ---------------------------------------------------------------------------
extern "C" int sj_tile_stats(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S,
                             int64_t nS, const sj_grid *g, uint32_t *d_cnt_r, uint32_t *d_cnt_s,
                             uint32_t *d_pairs_per_tile) {
    GridDev gd;
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, &gd);
    if (st) return st;
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    Workspace &w = ctx->ws;
    Stats stats;
    if ((st = partition_and_count(ctx, w, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, &stats,
                                  false)))
        return st;
    cudaError_t e;
    const long long T = (long long)gd.nx * gd.ny;
    if (d_cnt_r || d_cnt_s) {
        PhaseScope ph(ctx, PH_OTHER, 1);
        if ((e = launch_tile_counts((const uint2 *)w.off.p, T, d_cnt_r, d_cnt_s, ctx->stream)))
            return cuda_fail(ctx, e, "tile counts");
    }
    if (d_pairs_per_tile) {
        if ((e = cudaMemsetAsync(d_pairs_per_tile, 0, 4ull * T, ctx->stream))) return cuda_fail(ctx, e, "memset");
        if ((st = enqueue_sweep(ctx, w, MODE_TILES, nullptr, 0, nullptr, d_pairs_per_tile, 4))) return st;
    }
    if ((st = read_stats(ctx, w, &stats))) return st;
    if (stats.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
    return SJ_OK;
}

// ---------------------------------------------------------------------------
// partitions as objects
// ---------------------------------------------------------------------------
extern "C" int sj_partition(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S,
                            int64_t nS, const sj_grid *g, sj_part **out) {
    GridDev gd;
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, &gd);
    if (st) return st;
    if (!out) return fail(ctx, SJ_EINVAL, "null out");
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    sj_part *p = new (std::nothrow) sj_part();
    if (!p) return fail(ctx, SJ_ENOMEM, "host allocation");
    p->ctx = ctx;
    p->grid = gd;
    p->nR = nR;
    p->nS = nS;
    Stats stats;
    if ((st = partition_and_count(ctx, p->ws, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, &stats,
                                  false))) {
        release(ctx, p->ws);
        delete p;
        return st;
    }
    p->e_r = stats.e_r;
    p->e_s = stats.e_s;
    *out = p;
    return SJ_OK;
}

extern "C" int sj_part_view_get(const sj_part *p, sj_part_view *v) {
    if (!p || !v) return SJ_EINVAL;
    v->n_tiles = (int64_t)p->grid.nx * p->grid.ny;
    v->e_r = (int64_t)p->e_r;
    v->e_s = (int64_t)p->e_s;
    v->off = p->ws.off.p;
    v->ent_r = p->ws.ent_r.p;
    v->id_r = p->ws.id_r.p;
    v->ent_s = p->ws.ent_s.p;
    v->id_s = p->ws.id_s.p;
    return SJ_OK;
}

extern "C" int sj_part_join(sj_ctx *ctx, sj_part *p, const sj_opts *o, sj_pair **d_pairs,
                            int64_t *npairs) {
    if (!ctx || !p || !d_pairs || !npairs) return SJ_EINVAL;
    if (p->ctx != ctx) return fail(ctx, SJ_EINVAL, "partition belongs to another context");
    int st = check_opts(ctx, o);
    if (st) return st;
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    Workspace &w = p->ws;
    cudaError_t e;
    const unsigned nslots = w.nch_cap + w.vb_cap;
    // reset the per-call counters but keep the partition's totals
    {
        PhaseScope ph(ctx, PH_RESET, 1);
        if ((e = launch_reset_counters((Stats *)w.stats.p, ctx->stream))) return cuda_fail(ctx, e, "reset");
        if ((e = zero_async(ctx, w.pc.p, 4ull * nslots))) return cuda_fail(ctx, e, "memset");
    }
    if ((st = enqueue_sweep(ctx, w, MODE_COUNT, nullptr, 0, nullptr, nullptr, 0))) return st;
    {
        PhaseScope ph(ctx, PH_PAIRSCAN, 1);
        if ((e = launch_scan_pairs((const unsigned *)w.pc.p, nslots, (unsigned long long *)w.poff.p,
                                   (Stats *)w.stats.p, ctx->stream)))
            return cuda_fail(ctx, e, "pair-count scan");
    }
    Stats stats;
    if ((st = read_stats(ctx, w, &stats))) return st;
    if (stats.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
    OutSpec os{OutSpec::LIB};
    *d_pairs = nullptr;
    if ((st = write_pass(ctx, w, stats, o, os, npairs))) return st;
    if ((st = check_tail(ctx, w))) {
        out_abandon(ctx, os);
        return st;
    }
    *d_pairs = (sj_pair *)os.got;
    return SJ_OK;
}

extern "C" void sj_part_free(sj_part *p) {
    if (!p) return;
    DeviceGuard dg(p->ctx->device);
    release(p->ctx, p->ws);
    delete p;
}
