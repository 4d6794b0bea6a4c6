// api_learned.cu -- C ABI of the learned result-count predictor (sj_mlp_*,
// sj_block_features, sj_set_model) and the one-pass join that uses it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "sj_internal.h"
#include "sj_learned.h"

using namespace sj;

struct sj_mlp {
    sj_ctx *ctx = nullptr;
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
    float *b1 = nullptr, *b2 = nullptr, *b3 = nullptr;
    void *block = nullptr;   // one allocation holding everything above
    int step = 0;
};

static MlpWeights weights_of(const sj_mlp *m) {
    MlpWeights w;
    w.w1 = m->w1;
    w.w2 = m->w2;
    w.w3 = m->w3;
    w.b1 = m->b1;
    w.b2 = m->b2;
    w.b3 = m->b3;
    return w;
}

static MlpParams params_of(const sj_mlp *m) {
    MlpParams p;
    p.master = m->master;
    p.m = m->m;
    p.v = m->v;
    return p;
}

extern "C" int sj_mlp_create(sj_ctx *ctx, sj_mlp **out) {
    if (!ctx || !out) return SJ_EINVAL;
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    sj_mlp *m = new (std::nothrow) sj_mlp();
    if (!m) return fail(ctx, SJ_ENOMEM, "host allocation");
    m->ctx = ctx;
    const size_t fp = 4ull * kParams;
    const size_t total = 5 * fp + 256 + 2ull * (kH1 * kFeat + kH2 * kH1 + kH2) + 4ull * (kH1 + kH2 + 1) + 1024;
    unsigned char *base = (unsigned char *)dev_alloc(ctx, total);
    if (!base) {
        delete m;
        return fail(ctx, SJ_ENOMEM, "model allocation");
    }
    m->block = base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base + off;
        off += bytes;
        return p;
    };
    m->master = (float *)take(fp);
    m->m = (float *)take(fp);
    m->v = (float *)take(fp);
    m->grad = (float *)take(fp);
    m->loss = (float *)take(256);
    m->w1 = (__nv_bfloat16 *)take(2ull * kH1 * kFeat);
    m->w2 = (__nv_bfloat16 *)take(2ull * kH2 * kH1);
    m->w3 = (__nv_bfloat16 *)take(2ull * kH2);
    m->b1 = (float *)take(4ull * kH1);
    m->b2 = (float *)take(4ull * kH2);
    m->b3 = (float *)take(4);
    cudaError_t e;
    if ((e = cudaMemsetAsync(base, 0, total, ctx->stream))) {
        dev_free(ctx, base);
        delete m;
        return cuda_fail(ctx, e, "memset");
    }
    *out = m;
    return SJ_OK;
}

extern "C" void sj_mlp_free(sj_mlp *m) {
    if (!m) return;
    DeviceGuard dg(m->ctx->device);
    if (m->ctx->model == m) {
        m->ctx->model = nullptr;
        m->ctx->mlp_loaded = false;
    }
    dev_free(m->ctx, m->block);
    delete m;
}

extern "C" int sj_mlp_set_params(sj_ctx *ctx, sj_mlp *m, const float *h_params) {
    if (!ctx || !m || !h_params) return SJ_EINVAL;
    DeviceGuard dg(ctx->device);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(m->master, h_params, 4ull * kParams, cudaMemcpyHostToDevice, ctx->stream)))
        return cuda_fail(ctx, e, "parameter upload");
    if ((e = cudaMemsetAsync(m->m, 0, 4ull * kParams, ctx->stream))) return cuda_fail(ctx, e, "memset");
    if ((e = cudaMemsetAsync(m->v, 0, 4ull * kParams, ctx->stream))) return cuda_fail(ctx, e, "memset");
    m->step = 0;
    PhaseScope ph(ctx, PH_MODEL, 1);
    if ((e = launch_mlp_publish(params_of(m), weights_of(m), ctx->stream))) return cuda_fail(ctx, e, "publish");
    // the host array may be freed by the caller right after return
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "sync");
    return SJ_OK;
}

// bf16 -> float on the host (exact: bf16 is the upper half of a float)
static float bf16_to_float(__nv_bfloat16 h) {
    unsigned short bits;
    memcpy(&bits, &h, 2);
    const unsigned u = (unsigned)bits << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

extern "C" int sj_mlp_get_params(sj_ctx *ctx, const sj_mlp *m, float *h_params, float *h_inference) {
    if (!ctx || !m) return SJ_EINVAL;
    DeviceGuard dg(ctx->device);
    cudaError_t e;
    if (h_params &&
        (e = cudaMemcpyAsync(h_params, m->master, 4ull * kParams, cudaMemcpyDeviceToHost, ctx->stream)))
        return cuda_fail(ctx, e, "parameter download");
    if (h_inference) {
        static_assert(sizeof(__nv_bfloat16) == 2, "bf16 size");
        __nv_bfloat16 w1[kH1 * kFeat], w2[kH2 * kH1], w3[kH2];
        float b1[kH1], b2[kH2], b3;
        if ((e = cudaMemcpyAsync(w1, m->w1, sizeof w1, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(w2, m->w2, sizeof w2, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(w3, m->w3, sizeof w3, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(b1, m->b1, sizeof b1, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(b2, m->b2, sizeof b2, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(&b3, m->b3, sizeof b3, cudaMemcpyDeviceToHost, ctx->stream)))
            return cuda_fail(ctx, e, "weight download");
        if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "sync");
        // the device keeps W1 and W2 input-major (w1[k][j] = W1[j][k]); the
        // parameter vector is row-major
        for (int k = 0; k < kH1 * kFeat; k++) h_inference[kOffW1 + k] = bf16_to_float(w1[(k % kFeat) * kH1 + k / kFeat]);
        for (int k = 0; k < kH1; k++) h_inference[kOffB1 + k] = b1[k];
        for (int k = 0; k < kH2 * kH1; k++) h_inference[kOffW2 + k] = bf16_to_float(w2[(k % kH1) * kH2 + k / kH1]);
        for (int k = 0; k < kH2; k++) h_inference[kOffB2 + k] = b2[k];
        for (int k = 0; k < kH2; k++) h_inference[kOffW3 + k] = bf16_to_float(w3[k]);
        h_inference[kOffB3] = b3;
    }
    if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "sync");
    return SJ_OK;
}

static int mlp_grid(sj_ctx *ctx, int64_t n) {
    const long long per = 8;   // samples per warp-iteration group
    long long g = (n + per * 8 - 1) / (per * 8);
    const long long cap = (long long)ctx->num_sms * 4;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// Inference: one thread per sample, 64 per CTA.
static int mlp_infer_grid(sj_ctx *ctx, int64_t n) {
    long long g = (n + 63) / 64;
    const long long cap = (long long)ctx->num_sms * 16;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

extern "C" int sj_mlp_forward(sj_ctx *ctx, const sj_mlp *m, const float *d_X, int64_t n, float *d_y) {
    if (!ctx || !m || n < 0 || (n && (!d_X || !d_y))) return SJ_EINVAL;
    if (n == 0) return SJ_OK;
    if (reinterpret_cast<uintptr_t>(d_X) & 15) return fail(ctx, SJ_EINVAL, "d_X must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    PhaseScope ph(ctx, PH_MODEL, 1);
    cudaError_t e = launch_mlp_forward(weights_of(m), d_X, n, nullptr, d_y, mlp_infer_grid(ctx, n), ctx->stream);
    return e ? cuda_fail(ctx, e, "mlp forward") : SJ_OK;
}

extern "C" int sj_mlp_grad(sj_ctx *ctx, const sj_mlp *m, const float *d_X, const float *d_Y, int64_t n,
                           float *d_grad, float *d_loss) {
    if (!ctx || !m || n < 0 || !d_grad || !d_loss || (n && (!d_X || !d_Y))) return SJ_EINVAL;
    DeviceGuard dg(ctx->device);
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_grad, 0, 4ull * kParams, ctx->stream))) return cuda_fail(ctx, e, "memset");
    if ((e = cudaMemsetAsync(d_loss, 0, 4, ctx->stream))) return cuda_fail(ctx, e, "memset");
    if (n == 0) return SJ_OK;
    PhaseScope ph(ctx, PH_MODEL, 1);
    e = launch_mlp_grad(weights_of(m), d_X, d_Y, n, d_grad, d_loss, mlp_grid(ctx, n), ctx->stream);
    return e ? cuda_fail(ctx, e, "mlp gradient") : SJ_OK;
}

extern "C" int sj_mlp_train_step(sj_ctx *ctx, sj_mlp *m, const float *d_X, const float *d_Y, int64_t n, float lr,
                                 float *d_loss) {
    if (!ctx || !m || n <= 0 || !d_X || !d_Y || !(lr > 0.0f)) return SJ_EINVAL;
    DeviceGuard dg(ctx->device);
    int st = sj_mlp_grad(ctx, m, d_X, d_Y, n, m->grad, m->loss);
    if (st) return st;
    m->step++;
    cudaError_t e;
    {
        PhaseScope ph(ctx, PH_MODEL, 2);
        if ((e = launch_adam(params_of(m), m->grad, lr, 0.9f, 0.999f, 1e-8f, m->step, ctx->stream)))
            return cuda_fail(ctx, e, "adam");
        if ((e = launch_mlp_publish(params_of(m), weights_of(m), ctx->stream))) return cuda_fail(ctx, e, "publish");
    }
    if (d_loss && (e = cudaMemcpyAsync(d_loss, m->loss, 4, cudaMemcpyDeviceToDevice, ctx->stream)))
        return cuda_fail(ctx, e, "loss copy");
    return SJ_OK;
}

extern "C" int sj_set_model(sj_ctx *ctx, const sj_mlp *m) {
    if (!ctx) return SJ_EINVAL;
    if (m && m->ctx != ctx) return fail(ctx, SJ_EINVAL, "model belongs to another context");
    ctx->model = m;
    ctx->mlp_loaded = m != nullptr;
    ctx->onepass_scale = 1.0f;   // a new model starts uncalibrated
    return SJ_OK;
}

// ---------------------------------------------------------------------------
// features + labels
// ---------------------------------------------------------------------------
int sj::size_learned(sj_ctx *ctx, Workspace &w, const BPlan &p) {
    int st;
    if ((st = ensure(ctx, w.bFeatRaw, 4ull * kRawPerBlock * p.nb))) return st;
    if ((st = ensure(ctx, w.bFeat, 4ull * kFeat * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bPred, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bOrder, 4ull * (p.nb + 1)))) return st;
    if ((st = ensure(ctx, w.bCapTot, kPlanScratch))) return st;
    return SJ_OK;
}

extern "C" int sj_block_features(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                                 const sj_grid *g, float *d_feat, float *d_label, int32_t *d_block, int64_t cap,
                                 int64_t *n_items) {
    GridDev gd;
    int st = check_inputs(ctx, d_R, nR, d_S, nS, g, &gd);
    if (st) return st;
    if (!n_items || cap < 0) return fail(ctx, SJ_EINVAL, "null n_items or negative cap");
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    BPlan p;
    if (!plan_blocked(ctx, gd, nR, nS, p)) return fail(ctx, SJ_EINVAL, "grid does not suit the two-level path");
    Workspace &w = ctx->ws;
    w.bcap_r = std::max<unsigned long long>(w.bcap_r, (unsigned long long)nR + nR / 8 + 1024);
    w.bcap_s = std::max<unsigned long long>(w.bcap_s, (unsigned long long)nS + nS / 8 + 1024);
    Stats stats;
    for (int attempt = 0; attempt < 3; attempt++) {
        if ((st = size_blocked(ctx, w, p)) || (st = size_learned(ctx, w, p))) return st;
        BArgs a = blocked_args(w, p, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd);
        a.feat_raw = (unsigned *)w.bFeatRaw.p;
        if (ctx->shared_cursors) a.cur = (unsigned *)w.bCur.p;
        cudaError_t e;
        if ((e = cudaMemsetAsync(w.bFeatRaw.p, 0, 4ull * kRawPerBlock * p.nb, ctx->stream)))
            return cuda_fail(ctx, e, "memset");
        if ((st = enqueue_blocked_partition(ctx, w, p, a))) return st;
        {
            PhaseScope ph(ctx, PH_MODEL, 2);
            if ((e = launch_bfeat_sample(a, ctx->num_sms * 4, ctx->stream))) return cuda_fail(ctx, e, "sampling");
            if ((e = launch_features((const unsigned *)w.bFeatRaw.p, a.items, a.btot, p.nb, a.st,
                                     (float *)w.bFeat.p, ctx->num_sms * 2, ctx->stream)))
                return cuda_fail(ctx, e, "features");
        }
        {
            PhaseScope ph(ctx, PH_SWEEP_COUNT, 1);
            if ((e = launch_bjoin(MODE_COUNT, a, bjoin_out(w, 0), ctx->num_sms * ctx->bjoin_bps, ctx->stream)))
                return cuda_fail(ctx, e, "block join kernel");
        }
        {
            PhaseScope ph(ctx, PH_MODEL, 1);
            if ((e = launch_labels((const unsigned *)w.bPc.p, a.st, (float *)w.bPred.p, ctx->num_sms * 2,
                                   ctx->stream)))
                return cuda_fail(ctx, e, "labels");
        }
        if ((st = read_stats(ctx, w, &stats))) return st;
        if (stats.err & kErrBadRect) return fail(ctx, SJ_EINVAL, "invalid rectangle");
        if (stats.err & kErrEntCap) {
            w.bcap_r = std::max<unsigned long long>(w.bcap_r, stats.e_r + stats.e_r / 8 + 1024);
            w.bcap_s = std::max<unsigned long long>(w.bcap_s, stats.e_s + stats.e_s / 8 + 1024);
            continue;
        }
        if (stats.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
        const int64_t n = stats.nchunks;
        if (stats.need_direct) {
            // a tile exceeds shared memory: the blocks' features stand, and
            // their labels come from the per-tile pair counts of the
            // single-level path, added up per block
            const long long T = (long long)gd.nx * gd.ny;
            if ((st = ensure(ctx, w.tpairs, 4ull * T + 16)) || (st = ensure(ctx, w.item_of, 4ull * p.nb + 16)) ||
                (st = ensure(ctx, w.cnt64, 8ull * (n + 1))))
                return st;
            Stats s2;
            if ((st = partition_and_count(ctx, w, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd, &s2, false)))
                return st;
            if ((e = cudaMemsetAsync(w.tpairs.p, 0, 4ull * T, ctx->stream)) ||
                (e = cudaMemsetAsync(w.item_of.p, 0xff, 4ull * p.nb, ctx->stream)) ||
                (e = cudaMemsetAsync(w.cnt64.p, 0, 8ull * (n + 1), ctx->stream)))
                return cuda_fail(ctx, e, "memset");
            if ((st = enqueue_sweep(ctx, w, MODE_TILES, nullptr, 0, nullptr, (unsigned *)w.tpairs.p, 4))) return st;
            {
                PhaseScope ph(ctx, PH_MODEL, 3);
                if ((e = launch_labels_from_tiles((const unsigned *)w.bItems.p, (unsigned)n, (unsigned *)w.item_of.p,
                                                  (const unsigned *)w.tpairs.p, gd.nx, T, p.G, p.bx,
                                                  (unsigned long long *)w.cnt64.p, (float *)w.bPred.p,
                                                  ctx->num_sms * 4, ctx->stream)))
                    return cuda_fail(ctx, e, "labels");
            }
            if ((st = read_stats(ctx, w, &s2))) return st;
            if (s2.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", s2.err);
        }
        *n_items = n;
        ctx->last = sj_stats{};
        ctx->last.path = 1;
        ctx->last.block_side = p.G;
        ctx->last.blocks = p.nb;
        ctx->last.work_items = n;
        ctx->last.l1_entries_r = (int64_t)stats.e_r;
        ctx->last.l1_entries_s = (int64_t)stats.e_s;
        if (n > cap) return fail(ctx, SJ_EOVERFLOW, "need %lld rows, cap %lld", (long long)n, (long long)cap);
        if (n && (!d_feat || !d_label)) return fail(ctx, SJ_EINVAL, "null output");
        if (n && ((e = cudaMemcpyAsync(d_feat, w.bFeat.p, 4ull * kFeat * n, cudaMemcpyDeviceToDevice, ctx->stream)) ||
                  (e = cudaMemcpyAsync(d_label, w.bPred.p, 4ull * n, cudaMemcpyDeviceToDevice, ctx->stream)) ||
                  (d_block &&
                   (e = cudaMemcpyAsync(d_block, w.bItems.p, 4ull * n, cudaMemcpyDeviceToDevice, ctx->stream)))))
            return cuda_fail(ctx, e, "copy");
        return SJ_OK;
    }
    return fail(ctx, SJ_EINTERNAL, "workspace did not converge");
}

// Features of every work item from the sampled histograms, the predicted
// pairs (the model, or the Eq. 2 estimate), the capacity plan and the
// heaviest-first order, for nb blocks (one join or a whole batch); the
// capacity total lands in w.bCapTot.
int sj::enqueue_prediction(sj_ctx *ctx, Workspace &w, int nb, const BArgs &a, int heuristic, float margin,
                           unsigned slack) {
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    if ((e = launch_features((const unsigned *)w.bFeatRaw.p, a.items, a.btot, nb, a.st, (float *)w.bFeat.p,
                             ctx->num_sms * 8, s)))
        return cuda_fail(ctx, e, "features");
    if (heuristic)
        e = launch_heur_pred((const float *)w.bFeat.p, a.items, a.btot, nb, a.st, (float *)w.bPred.p,
                             ctx->num_sms * 2, s);
    else
        e = launch_mlp_forward(weights_of(ctx->model), (const float *)w.bFeat.p, 0, &a.st->nchunks,
                               (float *)w.bPred.p, mlp_infer_grid(ctx, nb), s);
    if (e) return cuda_fail(ctx, e, "prediction");
    if ((e = zero_async(ctx, w.bCapTot.p, kPlanScratch)) ||
        (e = launch_plan((const float *)w.bPred.p, a.imeta, a.ins, a.st, margin, slack,
                         (unsigned long long *)w.bCapTot.p, (unsigned *)w.bOrder.p, ctx->num_sms, s)))
        return cuda_fail(ctx, e, "plan");
    return SJ_OK;
}

// ---------------------------------------------------------------------------
// the one-pass join
// ---------------------------------------------------------------------------
// Upward-only calibration of the one-pass capacity.  Blocks reserve their
// ranges heaviest first until the planned total is used up; every block after
// that is re-run exactly.  So only the predicted total matters, and a model
// that meets data unlike its training joins (the squares of the distance
// join have other extents than the rectangles it learned from) under-sizes
// every call the same way.  When a join finds more pairs than its plan held,
// later joins on this context scale their capacities by the shortfall (plus
// 10 %); when the plan holds more than twice the pairs, the factor decays
// back towards 1.  Bounded to [1, 8], so that one odd join (or a model that
// predicts nothing) cannot inflate later buffers without limit.  Exactness
// never depends on it.
void sj::calibrate_capacity(sj_ctx *ctx, unsigned long long P, unsigned long long planned) {
    const double c = (double)std::max<unsigned long long>(planned, 1);
    double f = ctx->onepass_scale;
    if ((double)P > c) f *= 1.1 * (double)P / c;
    else if (f > 1.0 && 2.0 * (double)P < c) f *= 1.5 * (double)P / c;
    ctx->onepass_scale = (float)std::min(8.0, std::max(1.0, f));
}

// Partition (with sampled features) -> predict every block's pairs (model,
// or the Eq. 2 estimate) -> capacity = sum of ceil(pred * (1 + margin)) + slack,
// heaviest-first order -> (copy of the capacity to the host overlaps the L1
// write) -> one fused pass that counts each block in shared memory, reserves
// its range with one atomic and writes it if it fits.  Blocks that do not
// fit are re-run exactly into a buffer of the exact size (all reserved ranges
// are known by then).
int sj::join_one_pass_spec(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S, long long nS,
                           const GridDev &gd, const sj_opts *o, int heuristic, OutSpec &os, int64_t *npairs,
                           sj_pair **lib_out) {
    if (!heuristic && !ctx->model) return fail(ctx, SJ_EINVAL, "SJ_ONE_PASS needs a model (sj_set_model)");
    BPlan p;
    if (!plan_blocked(ctx, gd, nR, nS, p)) return ONE_PASS_UNSUITED;
    // capacity of a block = ceil(pred * (1 + margin) * calibration) + slack
    const float margin = (o ? 1.0f + o->margin : 1.25f) * ctx->onepass_scale - 1.0f;
    const unsigned slack = 2;
    w.bcap_r = std::max<unsigned long long>(w.bcap_r, (unsigned long long)nR + nR / 8 + 1024);
    w.bcap_s = std::max<unsigned long long>(w.bcap_s, (unsigned long long)nS + nS / 8 + 1024);
    cudaStream_t s = ctx->stream;
    for (int attempt = 0; attempt < 3; attempt++) {
        int st;
        if ((st = size_blocked(ctx, w, p)) || (st = size_learned(ctx, w, p))) return st;
        BArgs a = blocked_args(w, p, R, nR, S, nS, gd);
        a.feat_raw = (unsigned *)w.bFeatRaw.p;
        a.stop_direct = 1;
        if (ctx->shared_cursors) a.cur = (unsigned *)w.bCur.p;
        a.adaptive = o && (o->flags & SJ_SWEEP_ADAPTIVE);
        a.gbda = o && (o->flags & SJ_DEDUP_GBDA);
        cudaError_t e;
        {
            PhaseScope ph(ctx, PH_RESET, 0);
            if ((e = zero_async(ctx, w.stats.p, sizeof(Stats))) ||
                (e = zero_async(ctx, w.bFeatRaw.p, 4ull * kRawPerBlock * p.nb)))
                return cuda_fail(ctx, e, "memset");
        }
        if ((st = upload_single_join(ctx, w, a))) return st;
        {
            PhaseScope ph(ctx, PH_COUNT, 1);
            if ((e = launch_bcount(a, p.nc, s))) return cuda_fail(ctx, e, "block count kernel");
        }
        {
            PhaseScope ph(ctx, PH_SCAN, 2);
            if ((e = launch_bscan(a, p.nc, s))) return cuda_fail(ctx, e, "block scan kernels");
        }
        unsigned long long *d_cap = (unsigned long long *)w.bCapTot.p;
        {
            PhaseScope ph(ctx, PH_MODEL, 5);
            if ((e = launch_bfeat_sample(a, ctx->num_sms * 4, s))) return cuda_fail(ctx, e, "sampling");
            if ((e = launch_features((const unsigned *)w.bFeatRaw.p, a.items, a.btot, p.nb, a.st, (float *)w.bFeat.p,
                                     ctx->num_sms * 8, s)))
                return cuda_fail(ctx, e, "features");
            if (heuristic) {
                e = launch_heur_pred((const float *)w.bFeat.p, a.items, a.btot, p.nb, a.st, (float *)w.bPred.p,
                                     ctx->num_sms * 2, s);
            } else {
                e = launch_mlp_forward(weights_of(ctx->model), (const float *)w.bFeat.p, 0, &a.st->nchunks,
                                       (float *)w.bPred.p, mlp_infer_grid(ctx, p.nb), s);
            }
            if (e) return cuda_fail(ctx, e, "prediction");
            if ((e = zero_async(ctx, d_cap, kPlanScratch)) ||
                (e = launch_plan((const float *)w.bPred.p, a.imeta, a.ins, a.st, margin, slack, d_cap,
                                 (unsigned *)w.bOrder.p, ctx->num_sms, s)))
                return cuda_fail(ctx, e, "plan");
            if ((e = copy_async(ctx, ctx->h_aux, d_cap, 8)) ||
                (e = cudaEventRecord(ctx->ev_aux, s)))
                return cuda_fail(ctx, e, "capacity copy");
        }
        {
            PhaseScope ph(ctx, PH_SCATTER, 1);
            if ((e = launch_bscatter(a, p.nc, s))) return cuda_fail(ctx, e, "block write kernel");
        }
        // the capacity reached the host while the write kernel runs
        if ((e = cudaEventSynchronize(ctx->ev_aux))) return cuda_fail(ctx, e, "event sync");
        unsigned long long C = *(volatile unsigned long long *)ctx->h_aux;
        const unsigned long long planned = C;
        if (os.kind == OutSpec::INTO) {
            C = (unsigned long long)os.cap;
            os.got = (int2 *)os.into;
            if (C && !os.got) return fail(ctx, SJ_EINVAL, "null output buffer");
        } else {
            if (C < 1024) C = 1024;
            os.got = nullptr;
            if ((st = out_acquire(ctx, w, os, C))) return st;
        }
        BJoinOut bo = bjoin_out(w, 2);
        bo.list = ctx->lpt ? (const unsigned *)w.bOrder.p : nullptr;   // heaviest first, or item order
        bo.list_n = &a.st->nchunks;
        bo.out = os.got;
        bo.cap = C;
        {
            PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
            if ((e = launch_bjoin(MODE_RESERVE, a, bo, ctx->num_sms * ctx->bjoin_bps, s))) {
                out_abandon(ctx, os);
                return cuda_fail(ctx, e, "block join kernel");
            }
        }
        Stats stats;
        if ((st = read_stats(ctx, w, &stats))) {
            out_abandon(ctx, os);
            return st;
        }
        if (stats.err & kErrBadRect) {
            out_abandon(ctx, os);
            return fail(ctx, SJ_EINVAL, "invalid rectangle: NaN/Inf coordinate or xl > xu / yl > yu");
        }
        if (stats.err & kErrEntCap) {
            out_abandon(ctx, os);
            w.bcap_r = std::max<unsigned long long>(w.bcap_r, stats.e_r + stats.e_r / 8 + 1024);
            w.bcap_s = std::max<unsigned long long>(w.bcap_s, stats.e_s + stats.e_s / 8 + 1024);
            continue;
        }
        if (stats.err & kErrTimeout) {
            out_abandon(ctx, os);
            return fail(ctx, SJ_ETIMEOUT, "a device-side wait gave up");
        }
        if (stats.err) {
            out_abandon(ctx, os);
            return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
        }
        if (stats.need_direct) {
            out_abandon(ctx, os);
            return ONE_PASS_DIRECT;
        }
        const unsigned long long P = stats.npairs;
        *npairs = (int64_t)P;
        calibrate_capacity(ctx, P, planned);
        ctx->last = sj_stats{};
        ctx->last.path = 1;
        ctx->last.block_side = p.G;
        ctx->last.blocks = p.nb;
        ctx->last.work_items = stats.nchunks;
        ctx->last.l1_entries_r = (int64_t)stats.e_r;
        ctx->last.l1_entries_s = (int64_t)stats.e_s;
        ctx->last.npairs = (int64_t)P;
        ctx->last.one_pass = 1;
        ctx->last.capacity = (int64_t)C;
        ctx->last.refit_items = stats.nfail;
        ctx->last.y_sweep_tiles = a.adaptive ? (int64_t)stats.naxis_y : 0;
        ctx->last.dedup = a.gbda ? 1 : 0;
        if (os.kind == OutSpec::INTO && P > C)
            return fail(ctx, SJ_EOVERFLOW, "need %llu pairs, cap %llu", P, C);
        if (stats.nfail) {
            // exact re-run of the blocks that did not fit, at their reserved offsets
            OutSpec big = os;
            big.got = nullptr;
            Buf keep = w.out;   // WS: the first buffer must stay alive while copied
            if (os.kind == OutSpec::WS) w.out = Buf{};
            if ((st = out_acquire(ctx, w, big, P))) {
                if (os.kind == OutSpec::WS) {
                    dev_free(ctx, w.out.p);
                    w.out = keep;
                }
                out_abandon(ctx, os);
                return st;
            }
            if ((e = cudaMemcpyAsync(big.got, os.got, 8ull * std::min<unsigned long long>(C, P),
                                     cudaMemcpyDeviceToDevice, s)))
                return cuda_fail(ctx, e, "copy");
            if (os.kind == OutSpec::WS) dev_free(ctx, keep.p);
            else out_abandon(ctx, os);
            os.got = big.got;
            BJoinOut fo = bjoin_out(w, 3);
            fo.list = (const unsigned *)w.bFail.p;
            fo.list_n = &a.st->nfail;
            fo.off_in = (const unsigned long long *)w.bResv.p;
            fo.out = os.got;
            fo.cap = P;
            PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
            if ((e = launch_bjoin(MODE_WRITE, a, fo, ctx->num_sms * ctx->bjoin_bps, s))) {
                out_abandon(ctx, os);
                return cuda_fail(ctx, e, "block join kernel");
            }
        }
        if (o && o->sort_output && P && (st = sort_pairs(ctx, w, os.got, P))) {
            out_abandon(ctx, os);
            return st;
        }
        if (lib_out) *lib_out = (sj_pair *)os.got;
        return SJ_OK;
    }
    return fail(ctx, SJ_EINTERNAL, "workspace did not converge");
}
