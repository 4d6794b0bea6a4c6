// api_batch.cu -- many independent joins in one pass of the two-level
// kernels (sj_join_batch): every join keeps its own grid and blocks; all
// blocks share one index space, so one count, one scan, one write and one
// persistent block-join launch serve the whole batch.  Each phase is
// captured once into a CUDA graph on the context's internal stream and
// replayed while the arguments do not change.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sj_internal.h"
#include "sj_learned.h"

using namespace sj;

namespace {

struct GraphCache {
    unsigned long long key = 0;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;   // kernels of this library in the graph
};

unsigned long long fnv(unsigned long long h, const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; i++) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

struct sj_batch_state {
    cudaStream_t gs = nullptr;          // internal stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    GraphCache g1, g2;
    unsigned long long grid_key = 0;    // inputs of the last rule-of-thumb grids
    std::vector<sj_grid> grids;
};

static int batch_state(sj_ctx *ctx, sj_batch_state **out) {
    if (!ctx->batch) {
        sj_batch_state *b = new (std::nothrow) sj_batch_state();
        if (!b) return fail(ctx, SJ_ENOMEM, "host allocation");
        if (cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return fail(ctx, SJ_ECUDA, "stream / event creation");
        }
        ctx->batch = b;
    }
    *out = ctx->batch;
    return SJ_OK;
}

void sj::batch_release(sj_ctx *ctx) {
    sj_batch_state *b = ctx->batch;
    if (!b) return;
    cudaStreamSynchronize(b->gs);
    if (b->g1.exec) cudaGraphExecDestroy(b->g1.exec);
    if (b->g2.exec) cudaGraphExecDestroy(b->g2.exec);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
    cudaStreamDestroy(b->gs);
    delete b;
    ctx->batch = nullptr;
}

// Run `body` on the internal stream as a graph cached under `key`.
template <typename F>
static int run_graph(sj_ctx *ctx, sj_batch_state *b, GraphCache &gc, unsigned long long key, F body) {
    // without graphs: the same kernels launched directly on the caller's
    // stream (their phases can then be timed)
    if (!ctx->batch_graphs) return body();
    cudaError_t e;
    if (!(gc.exec && gc.key == key)) {
        if (gc.exec) {
            cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
        }
        cudaStream_t user = ctx->stream;
        const bool timer = ctx->timer.on;
        const long long launches0 = ctx->launches;
        ctx->stream = b->gs;
        ctx->timer.on = false;   // no timing events inside a captured graph
        if ((e = cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal))) {
            ctx->stream = user;
            ctx->timer.on = timer;
            return cuda_fail(ctx, e, "graph capture");
        }
        int st = body();
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->gs, &graph);
        ctx->stream = user;
        ctx->timer.on = timer;
        gc.kernels = ctx->launches - launches0;
        ctx->launches = launches0;   // counted when the graph runs
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e) return cuda_fail(ctx, e, "graph capture");
        e = cudaGraphInstantiate(&gc.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e) {
            gc.exec = nullptr;
            return cuda_fail(ctx, e, "graph instantiate");
        }
        gc.key = key;
    }
    ctx->launches += gc.kernels;
    // order after the caller's stream, run, and make the caller's stream wait
    if ((e = cudaEventRecord(b->ev_in, ctx->stream)) || (e = cudaStreamWaitEvent(b->gs, b->ev_in, 0)) ||
        (e = cudaGraphLaunch(gc.exec, b->gs)) || (e = cudaEventRecord(b->ev_out, b->gs)) ||
        (e = cudaStreamWaitEvent(ctx->stream, b->ev_out, 0)))
        return cuda_fail(ctx, e, "graph launch");
    return SJ_OK;
}

// Grid of every join by the rule of Sec. 4.3 (tile extent about ten times
// the average rectangle extent) over the unit square.
static int rule_grids(sj_ctx *ctx, Workspace &w, std::vector<JoinDesc> &jd, std::vector<sj_grid> &grids) {
    const int nj = (int)jd.size();
    int st;
    if ((st = upload_joins(ctx, w, jd.data(), nj))) return st;
    if ((st = ensure(ctx, w.bJoff, 32ull * (nj + 1)))) return st;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.bJoff.p, 0, 32ull * nj, ctx->stream))) return cuda_fail(ctx, e, "memset");
    BArgs a;
    memset(&a, 0, sizeof a);
    a.jd = (const JoinDesc *)w.bJd.p;
    a.nj = nj;
    {
        PhaseScope ph(ctx, PH_OTHER, 1);
        if ((e = launch_extent_stats(a, (double *)w.bJoff.p, ctx->num_sms * 8, ctx->stream)))
            return cuda_fail(ctx, e, "extent statistics");
    }
    std::vector<double> sums(4ull * nj);
    if ((e = cudaMemcpyAsync(sums.data(), w.bJoff.p, 32ull * nj, cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "extent statistics copy");
    for (int j = 0; j < nj; j++) {
        const double n = 2.0 * (double)(jd[j].nR + jd[j].nS);
        const double mean = n > 0 ? (sums[4 * j] + sums[4 * j + 1] + sums[4 * j + 2] + sums[4 * j + 3]) / n : 1e-3;
        double k = mean > 0 ? 1.0 / (10.0 * mean) : 4096.0;
        k = std::min(4096.0, std::max(1.0, floor(k + 0.5)));
        grids[j] = sj_grid{(int32_t)k, (int32_t)k, 0.0f, 0.0f, 1.0f, 1.0f};
    }
    return SJ_OK;
}

// The batch in one pass: the join-aware Eq. 2 sample of every block, the
// predicted pairs (model or Eq. 2), the capacity plan and heaviest-first
// order over all joins' blocks, one reserve-and-write block-join launch into
// a workspace buffer, an exact re-run of the blocks that did not fit, and a
// regroup of every block's pairs into its join's range of d_out (blocks of a
// join are consecutive work items, so the scan of the per-item counts in item
// order gives every block's place).  Direct launches, no graphs: the
// capacity is read back between the phases.  Returns BATCH_TWO_PASS when a
// tile exceeds shared memory (the caller then runs the exact two-pass batch).
constexpr int BATCH_TWO_PASS = -4;

static int batch_one_pass(sj_ctx *ctx, std::vector<JoinDesc> &jd, int nbt, long long tot_r, long long tot_s,
                          const sj_opts *o, int heuristic, sj_pair *d_out, int64_t cap, int64_t *h_offsets) {
    Workspace &w = ctx->ws;
    const int nj = (int)jd.size();
    long long nsamp = 0;
    for (int j = 0; j < nj; j++) {
        jd[j].samp_off = nsamp;
        nsamp += (jd[j].nR + kPhi - 1) / kPhi + (jd[j].nS + kPhi - 1) / kPhi;
    }
    const float margin = (o ? 1.0f + o->margin : 1.25f) * ctx->onepass_scale - 1.0f;
    w.bcap_r = std::max<unsigned long long>(w.bcap_r, (unsigned long long)tot_r + tot_r / 8 + 1024);
    w.bcap_s = std::max<unsigned long long>(w.bcap_s, (unsigned long long)tot_s + tot_s / 8 + 1024);
    cudaStream_t s = ctx->stream;
    for (int attempt = 0; attempt < 3; attempt++) {
        BPlan p;
        p.nb = nbt;
        p.nc = 1;
        p.G = 1;
        p.bx = nbt;
        p.by = 1;
        int st;
        if ((st = size_blocked(ctx, w, p)) || (st = size_learned(ctx, w, p)) ||
            (st = upload_joins(ctx, w, jd.data(), nj)) || (st = ensure(ctx, w.bIjoin, 4ull * (nbt + 1))) ||
            (st = ensure(ctx, w.bJfirst, 4ull * (nj + 1))) || (st = ensure(ctx, w.bJoff, 32ull * (nj + 1))) ||
            (st = ensure(ctx, w.dstats, 2 * sizeof(Stats))))
            return st;
        BArgs a;
        memset(&a, 0, sizeof a);
        a.nb = nbt;
        a.nbt = nbt;
        a.nj = nj;
        a.jd = (const JoinDesc *)w.bJd.p;
        a.btot = (unsigned *)w.bTot.p;
        a.bo_r = (unsigned *)w.bBoR.p;
        a.bo_s = (unsigned *)w.bBoS.p;
        a.items = (unsigned *)w.bItems.p;
        a.imeta = (uint4 *)w.bImeta.p;
        a.ins = (unsigned *)w.bIns.p;
        a.ijoin = (unsigned *)w.bIjoin.p;
        a.jfirst = (unsigned *)w.bJfirst.p;
        a.bent_r = (BEnt *)w.bEntR.p;
        a.bent_s = (BEnt *)w.bEntS.p;
        a.cap_r = w.bcap_r;
        a.cap_s = w.bcap_s;
        a.cur = (unsigned *)w.bCur.p;
        a.lpool = (unsigned *)w.bList.p;
        a.lpool_cap = list_pool_cap(w);
        a.scan_part = (unsigned long long *)w.bScanPart.p;
        a.feat_raw = (unsigned *)w.bFeatRaw.p;
        a.fine_cap = kFineCap;
        a.adaptive = o && (o->flags & SJ_SWEEP_ADAPTIVE);
        a.gbda = o && (o->flags & SJ_DEDUP_GBDA);
        a.st = (Stats *)w.stats.p;
        cudaError_t e;
        {
            PhaseScope ph(ctx, PH_RESET, 0);
            if ((e = zero_async(ctx, w.stats.p, sizeof(Stats))) || (e = zero_async(ctx, w.bTot.p, 8ull * nbt)) ||
                (e = zero_async(ctx, w.bPc.p, 4ull * (nbt + 1))) ||
                (e = zero_async(ctx, w.bFeatRaw.p, 4ull * kRawPerBlock * nbt)))
                return cuda_fail(ctx, e, "memset");
        }
        {
            PhaseScope ph(ctx, PH_COUNT, 1);
            e = ctx->batch_count_local ? launch_bcount_local(a, ctx->num_sms * 2, s)
                                       : launch_bcount_global(a, ctx->num_sms * 8, s);
            if (e) return cuda_fail(ctx, e, "batch count");
        }
        {
            PhaseScope ph(ctx, PH_SCAN, 1);
            if ((e = launch_bscan_blocks_only(a, s))) return cuda_fail(ctx, e, "batch scan");
        }
        {
            PhaseScope ph(ctx, PH_MODEL, 1);
            if ((e = launch_bfeat_sample_batch(a, nsamp, ctx->num_sms * 4, s))) return cuda_fail(ctx, e, "sampling");
        }
        {
            PhaseScope ph(ctx, PH_MODEL, 4);
            if ((st = enqueue_prediction(ctx, w, nbt, a, heuristic, margin, 2))) return st;
            if ((e = copy_async(ctx, ctx->h_aux, w.bCapTot.p, 8)) || (e = cudaEventRecord(ctx->ev_aux, s)))
                return cuda_fail(ctx, e, "capacity copy");
        }
        {
            PhaseScope ph(ctx, PH_SCATTER, 1);
            if ((e = launch_bscatter(a, ctx->num_sms, s))) return cuda_fail(ctx, e, "batch write");
        }
        if ((e = cudaEventSynchronize(ctx->ev_aux))) return cuda_fail(ctx, e, "event sync");
        const unsigned long long planned = *(volatile unsigned long long *)ctx->h_aux;
        const unsigned long long C = std::max<unsigned long long>(planned, 1024ull);
        if ((st = ensure(ctx, w.out, 8ull * C))) return st;
        BJoinOut bo = bjoin_out(w, 2);
        bo.list = ctx->lpt ? (const unsigned *)w.bOrder.p : nullptr;
        bo.list_n = &a.st->nchunks;
        bo.out = (int2 *)w.out.p;
        bo.cap = C;
        {
            PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
            if ((e = launch_bjoin(MODE_RESERVE, a, bo, ctx->num_sms * ctx->bjoin_bps, s)))
                return cuda_fail(ctx, e, "batch join");
        }
        Stats stats;
        if ((st = read_stats(ctx, w, &stats))) return st;
        if (stats.err & kErrBadRect) return fail(ctx, SJ_EINVAL, "invalid rectangle in the batch");
        if (stats.err & kErrEntCap) {
            w.bcap_r = std::max<unsigned long long>(w.bcap_r, stats.e_r + stats.e_r / 8 + 1024);
            w.bcap_s = std::max<unsigned long long>(w.bcap_s, stats.e_s + stats.e_s / 8 + 1024);
            continue;
        }
        if (stats.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
        if (stats.need_direct) return BATCH_TWO_PASS;
        const unsigned long long P = stats.npairs;
        calibrate_capacity(ctx, P, planned);
        const int2 *src = (const int2 *)w.out.p;
        Buf big;
        if (stats.nfail) {
            // the blocks that did not fit, exactly, at their reserved offsets
            if ((st = ensure(ctx, big, 8ull * P))) return st;
            if ((e = cudaMemcpyAsync(big.p, w.out.p, 8ull * std::min(C, P), cudaMemcpyDeviceToDevice, s)))
                return cuda_fail(ctx, e, "copy");
            BJoinOut fo = bjoin_out(w, 3);
            fo.list = (const unsigned *)w.bFail.p;
            fo.list_n = &a.st->nfail;
            fo.off_in = (const unsigned long long *)w.bResv.p;
            fo.out = (int2 *)big.p;
            fo.cap = P;
            PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
            if ((e = launch_bjoin(MODE_WRITE, a, fo, ctx->num_sms * ctx->bjoin_bps, s))) {
                dev_free(ctx, big.p);
                return cuda_fail(ctx, e, "batch join");
            }
            src = (const int2 *)big.p;
        }
        // every block's place in item order, every join's offset
        unsigned long long *d_joff = (unsigned long long *)w.bJoff.p;
        {
            PhaseScope ph(ctx, PH_PAIRSCAN, 2);
            if ((e = launch_scan_pairs((const unsigned *)w.bPc.p, (unsigned)nbt, (unsigned long long *)w.bPoff.p,
                                       (Stats *)w.dstats.p, s)) ||
                (e = launch_join_offsets(a, (const unsigned long long *)w.bPoff.p, d_joff, s)))
                return cuda_fail(ctx, e, "pair scan");
        }
        if ((e = cudaMemcpyAsync(ctx->h_joff, d_joff, 8ull * (nj + 1), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s))) {
            if (big.p) dev_free(ctx, big.p);
            return cuda_fail(ctx, e, "copy");
        }
        const unsigned long long *joff = (const unsigned long long *)ctx->h_joff;
        for (int j = 0; j <= nj; j++) h_offsets[j] = (int64_t)joff[j];
        memset(&ctx->last, 0, sizeof ctx->last);
        ctx->last.path = 1;
        ctx->last.blocks = nbt;
        ctx->last.work_items = stats.nchunks;
        ctx->last.l1_entries_r = (int64_t)stats.e_r;
        ctx->last.l1_entries_s = (int64_t)stats.e_s;
        ctx->last.npairs = (int64_t)P;
        ctx->last.one_pass = 1;
        ctx->last.capacity = (int64_t)C;
        ctx->last.refit_items = stats.nfail;
        int rc = SJ_OK;
        if ((unsigned long long)cap < P) {
            rc = fail(ctx, SJ_EOVERFLOW, "need %llu pairs, cap %lld", P, (long long)cap);
        } else if (P && !d_out) {
            rc = fail(ctx, SJ_EINVAL, "null output buffer");
        } else if (P) {
            PhaseScope ph(ctx, PH_OTHER, 1);
            if ((e = launch_regroup((const unsigned *)w.bPc.p, (const unsigned long long *)w.bResv.p,
                                    (const unsigned long long *)w.bPoff.p, &a.st->nchunks, src, (int2 *)d_out,
                                    ctx->num_sms * 8, s)))
                rc = cuda_fail(ctx, e, "regroup");
        }
        if (big.p) dev_free(ctx, big.p);
        return rc;
    }
    return fail(ctx, SJ_EINTERNAL, "batch workspace did not converge");
}

static int join_batch_body(sj_ctx *ctx, int nj, const sj_rect *const *d_R, const int64_t *nR,
                           const sj_rect *const *d_S, const int64_t *nS, const sj_grid *g_in, const sj_opts *o,
                           sj_pair *d_out, int64_t cap, int64_t *h_offsets);

extern "C" int sj_join_batch(sj_ctx *ctx, int nj, const sj_rect *const *d_R, const int64_t *nR,
                             const sj_rect *const *d_S, const int64_t *nS, const sj_grid *g_in,
                             const sj_opts *o, sj_pair *d_out, int64_t cap, int64_t *h_offsets) {
    int st = join_batch_body(ctx, nj, d_R, nR, d_S, nS, g_in, o, d_out, cap, h_offsets);
    if (st == SJ_OK) {
        DeviceGuard dg(ctx->device);
        if (o && o->sort_output) st = sort_pairs_by_join(ctx, ctx->ws, (int2 *)d_out, h_offsets, nR, nj);
        if (st == SJ_OK) st = check_tail(ctx, ctx->ws);
    }
    return st;
}

static int join_batch_body(sj_ctx *ctx, int nj, const sj_rect *const *d_R, const int64_t *nR,
                           const sj_rect *const *d_S, const int64_t *nS, const sj_grid *g_in, const sj_opts *o,
                           sj_pair *d_out, int64_t cap, int64_t *h_offsets) {
    if (!ctx) return SJ_EINVAL;
    if (nj < 1 || nj > kMaxJoins) return fail(ctx, SJ_EINVAL, "1 <= joins <= %d", kMaxJoins);
    if (!d_R || !nR || !d_S || !nS || !h_offsets || cap < 0) return fail(ctx, SJ_EINVAL, "null argument");
    int st = check_opts(ctx, o);
    if (st) return st;
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    Workspace &w = ctx->ws;
    sj_batch_state *bs = nullptr;
    if ((st = batch_state(ctx, &bs))) return st;

    // per-join descriptors: inputs, grids, block plans, offsets
    std::vector<JoinDesc> jd(nj);
    std::vector<sj_grid> grids(nj);
    long long in_off = 0, tot_r = 0, tot_s = 0;
    for (int j = 0; j < nj; j++) {
        memset(&jd[j], 0, sizeof(JoinDesc));
        jd[j].R = (const float4 *)d_R[j];
        jd[j].S = (const float4 *)d_S[j];
        jd[j].nR = nR[j];
        jd[j].nS = nS[j];
        jd[j].in_off = in_off;
        if (nR[j] < 0 || nS[j] < 0 || nR[j] >= SJ_MAX_N || nS[j] >= SJ_MAX_N)
            return fail(ctx, SJ_EINVAL, "join %d: bad sizes", j);
        in_off += nR[j] + nS[j];
        tot_r += nR[j];
        tot_s += nS[j];
    }
    if (g_in) {
        for (int j = 0; j < nj; j++) grids[j] = g_in[j];
    } else {
        // the rule needs a pass over the inputs; the grids of the previous
        // call are reused when it joined the same buffers and sizes (the
        // grid only shapes the partitioning, never the result)
        unsigned long long gk = 1469598103934665603ull;
        gk = fnv(gk, jd.data(), sizeof(JoinDesc) * nj);
        if (bs->grid_key == gk && (int)bs->grids.size() == nj) {
            grids = bs->grids;
        } else {
            if ((st = rule_grids(ctx, w, jd, grids))) return st;
            bs->grid_key = gk;
            bs->grids = grids;
        }
    }
    int nbt = 0;
    for (int j = 0; j < nj; j++) {
        GridDev gd;
        if ((st = check_inputs(ctx, d_R[j], nR[j], d_S[j], nS[j], &grids[j], &gd))) return st;
        if (gd.nx > 65535 || gd.ny > 65535) return fail(ctx, SJ_EINVAL, "join %d: grid too large for batches", j);
        const double est = (double)(nR[j] + nS[j]) * 1.1 + 1.0;
        const double nbtj = std::max(1.0, est / (double)ctx->block_target);
        int G = (int)ceil(sqrt((double)gd.nx * (double)gd.ny / nbtj));
        G = std::max(1, std::min(kMaxG, G));
        jd[j].g = gd;
        jd[j].G = G;
        jd[j].gmul = G > 1 ? (unsigned)(0xFFFFFFFFull / (unsigned long long)G + 1ull) : 0u;
        jd[j].bx = (gd.nx + G - 1) / G;
        jd[j].by = (gd.ny + G - 1) / G;
        jd[j].boff = nbt;
        if ((long long)nbt + (long long)jd[j].bx * jd[j].by > (1ll << 30)) return fail(ctx, SJ_EINVAL, "too many blocks");
        nbt += jd[j].bx * jd[j].by;
    }

    {   // learned (or Eq. 2) one-pass sizing of the whole batch
        const int mode = o ? o->mode : SJ_TWO_PASS;
        const bool one_pass = mode == SJ_ONE_PASS || mode == SJ_ONE_PASS_HEUR || (mode == SJ_AUTO && ctx->mlp_loaded);
        if (mode == SJ_ONE_PASS && !ctx->model) return fail(ctx, SJ_EINVAL, "SJ_ONE_PASS needs a model (sj_set_model)");
        if (one_pass) {
            st = batch_one_pass(ctx, jd, nbt, tot_r, tot_s, o, mode == SJ_ONE_PASS_HEUR ? 1 : 0, d_out, cap,
                                h_offsets);
            if (st != BATCH_TWO_PASS) return st;
        }
    }
    w.bcap_r = std::max<unsigned long long>(w.bcap_r, (unsigned long long)tot_r + tot_r / 8 + 1024);
    w.bcap_s = std::max<unsigned long long>(w.bcap_s, (unsigned long long)tot_s + tot_s / 8 + 1024);
    cudaError_t e;
    for (int attempt = 0; attempt < 3; attempt++) {
        BPlan p;
        p.nb = nbt;
        p.nc = 1;
        p.G = 1;
        p.bx = nbt;
        p.by = 1;
        if ((st = size_blocked(ctx, w, p)) || (st = upload_joins(ctx, w, jd.data(), nj)) ||
            (st = ensure(ctx, w.bIjoin, 4ull * (nbt + 1))) || (st = ensure(ctx, w.bJfirst, 4ull * (nj + 1))) ||
            (st = ensure(ctx, w.bJoff, 32ull * (nj + 1))))
            return st;
        BArgs a;
        memset(&a, 0, sizeof a);
        a.nb = nbt;
        a.nbt = nbt;
        a.nj = nj;
        a.jd = (const JoinDesc *)w.bJd.p;
        a.btot = (unsigned *)w.bTot.p;
        a.bo_r = (unsigned *)w.bBoR.p;
        a.bo_s = (unsigned *)w.bBoS.p;
        a.items = (unsigned *)w.bItems.p;
        a.imeta = (uint4 *)w.bImeta.p;
        a.ins = (unsigned *)w.bIns.p;
        a.ijoin = (unsigned *)w.bIjoin.p;
        a.jfirst = (unsigned *)w.bJfirst.p;
        a.bent_r = (BEnt *)w.bEntR.p;
        a.bent_s = (BEnt *)w.bEntS.p;
        a.cap_r = w.bcap_r;
        a.cap_s = w.bcap_s;
        a.cur = (unsigned *)w.bCur.p;
        a.lpool = (unsigned *)w.bList.p;
        a.lpool_cap = list_pool_cap(w);
        a.scan_part = (unsigned long long *)w.bScanPart.p;
        a.fine_cap = kFineCap;
        a.adaptive = o && (o->flags & SJ_SWEEP_ADAPTIVE);
        a.gbda = o && (o->flags & SJ_DEDUP_GBDA);
        a.st = (Stats *)w.stats.p;
        // the arguments that shape the captured work
        unsigned long long key = 1469598103934665603ull;
        key = fnv(key, jd.data(), sizeof(JoinDesc) * nj);
        key = fnv(key, &a, sizeof a);
        key = fnv(key, &nj, sizeof nj);
        const int grid_l1 = ctx->num_sms * 8;
        const int grid_bj = ctx->num_sms * ctx->bjoin_bps;
        unsigned long long *d_joff = (unsigned long long *)w.bJoff.p;
        st = run_graph(ctx, bs, bs->g1, key, [&]() -> int {
            cudaStream_t s = ctx->stream;
            cudaError_t e2;
            if ((e2 = cudaMemsetAsync(w.stats.p, 0, sizeof(Stats), s)) ||
                (e2 = cudaMemsetAsync(w.bTot.p, 0, 8ull * nbt, s)) ||
                (e2 = cudaMemsetAsync(w.bPc.p, 0, 4ull * (nbt + 1), s)))
                return cuda_fail(ctx, e2, "memset");
            {
                PhaseScope ph(ctx, PH_COUNT, 1);
                e2 = ctx->batch_count_local ? launch_bcount_local(a, ctx->num_sms * 2, s)
                                            : launch_bcount_global(a, grid_l1, s);
                if (e2) return cuda_fail(ctx, e2, "batch count");
            }
            {
                PhaseScope ph(ctx, PH_SCAN, 1);
                if ((e2 = launch_bscan_blocks_only(a, s))) return cuda_fail(ctx, e2, "batch scan");
            }
            {
                PhaseScope ph(ctx, PH_SCATTER, 1);
                if ((e2 = launch_bscatter(a, ctx->num_sms, s))) return cuda_fail(ctx, e2, "batch write");
            }
            {
                PhaseScope ph(ctx, PH_SWEEP_COUNT, 1);
                if ((e2 = launch_bjoin(MODE_COUNT, a, bjoin_out(w, 0), grid_bj, s))) return cuda_fail(ctx, e2, "batch join");
            }
            {
                PhaseScope ph(ctx, PH_PAIRSCAN, 2);
                if ((e2 = launch_scan_pairs((const unsigned *)w.bPc.p, (unsigned)nbt, (unsigned long long *)w.bPoff.p,
                                            (Stats *)w.stats.p, s)))
                    return cuda_fail(ctx, e2, "pair scan");
                if ((e2 = launch_join_offsets(a, (const unsigned long long *)w.bPoff.p, d_joff, s)))
                    return cuda_fail(ctx, e2, "join offsets");
            }
            if ((e2 = cudaMemcpyAsync(ctx->h_stats, w.stats.p, sizeof(Stats), cudaMemcpyDeviceToHost, s)) ||
                (e2 = cudaMemcpyAsync(ctx->h_joff, d_joff, 8ull * (nj + 1), cudaMemcpyDeviceToHost, s)))
                return cuda_fail(ctx, e2, "copy");
            return SJ_OK;
        });
        if (st) return st;
        if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
        Stats stats;
        memcpy(&stats, ctx->h_stats, sizeof stats);
        if (stats.err & kErrBadRect) return fail(ctx, SJ_EINVAL, "invalid rectangle in the batch");
        if (stats.err & kErrEntCap) {
            w.bcap_r = std::max<unsigned long long>(w.bcap_r, stats.e_r + stats.e_r / 8 + 1024);
            w.bcap_s = std::max<unsigned long long>(w.bcap_s, stats.e_s + stats.e_s / 8 + 1024);
            continue;
        }
        if (stats.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
        const unsigned long long *joff = (const unsigned long long *)ctx->h_joff;
        for (int j = 0; j <= nj; j++) h_offsets[j] = (int64_t)joff[j];
        const unsigned long long P = stats.npairs;
        memset(&ctx->last, 0, sizeof ctx->last);
        ctx->last.path = 1;
        ctx->last.blocks = nbt;
        ctx->last.work_items = stats.nchunks;
        ctx->last.l1_entries_r = (int64_t)stats.e_r;
        ctx->last.l1_entries_s = (int64_t)stats.e_s;
        ctx->last.npairs = (int64_t)P;
        if (stats.need_direct) {
            // a tile of some join exceeds shared memory: count and join each one
            // exactly on its own (the blocked counts skipped that join's block)
            h_offsets[0] = 0;
            for (int j = 0; j < nj; j++) {
                int64_t n = 0;
                if ((st = sj_count(ctx, d_R[j], nR[j], d_S[j], nS[j], &grids[j], &n))) return st;
                h_offsets[j + 1] = h_offsets[j] + n;
            }
            if (cap < h_offsets[nj])
                return fail(ctx, SJ_EOVERFLOW, "need %lld pairs, cap %lld", (long long)h_offsets[nj], (long long)cap);
            sj_opts each{SJ_TWO_PASS, 0, 0.25f, o ? o->flags : 0};   // the batch's sweep options, exact
            for (int j = 0; j < nj; j++) {
                int64_t n = 0;
                if (h_offsets[j + 1] == h_offsets[j]) continue;
                if ((st = sj_join_into(ctx, d_R[j], nR[j], d_S[j], nS[j], &grids[j], &each, d_out + h_offsets[j],
                                       h_offsets[j + 1] - h_offsets[j], &n)))
                    return st;
            }
            ctx->last.npairs = h_offsets[nj];
            return SJ_OK;
        }
        if ((unsigned long long)cap < P) return fail(ctx, SJ_EOVERFLOW, "need %llu pairs, cap %lld", P, (long long)cap);
        if (P == 0) return SJ_OK;
        if (!d_out) return fail(ctx, SJ_EINVAL, "null output buffer");
        unsigned long long key2 = fnv(key, &d_out, sizeof d_out);
        key2 = fnv(key2, &P, sizeof P);
        return run_graph(ctx, bs, bs->g2, key2, [&]() -> int {
            BJoinOut bo = bjoin_out(w, 1);
            bo.out = (int2 *)d_out;
            bo.cap = P;
            PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
            cudaError_t e2 = launch_bjoin(MODE_WRITE, a, bo, grid_bj, ctx->stream);
            return e2 ? cuda_fail(ctx, e2, "batch join") : SJ_OK;
        });
    }
    return fail(ctx, SJ_EINTERNAL, "batch workspace did not converge");
}

extern "C" int sj_extent_stats(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                               double *out) {
    if (!ctx || !out) return SJ_EINVAL;
    if (nR < 0 || nS < 0 || (nR && !d_R) || (nS && !d_S)) return fail(ctx, SJ_EINVAL, "bad inputs");
    DeviceGuard dg(ctx->device);
    std::vector<JoinDesc> jd(1);
    memset(jd.data(), 0, sizeof(JoinDesc));
    jd[0].R = (const float4 *)d_R;
    jd[0].S = (const float4 *)d_S;
    jd[0].nR = nR;
    jd[0].nS = nS;
    std::vector<sj_grid> g(1);
    Workspace &w = ctx->ws;
    int st = ensure(ctx, w.bJoff, 64);
    if (st) return st;
    // reuse the grid rule's reduction and read back its sums
    if ((st = upload_joins(ctx, w, jd.data(), 1))) return st;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.bJoff.p, 0, 32, ctx->stream))) return cuda_fail(ctx, e, "memset");
    BArgs a;
    memset(&a, 0, sizeof a);
    a.jd = (const JoinDesc *)w.bJd.p;
    a.nj = 1;
    {
        PhaseScope ph(ctx, PH_OTHER, 1);
        if ((e = launch_extent_stats(a, (double *)w.bJoff.p, ctx->num_sms * 8, ctx->stream)))
            return cuda_fail(ctx, e, "extent statistics");
    }
    if ((e = cudaMemcpyAsync(out, w.bJoff.p, 32, cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "copy");
    return SJ_OK;
}

extern "C" int sj_set_schedule(sj_ctx *ctx, int heaviest_first) {
    if (!ctx) return SJ_EINVAL;
    ctx->lpt = heaviest_first ? 1 : 0;
    return SJ_OK;
}

extern "C" int sj_set_tuning(sj_ctx *ctx, int block_target) {
    if (!ctx || block_target < 64) return SJ_EINVAL;
    ctx->block_target = block_target;
    return SJ_OK;
}
