// hoststream.cu -- a stream of independent joins from HOST buffers, with the
// host -> device copy of join i+1's inputs overlapping join i.
//
// sj_join_host copies a join's inputs, joins them and copies the pairs back,
// one after the other; on a host link of ~200 GB/s the input copy of a large
// join takes as long as the join itself.  For a sequence of joins the copy
// of the next inputs needs neither the device's compute nor the current
// join's buffers, so it runs on a second (copy) stream into the other of two
// device staging buffers:
//
//   copy stream:    H2D(0) | H2D(1)           | H2D(2)           | ...
//   context stream:        | join(0) D2H(0)   | join(1) D2H(1)   | ...
//
// H2D(i) waits for the event recorded after join(i-2), the last join that
// read its staging buffer; join(i) waits for H2D(i).  The pairs of join i go
// back on the context stream right after it, before join i+1 can overwrite
// the workspace's output buffer.
#include <algorithm>
#include <new>

#include "sj_internal.h"

using namespace sj;

struct sj_hoststream_state {
    cudaStream_t cs = nullptr;   // copy stream
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    Buf in_r[2], in_s[2];        // device staging, ping-pong
};

void sj::hoststream_release(sj_ctx *ctx) {
    sj_hoststream_state *h = ctx->hs;
    if (!h) return;
    if (h->cs) cudaStreamSynchronize(h->cs);
    for (int b = 0; b < 2; b++) {
        dev_free(ctx, h->in_r[b].p);
        dev_free(ctx, h->in_s[b].p);
        if (h->ev_in[b]) cudaEventDestroy(h->ev_in[b]);
        if (h->ev_free[b]) cudaEventDestroy(h->ev_free[b]);
    }
    if (h->cs) cudaStreamDestroy(h->cs);
    delete h;
    ctx->hs = nullptr;
}

static int hoststream_state(sj_ctx *ctx, sj_hoststream_state **out) {
    if (!ctx->hs) {
        sj_hoststream_state *h = new (std::nothrow) sj_hoststream_state;
        if (!h) return fail(ctx, SJ_ENOMEM, "host-stream state");
        ctx->hs = h;
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking))) {
            hoststream_release(ctx);
            return cuda_fail(ctx, e, "copy stream");
        }
        for (int b = 0; b < 2; b++)
            if ((e = cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming)) ||
                (e = cudaEventCreateWithFlags(&h->ev_free[b], cudaEventDisableTiming))) {
                hoststream_release(ctx);
                return cuda_fail(ctx, e, "copy events");
            }
        // nothing has used the staging buffers yet
        for (int b = 0; b < 2; b++)
            if ((e = cudaEventRecord(h->ev_free[b], ctx->stream))) return cuda_fail(ctx, e, "event");
    }
    *out = ctx->hs;
    return SJ_OK;
}

extern "C" int sj_join_host_many(sj_ctx *ctx, int n, const sj_rect *const *h_R, const int64_t *nR,
                                 const sj_rect *const *h_S, const int64_t *nS, const sj_grid *g,
                                 const sj_opts *o, sj_pair *const *h_out, const int64_t *cap, int64_t *npairs) {
    if (!ctx) return SJ_EINVAL;
    if (n < 0 || (n && (!h_R || !nR || !h_S || !nS || !g || !h_out || !cap || !npairs)))
        return fail(ctx, SJ_EINVAL, "null argument array");
    int st;
    if ((st = check_opts(ctx, o))) return st;
    std::vector<GridDev> gd(n > 0 ? n : 1);
    unsigned long long need_r[2] = {16, 16}, need_s[2] = {16, 16};
    for (int i = 0; i < n; i++) {   // every argument is checked before any work
        if (nR[i] < 0 || nS[i] < 0 || nR[i] >= SJ_MAX_N || nS[i] >= SJ_MAX_N)
            return fail(ctx, SJ_EINVAL, "join %d: sizes must satisfy 0 <= n < 2^30", i);
        if ((nR[i] && !h_R[i]) || (nS[i] && !h_S[i])) return fail(ctx, SJ_EINVAL, "join %d: null rectangles", i);
        if (cap[i] < 0 || (cap[i] && !h_out[i])) return fail(ctx, SJ_EINVAL, "join %d: bad output buffer", i);
        if ((st = check_inputs(ctx, nullptr, 0, nullptr, 0, &g[i], &gd[i]))) return st;
        need_r[i & 1] = std::max<unsigned long long>(need_r[i & 1], 16ull * nR[i] + 16);
        need_s[i & 1] = std::max<unsigned long long>(need_s[i & 1], 16ull * nS[i] + 16);
        npairs[i] = 0;
    }
    if (n == 0) return SJ_OK;
    DeviceGuard dg(ctx->device);
    ctx->msg[0] = 0;
    sj_hoststream_state *h;
    if ((st = hoststream_state(ctx, &h))) return st;
    // staging sized for every join up front: no buffer is reallocated while in use
    for (int b = 0; b < 2; b++) {
        if (h->in_r[b].bytes < need_r[b] || h->in_s[b].bytes < need_s[b]) {
            cudaError_t e = cudaStreamSynchronize(h->cs);
            if (e) return cuda_fail(ctx, e, "copy stream sync");
            if ((e = cudaStreamSynchronize(ctx->stream))) return cuda_fail(ctx, e, "stream sync");
        }
        if ((st = ensure(ctx, h->in_r[b], need_r[b])) || (st = ensure(ctx, h->in_s[b], need_s[b]))) return st;
    }
    cudaError_t e;
    // a failed call returns only after both streams are idle, so that no copy
    // still reads or writes the caller's host buffers
    auto drain = [&](int status) {
        cudaStreamSynchronize(h->cs);
        cudaStreamSynchronize(ctx->stream);
        return status;
    };
    auto h2d = [&](int i) -> int {
        const int b = i & 1;
        if ((e = cudaStreamWaitEvent(h->cs, h->ev_free[b], 0))) return cuda_fail(ctx, e, "copy stream wait");
        if (nR[i] && (e = cudaMemcpyAsync(h->in_r[b].p, h_R[i], 16ull * nR[i], cudaMemcpyHostToDevice, h->cs)))
            return cuda_fail(ctx, e, "copy of R to the device");
        if (nS[i] && (e = cudaMemcpyAsync(h->in_s[b].p, h_S[i], 16ull * nS[i], cudaMemcpyHostToDevice, h->cs)))
            return cuda_fail(ctx, e, "copy of S to the device");
        if ((e = cudaEventRecord(h->ev_in[b], h->cs))) return cuda_fail(ctx, e, "copy event");
        return SJ_OK;
    };
    int result = SJ_OK;
    if ((st = h2d(0))) return drain(st);
    for (int i = 0; i < n; i++) {
        const int b = i & 1;
        if (i + 1 < n && (st = h2d(i + 1))) return drain(st);
        if ((e = cudaStreamWaitEvent(ctx->stream, h->ev_in[b], 0))) return drain(cuda_fail(ctx, e, "stream wait"));
        OutSpec os{OutSpec::WS};
        int64_t np = 0;
        st = join_core(ctx, ctx->ws, (const sj_rect *)h->in_r[b].p, nR[i], (const sj_rect *)h->in_s[b].p, nS[i],
                       gd[i], o, os, &np);
        if ((e = cudaEventRecord(h->ev_free[b], ctx->stream))) return drain(cuda_fail(ctx, e, "event"));
        if (st) return drain(st);
        npairs[i] = np;
        if (np > cap[i]) {
            result = SJ_EOVERFLOW;
            continue;
        }
        if (np && (e = cudaMemcpyAsync(h_out[i], os.got, 8ull * np, cudaMemcpyDeviceToHost, ctx->stream)))
            return drain(cuda_fail(ctx, e, "copy of the pairs to the host"));
    }
    if ((e = cudaStreamSynchronize(ctx->stream)) || (e = cudaStreamSynchronize(h->cs)))
        return cuda_fail(ctx, e, "stream sync");
    if (result == SJ_EOVERFLOW) return fail(ctx, SJ_EOVERFLOW, "a join's pairs exceed its output capacity");
    return SJ_OK;
}
