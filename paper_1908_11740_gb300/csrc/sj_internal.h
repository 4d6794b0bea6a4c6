// sj_internal.h -- host-side state of the library (contexts, workspaces) and
// the internal entry points shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sj.h"
#include "sj_blocked.h"
#include "sj_common.cuh"
#include "sj_kernels.h"

namespace sj {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Device workspace of one join (grow-only; reused across calls).
struct Workspace {
    Buf stats, cnt, off, bsum, ts, large;
    Buf ent_r, id_r, ent_s, id_s;
    Buf seg_off, seg_src, seg_vb, hist, key_a, key_b, val_a, val_b, lmbr, lid;
    Buf pc, poff, resv, fail_c, fail_l;
    Buf sort_tmp, ps_hist, ps_part;   // sorted output: ping-pong pairs, digit table, scan parts
    Buf in_r, in_s, out;      // staging of sj_join_host
    // blocked (two-level) path
    Buf bH, bTot, bBoR, bBoS, bItems, bEntR, bEntS, bPc, bPoff, bResv, bFail, bImeta, bIns;
    Buf bFeatRaw, bFeat, bPred, bOrder, bCapTot;   // learned one-pass sizing
    Buf bCur;                                      // shared L1 write cursors
    Buf bList;                                     // row lists of multi-band blocks
    Buf bSpill;                                    // one-pass pair spill per block-join CTA
    Buf bJd, bIjoin, bJfirst, bJoff;               // join table (batches: per-join offsets)
    Buf bScanPart;                                 // block scan: sums per chunk of blocks
    Buf bSortOff;                                  // sorted batch output: pair and R offsets per join
    Buf lstart, lcoff, lvb, ly;                    // candidate-parallel sweep of the large tiles
    Buf st_order;                                  // stripe kernel: every stripe's sorted keys and order
    Buf dsq_r, dsq_s, dmask, dcnt, doff, dstats;   // eps-distance join: squares, refinement
    Buf band_r, band_s, band_ir, band_is;          // row band of a join: its rectangles and their indices
    Buf tpairs, item_of, cnt64;                    // block labels from per-tile pair counts
    unsigned long long bcap_r = 0, bcap_s = 0;
    unsigned long long cap_r = 0, cap_s = 0;   // entry capacities per side
    long long T = 0;
    unsigned nch_cap = 0, nl_cap = 0, vb_cap = 0;
    unsigned long long items_cap = 0;
    // point inputs (the distance join): R, S of the current join are float2
    // points that the two-level kernels read as squares of half-width in_h
    int in_pts = 0;
    float in_h = 0.0f;
};

struct MlpState;   // learned per-tile result-count predictor (mlp.cu)
void batch_release(sj_ctx *ctx);
void hoststream_release(sj_ctx *ctx);

// Phases of a join, for the device-side timing of sj_timing_*.
enum Phase {
    PH_RESET = 0, PH_COUNT, PH_SCAN, PH_SCATTER, PH_LSORT, PH_SWEEP_COUNT, PH_PAIRSCAN,
    PH_SWEEP_WRITE, PH_LSWEEP_COUNT, PH_LSWEEP_WRITE, PH_MODEL, PH_OTHER, PH_REFINE, PH_N
};

struct Timer {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Rec { int phase; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    double ms[PH_N] = {};
    long long n[PH_N] = {};
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int fail(sj_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(sj_ctx *ctx, cudaError_t e, const char *where);
void *dev_alloc(sj_ctx *ctx, size_t bytes);
void dev_free(sj_ctx *ctx, void *p);
int ensure(sj_ctx *ctx, Buf &b, size_t bytes);
void release(sj_ctx *ctx, Workspace &w);
int check_inputs(sj_ctx *ctx, const sj_rect *R, int64_t nR, const sj_rect *S, int64_t nS,
                 const sj_grid *g, GridDev *gd);
int size_workspace(sj_ctx *ctx, Workspace &w, long long T);
LargeArgs large_args(Workspace &w);
SweepArgs sweep_args(Workspace &w);
int enqueue_partition(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S,
                      long long nS, const GridDev &g);
int enqueue_sweep(sj_ctx *ctx, Workspace &w, int mode, int2 *out, unsigned long long cap,
                  const unsigned long long *off_in, unsigned *tile_pairs, int slot_base);
int read_stats(sj_ctx *ctx, Workspace &w, Stats *out);
int check_failed(sj_ctx *ctx, unsigned site);
int check_tail(sj_ctx *ctx, Workspace &w);
int partition_and_count(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S,
                        long long nS, const GridDev &g, Stats *stats, bool count_pass);
struct OutSpec;
// returned by join_one_pass_spec when the grid or the data do not suit the
// two-level path; the caller then runs the exact two-pass join
constexpr int ONE_PASS_UNSUITED = -1;
// ... and when a tile exceeds shared memory (the caller then goes straight to
// the single-level path)
constexpr int ONE_PASS_DIRECT = -5;
// returned by join_core for point inputs when the two-level path does not
// suit the data (the caller then materialises the squares)
constexpr int PTS_UNSUITED = -2;
// returned by join_stripes when the grid is not 1D or a stripe exceeds shared
// memory (the caller then runs the general path)
constexpr int STRIPES_UNSUITED = -3;
int join_stripes(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S, long long nS,
                 const GridDev &gd, const sj_opts *o, OutSpec &os, int64_t *npairs);
int join_one_pass_spec(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S, long long nS,
                       const GridDev &gd, const sj_opts *o, int heuristic, OutSpec &os, int64_t *npairs,
                       sj_pair **lib_out);
int sort_pairs(sj_ctx *ctx, Workspace &w, int2 *pairs, unsigned long long n);
// the pairs of every join of a batch (ranges h_off[j] .. h_off[j + 1]) sorted by (r, s)
int sort_pairs_by_join(sj_ctx *ctx, Workspace &w, int2 *pairs, const int64_t *h_off, const int64_t *nR, int nj);
void mlp_release(sj_ctx *ctx);

// Where the pairs of a join go once their number P is known.
struct OutSpec {
    enum Kind { LIB, INTO, WS } kind;
    sj_pair *into = nullptr;   // INTO: caller buffer
    int64_t cap = 0;           // INTO: its capacity
    int2 *got = nullptr;       // the buffer written
};

struct BPlan {
    int G = 0, bx = 0, by = 0, nb = 0, nc = 0;
};

int out_acquire(sj_ctx *ctx, Workspace &w, OutSpec &os, unsigned long long P);
void out_abandon(sj_ctx *ctx, OutSpec &os);
bool plan_blocked(sj_ctx *ctx, const GridDev &g, long long nR, long long nS, BPlan &p);
int size_blocked(sj_ctx *ctx, Workspace &w, const BPlan &p);
// Entries of the row-list pool: 5/4 of the L1 capacity (a block that finds
// the pool exhausted stages its bands from the whole L1 range instead).
inline unsigned long long list_pool_cap(const Workspace &w) { return (w.bcap_r + w.bcap_s) * 5 / 4 + 1024; }
BArgs blocked_args(Workspace &w, const BPlan &p, const float4 *R, long long nR, const float4 *S, long long nS,
                   const GridDev &g);
BJoinOut bjoin_out(Workspace &w, int slot);
int enqueue_blocked_partition(sj_ctx *ctx, Workspace &w, const BPlan &p, const BArgs &a);
int blocked_partition_count(sj_ctx *ctx, Workspace &w, const BPlan &p, const float4 *R, long long nR,
                            const float4 *S, long long nS, const GridDev &g, Stats *stats, bool *use_direct,
                            int flags, unsigned char *tile_axis = nullptr);
int check_opts(sj_ctx *ctx, const sj_opts *o);
// Learned sizing buffers of nb blocks, and the prediction + capacity plan of
// their work items (features, model or Eq. 2, plan, heaviest-first order).
int size_learned(sj_ctx *ctx, Workspace &w, const BPlan &p);
int enqueue_prediction(sj_ctx *ctx, Workspace &w, int nb, const BArgs &a, int heuristic, float margin,
                       unsigned slack);
// One-pass factor of the capacity calibration of a context (see api_learned.cu).
void calibrate_capacity(sj_ctx *ctx, unsigned long long P, unsigned long long planned);
// The join of sj_join / sj_join_into / sj_join_host on checked inputs.
int join_core(sj_ctx *ctx, Workspace &w, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
              const GridDev &gd, const sj_opts *o, OutSpec &os, int64_t *npairs);
int upload_joins(sj_ctx *ctx, Workspace &w, const JoinDesc *h, int nj);
int upload_single_join(sj_ctx *ctx, Workspace &w, const BArgs &a);

// misc.cu
cudaError_t launch_tile_counts(const uint2 *off, long long T, unsigned *cnt_r, unsigned *cnt_s,
                               cudaStream_t s);
cudaError_t launch_reset_counters(Stats *st, cudaStream_t s);

// timing (api.cu): brackets the launches of one phase with events when on,
// and counts the kernels launched.
struct PhaseScope {
    sj_ctx *ctx;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseScope(sj_ctx *c, int ph, int kernels);
    ~PhaseScope();
};

}  // namespace sj

struct sj_batch_state;
struct sj_hoststream_state;

struct sj_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 1;
    int sweep_bps = 1;
    int bjoin_bps = 1;
    int use_blocked = 1;      // the two-level path when the grid allows it
    int use_stripes = 1;      // the stripe kernel for 1D grids
    int batch_graphs = 1;     // batched joins replay captured CUDA graphs (else direct launches)
    int batch_count_local = 1;   // batch L1 count with per-join shared histograms (else global atomics)
    int shared_cursors = 1;   // L1 write through shared per-block cursors
    int block_target = 1536;  // L1 entries a block should hold (two-level plan)
    int lpt = 1;              // one-pass join: blocks heaviest predicted cost first (else item order)
    float onepass_scale = 1.0f;   // one-pass capacity calibration (api_learned.cu), in [1, 8]
    sj_alloc_fn alloc = nullptr;
    sj_free_fn free_fn = nullptr;
    void *user = nullptr;
    sj::Workspace ws;
    void *h_stats = nullptr;   // pinned copy of sj::Stats
    sj::Timer timer;
    sj_stats last = {};
    long long launches = 0;
    bool mlp_loaded = false;
    const sj_mlp *model = nullptr;      // predictor of SJ_ONE_PASS (not owned)
    void *h_aux = nullptr;              // pinned: one-pass capacity
    void *h_jd = nullptr;               // pinned: join table staging (kMaxJoins)
    void *h_joff = nullptr;             // pinned: per-join pair offsets of a batch
    sj_batch_state *batch = nullptr;    // internal stream and cached graphs of sj_join_batch
    sj_hoststream_state *hs = nullptr;  // copy stream and staging of sj_join_host_many
    cudaEvent_t ev_aux = nullptr;
    char msg[512];
};

namespace sj {
// zero_words_async / copy_words_async on the context's stream, counted among
// the library's kernel launches (sj_timing.launches).
inline cudaError_t zero_async(sj_ctx *ctx, void *p, size_t bytes) {
    if (bytes >= 4) ctx->launches++;
    return zero_words_async(p, bytes, ctx->stream);
}
inline cudaError_t copy_async(sj_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (bytes >= 4) ctx->launches++;
    return copy_words_async(dst, src, bytes, ctx->stream);
}
}  // namespace sj

struct sj_part {
    sj_ctx *ctx = nullptr;
    sj::GridDev grid;
    long long nR = 0, nS = 0;
    unsigned long long e_r = 0, e_s = 0;
    sj::Workspace ws;
};
