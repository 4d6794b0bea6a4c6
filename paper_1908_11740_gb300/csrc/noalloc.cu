// noalloc.cu -- a join entry point that never allocates device memory.
//
// Some callers cannot call cudaMalloc: plug-ins whose host process owns every
// device allocation (a fixed memory budget or a custom pool that nothing may
// bypass), and callers on a latency-critical path that cannot pay an
// allocation's latency or the device-wide synchronisation cudaFree implies.
// sj_join_noalloc runs
// the same two-pass join as sj_join_into, but every scratch buffer it needs
// lives in the file-scope device array below, which the CUDA runtime creates
// when this library's module is loaded on a device and keeps until exit.
//
// Limits (checked before any work, SJ_EINVAL beyond them): at most
// kNaMaxN rectangles per side, kNaMaxTiles tiles, and kNaMaxEnt replicated
// entries per side (detected on the device; then nothing is written and
// SJ_EINVAL is returned).
#define SJ_FILE_CODE 9
#include <mutex>

#include "sj_internal.h"

namespace {

constexpr long long kNaMaxN = 1ll << 16;
constexpr long long kNaMaxTiles = 1ll << 16;
constexpr unsigned long long kNaMaxEnt = 1ull << 17;
constexpr size_t kNaScratchBytes = 20ull << 20;   // 20 MiB per device

// The shared scratch.  In host code this name is only a stand-in, never a
// device address: host code passes the address obtained from
// cudaGetSymbolAddress (per device) to the kernels.
static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

struct NaDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_na_scratch
    int num_sms = 1;
    int sweep_bps = 1;
};

constexpr int kNaMaxDevices = 64;
NaDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mu;

// Once per device, with that device current: resolve the scratch address
// and the launch parameters.
int na_setup(int dev, NaDevice **out) {
    if (dev < 0 || dev >= kNaMaxDevices) return SJ_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mu);
    NaDevice &d = g_na_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SJ_ECUDA;
        }
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return SJ_ECUDA;
        }
        if (sj::sweep_setup() != cudaSuccess) {
            cudaGetLastError();
            return SJ_ECUDA;
        }
        d.sweep_bps = sj::sweep_blocks_per_sm();
        d.scratch = (unsigned char *)p;
        d.ready = true;
    }
    *out = &d;
    return SJ_OK;
}

// Lay the workspace of a join with the limits above over the scratch.
// Returns false if the layout would not fit (a build-time mistake).
bool na_carve(unsigned char *base, long long T, sj::Workspace &w) {
    using sj::Buf;
    w.cap_r = w.cap_s = kNaMaxEnt;
    const unsigned long long ecap = w.cap_r + w.cap_s;
    w.T = T;
    w.nch_cap = (unsigned)((ecap + kNaMaxTiles) / sj::kChunk + 2);
    w.nl_cap = (unsigned)((ecap + kNaMaxTiles) / (sj::kChunk + 1) + 1);
    w.items_cap = ecap;
    w.vb_cap = (unsigned)(ecap / sj::kRadixBlock + 2ull * w.nl_cap + 1);
    const unsigned long long nslots = (unsigned long long)w.nch_cap + w.vb_cap;
    size_t off = 0;
    auto take = [&](Buf &b, size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        b.p = base + off;
        b.bytes = bytes;
        off += bytes;
    };
    take(w.stats, sizeof(sj::Stats));
    take(w.cnt, 8ull * kNaMaxTiles);
    take(w.off, 8ull * (kNaMaxTiles + 1));
    take(w.bsum, 16ull * (sj::scan_blocks(kNaMaxTiles) + 1));
    take(w.ts, 4ull * (w.nch_cap + 1));
    take(w.large, 4ull * (w.nl_cap + 1));
    take(w.ent_r, 16ull * (w.cap_r + 1));
    take(w.id_r, 4ull * (w.cap_r + 1));
    take(w.ent_s, 16ull * (w.cap_s + 1));
    take(w.id_s, 4ull * (w.cap_s + 1));
    take(w.seg_off, 4ull * (2ull * w.nl_cap + 2));
    take(w.seg_src, 4ull * (2ull * w.nl_cap + 2));
    take(w.seg_vb, 4ull * (2ull * w.nl_cap + 2));
    take(w.hist, 1024ull * (w.vb_cap + 1));
    take(w.key_a, 4ull * (w.items_cap + 1));
    take(w.key_b, 4ull * (w.items_cap + 1));
    take(w.val_a, 4ull * (w.items_cap + 1));
    take(w.val_b, 4ull * (w.items_cap + 1));
    take(w.lmbr, 16ull * (w.items_cap + 1));
    take(w.lid, 4ull * (w.items_cap + 1));
    take(w.pc, 4ull * nslots);
    take(w.poff, 8ull * nslots);
    take(w.resv, 8ull * nslots);
    take(w.fail_c, 4ull * (w.nch_cap + 1));
    take(w.fail_l, 4ull * (w.vb_cap + 1));
    return off <= kNaScratchBytes;
}

}  // namespace

extern "C" int sj_join_noalloc(const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                               const sj_grid *g, sj_pair *d_out, int64_t cap, int64_t *npairs,
                               void *cuda_stream) {
    if (!npairs || cap < 0) return SJ_EINVAL;
    *npairs = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SJ_ECUDA;
    }
    NaDevice *nd = nullptr;
    int st = na_setup(dev, &nd);
    if (st) return st;

    // A context that lives on the stack: it carries the stream and launch
    // parameters only; its allocator is never used on this path.
    sj_ctx c;
    c.device = dev;
    c.stream = (cudaStream_t)cuda_stream;
    c.num_sms = nd->num_sms;
    c.sweep_bps = nd->sweep_bps;
    c.msg[0] = 0;
    sj::GridDev gd;
    if ((st = sj::check_inputs(&c, d_R, nR, d_S, nS, g, &gd))) return st;
    const long long T = (long long)gd.nx * gd.ny;
    if (nR > kNaMaxN || nS > kNaMaxN || T > kNaMaxTiles) return SJ_EINVAL;
    if (cap > 0 && !d_out) return SJ_EINVAL;

    sj::Workspace w;
    if (!na_carve(nd->scratch, T, w)) return SJ_EINTERNAL;

    // Partition and count (every counter starts from a cleared state: the
    // partition clears the stats and the tile counts, and the pair counts
    // are cleared below; everything else is written before it is read).
    if ((st = sj::enqueue_partition(&c, w, (const float4 *)d_R, nR, (const float4 *)d_S, nS, gd))) return st;
    const unsigned nslots = w.nch_cap + w.vb_cap;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.pc.p, 0, 4ull * nslots, c.stream))) return SJ_ECUDA;
    if ((st = sj::enqueue_sweep(&c, w, sj::MODE_COUNT, nullptr, 0, nullptr, nullptr, 0))) return st;
    if ((e = sj::launch_scan_pairs((const unsigned *)w.pc.p, nslots, (unsigned long long *)w.poff.p,
                                   (sj::Stats *)w.stats.p, c.stream)))
        return SJ_ECUDA;
    sj::Stats stats;
    if ((e = cudaMemcpyAsync(&stats, w.stats.p, sizeof stats, cudaMemcpyDeviceToHost, c.stream))) return SJ_ECUDA;
    if ((e = cudaStreamSynchronize(c.stream))) return SJ_ECUDA;
    if (stats.err & sj::kErrBadRect) return SJ_EINVAL;
    // more replicated entries than the scratch holds: the input is too large
    if (stats.err & (sj::kErrEntCap | sj::kErrTooMany)) return SJ_EINVAL;
    if (stats.err & sj::kErrTimeout) return SJ_ETIMEOUT;   // a bounded device wait gave up
    if (stats.err) return SJ_EINTERNAL;                   // a table sized from the limits overflowed
    *npairs = (int64_t)stats.npairs;
    if ((unsigned long long)cap < stats.npairs) return SJ_EOVERFLOW;
    if (stats.npairs == 0) return SJ_OK;
#if SJ_CHECK
    // debug build: bounds checks that failed in the write pass
    if ((st = sj::enqueue_sweep(&c, w, sj::MODE_WRITE, (int2 *)d_out, stats.npairs, nullptr, nullptr, 2))) return st;
    if ((e = cudaMemcpyAsync(&stats, w.stats.p, sizeof stats, cudaMemcpyDeviceToHost, c.stream))) return SJ_ECUDA;
    if ((e = cudaStreamSynchronize(c.stream))) return SJ_ECUDA;
    return (stats.err & sj::kErrCheck) ? SJ_EINTERNAL : SJ_OK;
#else
    return sj::enqueue_sweep(&c, w, sj::MODE_WRITE, (int2 *)d_out, stats.npairs, nullptr, nullptr, 2);
#endif
}
