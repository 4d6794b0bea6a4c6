// sj_blocked.h -- the two-level (blocked) PBSM path: argument blocks,
// constants and launchers.  Internal to the library.
#pragma once
#include "sj_common.cuh"
#include "sj_kernels.h"

namespace sj {

constexpr int kL1Threads = 1024;     // L1 count / write CTAs
constexpr int kMaxBlocks = 24576;    // blocks per grid (2 * 4 bytes of shared memory each)
constexpr int kBJThreads = 512;      // fused block-join CTAs (two per SM)
constexpr int kFineCap = 3072;       // tile entries staged in shared memory per band
constexpr int kMaxG = 32;            // tiles per block side
constexpr int kLoadBatch = 4;        // entries a thread loads before using them
constexpr int kMaxJoins = 4096;      // joins in one batch
constexpr int kPairBuf = 768;        // pairs a one-pass block collects in shared memory
constexpr int kPairSpill = 16384;    // ... and then in its CTA's global spill area
constexpr int kMaxFine = kMaxG * kMaxG;

// An L1 entry: one aligned 32-byte sector.
struct __align__(32) BEnt {
    float4 mbr;
    unsigned id;   // original index
    unsigned cx;   // first | last tile column << 16
    unsigned cy;   // first | last tile row << 16
    unsigned pad;
};

// One L1 entry with one 256-bit load (read-only for the kernel that reads it).
__device__ __forceinline__ void load_bent(const uint4 *src, uint4 &h, uint4 &t) {
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(h.x), "=r"(h.y), "=r"(h.z), "=r"(h.w), "=r"(t.x), "=r"(t.y), "=r"(t.z), "=r"(t.w)
                 : "l"(src));
}

// One 32-byte store of an L1 entry (a whole sector in one instruction).
__device__ __forceinline__ void store_bent(BEnt *dst, uint4 h, uint4 t) {
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst), "r"(h.x), "r"(h.y), "r"(h.z),
                 "r"(h.w), "r"(t.x), "r"(t.y), "r"(t.z), "r"(t.w)
                 : "memory");
}

// One join of a (possibly batched) two-level partition: its inputs, grid,
// block plan and place in the global input and block index spaces.
struct JoinDesc {
    const float4 *R, *S;
    long long nR, nS;
    long long in_off;       // first global input index (R of this join, then S)
    GridDev g;
    int G;                  // tiles per block side
    unsigned gmul;          // 2^32 / G + 1
    int bx, by;             // blocks per axis
    int boff;               // first global block id
    int pad;
    float h;                // point inputs (BArgs::pts): half-width of their squares
    long long samp_off;     // batched one-pass: first feature sample of this join
};

struct BArgs {
    const float4 *R;
    long long nR;
    const float4 *S;
    long long nS;
    GridDev g;
    int G, bx, by, nb;          // tiles per block side, blocks per axis, blocks
    unsigned gmul;              // 2^32 / G + 1 (division by G, G > 1)
    unsigned *H;                // per-CTA block counts, CTA-major (nc x 2nb)
    unsigned *btot;             // entries per (side, block)
    unsigned *bo_r, *bo_s;      // block starts per side (nb + 1)
    unsigned *items;            // blocks with entries on both sides
    uint4 *imeta;               // per work item: block, R start, R count, S start
    unsigned *ins;              // per work item: S count
    BEnt *bent_r, *bent_s;
    unsigned long long cap_r, cap_s;
    unsigned *feat_raw;         // optional: sampled bucket counts per block (learned sizing)
    unsigned *cur;              // optional: shared per-block write cursors (2 nbt)
    const JoinDesc *jd;         // the joins (one for a single join)
    int nj;                     // number of joins
    int nbt;                    // blocks of all joins (== nb for a single join)
    unsigned *ijoin;            // join of every work item
    unsigned *jfirst;           // first work item of every join (nj + 1)
    unsigned long long *scan_part;   // block scan: 3 sums per chunk of blocks (bscan_chunks(nbt))
    unsigned *lpool;            // optional: row lists of blocks staged in several bands
    unsigned long long lpool_cap;
    int pts;                    // 1: R, S hold float2 points, read as squares of half-width h
    float h;
    int adaptive;               // sweep axis per tile from Eq. 2 histograms (Sec. 3.3)
    int gbda;                   // grouping-based duplicate avoidance instead of Eq. 1
    int fine_cap;               // entries one tile may hold for the consumer of the partition
    int stop_direct;            // one-pass sizing: skip the feature sample once a tile exceeds shared memory
    Stats *st;
};

// Point i of one side read as its square (the point inputs of the distance
// join): half-width h around the point, corners rounded outward.  The
// kernels that read inputs take it when their template parameter PTS is 1;
// with PTS = 0 they keep the plain rectangle load.
__device__ __forceinline__ float4 load_square(const float4 *base, long long i, float h) {
    float2 p;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];"
                 : "=f"(p.x), "=f"(p.y)
                 : "l"(reinterpret_cast<const float2 *>(base) + i));
    return make_float4(__fsub_rd(p.x, h), __fsub_rd(p.y, h), __fadd_ru(p.x, h), __fadd_ru(p.y, h));
}

struct BJoinOut {
    int work_slot;
    const unsigned *list;       // optional subset of work items
    const unsigned *list_n;
    unsigned *cnt_out;          // MODE_COUNT: pairs per item
    const unsigned long long *off_in;   // MODE_WRITE: offset per item
    unsigned long long *resv;   // MODE_RESERVE: reserved offset per item
    unsigned *fail;             // MODE_RESERVE: items that did not fit
    unsigned *nfail;
    int2 *out;
    unsigned long long cap;
    unsigned *tile_pairs;       // MODE_TILES
    int2 *spill;                // MODE_RESERVE, optional: kPairSpill pairs per CTA
    unsigned char *tile_axis;   // MODE_COUNT with adaptive axes, optional: axis of every tile (1 = y)
};

cudaError_t blocked_setup();
int bjoin_blocks_per_sm();
int l1_blocks_per_sm(int nb);
size_t bjoin_smem_bytes();
cudaError_t launch_bcount(const BArgs &a, int nc, cudaStream_t s);
cudaError_t launch_bcount_global(const BArgs &a, int grid, cudaStream_t s);
cudaError_t launch_bcount_local(const BArgs &a, int grid, cudaStream_t s);
cudaError_t launch_extent_stats(const BArgs &a, double *out, int grid, cudaStream_t s);
cudaError_t launch_join_offsets(const BArgs &a, const unsigned long long *poff, unsigned long long *joff,
                                cudaStream_t s);
cudaError_t launch_bscan(const BArgs &a, int nc, cudaStream_t s);
cudaError_t launch_bscan_blocks_only(const BArgs &a, cudaStream_t s);
int bscan_chunks(int nb);
cudaError_t launch_bscatter(const BArgs &a, int nc, cudaStream_t s);
cudaError_t launch_bfeat_sample(const BArgs &a, int grid, cudaStream_t s);
// batches: rectangles 0, kPhi, 2 kPhi, ... of every side of every join
cudaError_t launch_bfeat_sample_batch(const BArgs &a, long long nsamp, int grid, cudaStream_t s);
// pairs of every work item moved from its reserved range to its place in
// item order (batched one-pass join)
cudaError_t launch_regroup(const unsigned *cnt, const unsigned long long *resv, const unsigned long long *poff,
                           const unsigned *n_dev, const int2 *src, int2 *dst, int grid, cudaStream_t s);
cudaError_t launch_bjoin(int mode, const BArgs &a, const BJoinOut &o, int grid, cudaStream_t s);
// 1D grids: one CTA per stripe, R and S sorted along the stripe in shared
// memory, forward scan along the stripe (stripes.cu)
cudaError_t stripe_setup();
size_t stripe_smem_bytes();
cudaError_t launch_stripe_join(int mode, const BArgs &a, int vert, unsigned *skey, unsigned short *sval,
                               unsigned long long scap, const BJoinOut &o, int grid, cudaStream_t s);

}  // namespace sj
