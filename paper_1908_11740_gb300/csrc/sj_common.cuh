// sj_common.cuh -- device-side definitions shared by the kernels of the
// spatial-join filter step (PBSM, "Parallel In-Memory Evaluation of Spatial
// Joins").  Target: sm_103a only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sj {

// ---- sizes ---------------------------------------------------------------
// The small-tile sweep works on "chunks": runs of consecutive tiles whose
// weight (replicated entries + 1 per tile) starts inside one window of
// kChunk units.  A tile heavier than kChunk is "large" and is joined by the
// large-tile path (global segmented radix sort + multi-CTA sweep).  A chunk
// therefore holds fewer than 2*kChunk entries and at most kChunk tiles.
constexpr int kChunk = 1024;
constexpr int kChunkEnt = 2 * kChunk;        // entries staged per chunk
constexpr int kSweepThreads = 256;
constexpr int kItems = kChunkEnt / kSweepThreads;

// Radix sort of the large tiles: 8-bit digits, 4096 items per virtual block.
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixBlock = kRadixThreads * kRadixRounds;

// id word of an entry: original index in bits 0..29, bit 30 set when the
// tile is the first column the rectangle covers, bit 31 when it is the first
// row.  The pair (r, s) is reported in a tile iff the OR of the two words has
// both bits: max(cx0_r, cx0_s) == col and max(cy0_r, cy0_s) == row, which is
// Eq. 1 in tile-index form.
constexpr uint32_t kFlagCol = 1u << 30;
constexpr uint32_t kFlagRow = 1u << 31;
constexpr uint32_t kFlags = kFlagCol | kFlagRow;
constexpr uint32_t kIdMask = kFlagCol - 1u;

// error bits collected on the device
constexpr int kErrBadRect = 1;       // NaN/Inf coordinate or xl > xu / yl > yu
constexpr int kErrEntCap = 2;        // replicated entries exceed the workspace
constexpr int kErrTooMany = 4;       // more than 2^31 entries on a side
constexpr int kErrChunkCap = 8;      // chunk table overflow (internal)
constexpr int kErrLargeCap = 16;     // large-tile table overflow (internal)
constexpr int kErrOutCap = 32;       // one-pass output capacity exceeded
constexpr int kErrTimeout = 64;      // a bounded device-side wait gave up
constexpr int kErrCheck = 128;       // debug build: an index failed its bounds check

// Errors after which the partition is incomplete: every kernel that reads the
// partition returns at once (the host grows the workspace and starts over).
constexpr int kErrFatal = kErrEntCap | kErrTooMany | kErrChunkCap | kErrLargeCap | kErrTimeout | kErrCheck;

struct GridDev {
    int nx, ny;
    float x0, y0;
    float gx, gy;   // (float)nx / (x1 - x0), (float)ny / (y1 - y0)
};

// Device-resident counters of one join; zeroed at the start of a call.
struct Stats {
    unsigned long long e_r, e_s;        // replicated entries per side
    unsigned long long w_total;         // sum of tile weights
    unsigned long long large_items;     // entries in large tiles (R+S)
    unsigned long long npairs;          // result pairs (count pass / reserve)
    unsigned int nchunks;               // chunks of small tiles
    unsigned int nlarge;                // large tiles
    unsigned int nvb;                   // radix virtual blocks of large tiles
    unsigned int nfail;                 // one-pass chunks that did not fit
    unsigned int nfail_large;           // one-pass large-tile blocks that did not fit
    unsigned int work[8];               // work counters of persistent kernels
    unsigned long long lpool[4];        // blocked path: row-list pool cursor per work slot
    int err;
    int need_direct;                    // blocked path: a tile exceeds shared memory
    unsigned int check;                 // debug build: first failed bounds check (file << 16 | line)
    unsigned int nlch;                  // candidate chunks of the large-tile sweep
    unsigned int naxis_y;               // blocked path: work items swept along y (adaptive axis)
    unsigned long long apairs;          // large tiles appended in one pass (single-level one-pass)
};

// ---- debug build (-DSJ_CHECK=1) --------------------------------------------
// Bounds checks of the data-dependent indexes: offsets taken from atomics,
// scans, counts and searches.  A failed check records its site (the file
// code SJ_FILE_CODE of the translation unit << 16 | the source line) in
// Stats::check, the first one winning, sets kErrCheck (fatal: the remaining
// kernels of the call return at once) and skips the access; a checked read
// takes element 0 instead.  The call then fails with SJ_EINTERNAL and names
// the site.  In the normal build the checks compile to nothing.
#ifndef SJ_CHECK
#define SJ_CHECK 0
#endif
#ifndef SJ_FILE_CODE
#define SJ_FILE_CODE 0
#endif
__device__ __forceinline__ bool check_index(Stats *st, unsigned long long i, unsigned long long n, unsigned site) {
    if (i < n) return true;
    atomicCAS(&st->check, 0u, site);
    atomicOr(&st->err, kErrCheck);
    return false;
}
#if SJ_CHECK
// true when 0 <= i < n (i of any integer type; a negative i fails)
#define SJ_IN(st, i, n) \
    ::sj::check_index((st), (unsigned long long)(long long)(i), (unsigned long long)(n), \
                      ((unsigned)SJ_FILE_CODE << 16) | (unsigned)__LINE__)
// i when 0 <= i < n, else 0 (for reads)
#define SJ_AT(st, i, n) (SJ_IN(st, i, n) ? (i) : 0)
#else
#define SJ_IN(st, i, n) true
#define SJ_AT(st, i, n) (i)
#endif

// ---- the cell function (tile index of a coordinate) ------------------------
// clamp(floor((v - g0) * ginv), 0, n - 1) with both operations rounded to
// float32 (no contraction); monotone non-decreasing in v.
__device__ __forceinline__ int cell_of(float v, float g0, float ginv, int n) {
    float t = __fmul_rn(__fsub_rn(v, g0), ginv);
    float f = floorf(t);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(n - 1)) return n - 1;
    return (int)f;
}

// Order-preserving map float -> uint32 (ascending floats give ascending
// keys; -0 sorts just before +0, both compare equal as floats).
__device__ __forceinline__ uint32_t xkey(float x) {
    uint32_t b = __float_as_uint(x);
    return b ^ ((b >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}

__device__ __forceinline__ bool rect_ok(float4 m) {
    return isfinite(m.x) && isfinite(m.y) && isfinite(m.z) && isfinite(m.w) &&
           m.x <= m.z && m.y <= m.w;
}

// Streaming 16-byte load (read once, do not keep in L1).
__device__ __forceinline__ float4 ld_stream(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ bool reported_here(uint32_t a, uint32_t b) {
    return ((a | b) & kFlags) == kFlags;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Block-uniform test of the fatal error bits (one read by thread 0, shared
// with the block), so that all threads of a block leave together.
__device__ __forceinline__ bool block_skip(const Stats *st) {
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (*(volatile const int *)&st->err) & kErrFatal;
    __syncthreads();
    const int v = s_skip;
    __syncthreads();
    return v != 0;
}

// Same, and also when the two-level path has been found unsuitable (a tile
// exceeds shared memory): its remaining kernels would be wasted.
__device__ __forceinline__ bool block_skip_blocked(const Stats *st) {
    __shared__ int s_skip_b;
    if (threadIdx.x == 0)
        s_skip_b = ((*(volatile const int *)&st->err) & kErrFatal) | (*(volatile const int *)&st->need_direct);
    __syncthreads();
    const int v = s_skip_b;
    __syncthreads();
    return v != 0;
}

}  // namespace sj
