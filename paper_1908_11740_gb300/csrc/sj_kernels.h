// sj_kernels.h -- host-side launchers of the spatial-join kernels and the
// argument blocks they take.  Internal to the library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sj_common.cuh"

namespace sj {

// Stream-ordered zeroing and small copies done by the SMs instead of a copy
// engine (misc.cu).  A join issues them between its kernels; a copy engine
// that is busy with a large transfer on another stream (the next join's
// inputs in sj_join_host_many) would hold them, and with them the join,
// until that transfer ends.  bytes: a multiple of 4; pointers 4-byte
// aligned; either side of a copy may be page-locked host memory, which the
// device reaches directly (its writes are visible to the host once the
// kernel has completed, e.g. after a stream or event synchronisation).
cudaError_t zero_words_async(void *p, size_t bytes, cudaStream_t s);
cudaError_t copy_words_async(void *dst, const void *src, size_t bytes, cudaStream_t s);

enum { MODE_COUNT = 0, MODE_WRITE = 1, MODE_RESERVE = 2, MODE_TILES = 3, MODE_APPEND = 4 };

// Arguments of the sweep kernels (small-tile chunks and large tiles).
struct SweepArgs {
    const uint2 *off;                 // (R, S) tile offsets, T + 1
    const unsigned *ts;               // chunk table
    const float4 *ent_r;
    const unsigned *id_r;
    const float4 *ent_s;
    const unsigned *id_s;
    Stats *st;
    int work_slot;                    // which st->work counter hands out items
    const unsigned *list;             // optional: only these items (chunks / vbs)
    const unsigned *list_n;           // ... and their number (device)
    unsigned *cnt_out;                // MODE_COUNT: pairs per item
    const unsigned long long *off_in; // MODE_WRITE: output offset per item
    unsigned long long *resv;         // MODE_RESERVE: reserved offset per item
    unsigned *fail;                   // MODE_RESERVE: items that did not fit
    unsigned *nfail;                  // ... their number (device)
    unsigned cnt_base;                // large path: first slot in cnt_out/off_in/resv
    int2 *out;                        // pair buffer
    unsigned long long cap;           // MODE_RESERVE / MODE_APPEND: capacity of out
    unsigned *tile_pairs;             // MODE_TILES: pairs per tile
    unsigned long long base;          // MODE_APPEND: first slot of the appended pairs
    unsigned long long *append;       // MODE_APPEND: pairs appended so far (device counter)
};

// Arguments of the large-tile path (segmented radix sort + sweep).
struct LargeArgs {
    const uint2 *off;
    const unsigned *large;            // tile ids of the large tiles
    const float4 *ent_r;
    const unsigned *id_r;
    const float4 *ent_s;
    const unsigned *id_s;
    unsigned *seg_off;                // item offset of every segment (2*nlarge + 1)
    unsigned *seg_src;                // first entry of every segment in ent_r / ent_s
    unsigned *seg_vb;                 // first virtual block of every segment
    unsigned *hist;                   // 256 per virtual block
    unsigned *key_in, *val_in, *key_out, *val_out;
    float4 *lmbr;                     // sorted entries of the large tiles
    unsigned *lid;
    // candidate-parallel sweep (optional: all null -> one thread per pivot)
    unsigned *lstart;                 // first candidate of every pivot (position in the other segment)
    unsigned long long *lcoff;        // exclusive prefix of the pivots' candidate counts, per virtual block
    unsigned long long *vbc;          // candidates of every virtual block
    unsigned long long *vbpairs;      // pairs of every virtual block (count pass)
    unsigned long long *vbcur;        // write cursor of every virtual block (write pass)
    unsigned *vbch;                   // first candidate chunk of every virtual block (vb_cap + 1)
    float2 *ly;                       // (y_l, y_u) of the sorted entries: all a candidate test reads
    unsigned long long items_cap;
    unsigned vb_cap;
    Stats *st;
};

// partition.cu
cudaError_t launch_count(const float4 *R, long long nR, const float4 *S, long long nS, GridDev g,
                         unsigned *cnt, Stats *st, int grid, cudaStream_t s);
cudaError_t launch_scan(const uint2 *cnt, long long T, unsigned long long *bsum, uint2 *off,
                        unsigned *ts, unsigned nch_cap, unsigned *large, unsigned nl_cap, Stats *st,
                        cudaStream_t s);
long long scan_blocks(long long T);
cudaError_t launch_scatter(const float4 *R, long long nR, const float4 *S, long long nS, GridDev g,
                           unsigned *cnt, const uint2 *off, float4 *ent_r, unsigned *id_r,
                           unsigned long long cap_r, float4 *ent_s, unsigned *id_s,
                           unsigned long long cap_s, Stats *st, int grid, cudaStream_t s);

// sweep.cu
size_t sweep_smem_bytes();
cudaError_t sweep_setup();
int sweep_blocks_per_sm();
cudaError_t launch_sweep_chunks(int mode, const SweepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_large_sort(LargeArgs a, int grid, cudaStream_t s);
cudaError_t launch_sweep_large(int mode, const LargeArgs &a, const SweepArgs &o, int grid,
                               cudaStream_t s);
// one-pass large tiles: candidate ranges and chunks (sets st->nlch), then the
// candidate sweep appending every chunk's pairs at o.base + *o.append
constexpr int kLargeCandChunk = 4096;   // candidates per chunk of the large-tile sweep
cudaError_t launch_large_plan(const LargeArgs &a, int grid, cudaStream_t s);
cudaError_t launch_large_append(const LargeArgs &a, const SweepArgs &o, int grid, cudaStream_t s);
cudaError_t launch_scan_pairs(const unsigned *cnt, unsigned n, unsigned long long *off, Stats *st,
                              cudaStream_t s);

}  // namespace sj
