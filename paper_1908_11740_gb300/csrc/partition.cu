// partition.cu -- partitioning phase of PBSM on the GPU (Sec. 3.4 steps 2-4):
// count the rectangles of every tile, prefix-sum the counts into per-tile
// segments, then write every rectangle into every tile it overlaps
// (multi-assignment, Sec. 2.2).  The scan also cuts the tile sequence into
// sweep chunks and lists the tiles too heavy for one chunk.
#define SJ_FILE_CODE 3
#include "sj_common.cuh"
#include "sj_kernels.h"

namespace sj {

// ---- a2: per-tile counts -------------------------------------------------
// One thread per rectangle (grid-stride, U independent 16-byte loads in
// flight per thread).  R and S share the launch: index i < nR is R[i].
template <int U>
__global__ void __launch_bounds__(256) k_count(const float4 *__restrict__ R, long long nR,
                                               const float4 *__restrict__ S, long long nS,
                                               GridDev g, unsigned *__restrict__ cnt,
                                               Stats *__restrict__ st) {
    const long long n = nR + nS;
    const long long step = (long long)gridDim.x * blockDim.x * U;
    int bad = 0;
    for (long long base = (long long)blockIdx.x * blockDim.x * U + threadIdx.x; base < n;
         base += step) {
        float4 m[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            long long i = base + (long long)u * blockDim.x;
            if (i < n) m[u] = ld_stream(i < nR ? R + i : S + (i - nR));
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = base + (long long)u * blockDim.x;
            bool valid = i < n;
            if (valid && !rect_ok(m[u])) {
                bad = 1;
                valid = false;
            }
            const unsigned side = i >= nR;
            int cx0 = 0, cx1 = -1, cy0 = 0, cy1 = -1;
            if (valid) {
                cx0 = cell_of(m[u].x, g.x0, g.gx, g.nx), cx1 = cell_of(m[u].z, g.x0, g.gx, g.nx);
                cy0 = cell_of(m[u].y, g.y0, g.gy, g.ny), cy1 = cell_of(m[u].w, g.y0, g.gy, g.ny);
            }
            // the first tile: lanes of the warp that hit the same one add with
            // one atomic (dense tiles would otherwise serialise on one counter)
            const unsigned long long key =
                valid ? 2ull * ((unsigned long long)cy0 * (unsigned)g.nx + (unsigned)cx0) + side : ~0ull;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (valid && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(cnt + key, (unsigned)__popc(peers));
            for (int cy = cy0; cy <= cy1; cy++)
                for (int cx = cx0; cx <= cx1; cx++)
                    if (cy != cy0 || cx != cx0) atomicAdd(cnt + 2 * ((long long)cy * g.nx + cx) + side, 1u);
        }
    }
    if (bad) atomicOr(&st->err, kErrBadRect);
}

// ---- a3: exclusive scan of the (R, S) counts -------------------------------
// Reduce-then-scan: block sums, one-block scan of the sums, then a
// block-local scan that adds the block's offset.  kScanTile tiles per block.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kScanThreads * kScanPer;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if ((threadIdx.x & 31) >= d) v += o;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (NT = blockDim.x, a
// multiple of 32, at most 1024); returns the exclusive prefix and the block
// total in *total.  Ends with a barrier so it can be called back to back.
template <typename T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T *total) {
    __shared__ T warp_tot[NT / 32];
    __shared__ T s_total;
    const T inc = warp_incl_scan(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        const T x = l < NT / 32 ? warp_tot[l] : T(0);
        const T xi = warp_incl_scan(x);
        if (l < NT / 32) warp_tot[l] = xi - x;
        if (l == NT / 32 - 1) s_total = xi;
    }
    __syncthreads();
    const T res = warp_tot[w] + inc - v;
    *total = s_total;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint2 *__restrict__ cnt,
                                                              long long T,
                                                              unsigned long long *__restrict__ bsum) {
    const long long t0 = (long long)blockIdx.x * kScanTile;
    unsigned long long sr = 0, ss = 0;
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
        long long t = t0 + k;
        if (t < T) {
            uint2 c = cnt[t];
            sr += c.x;
            ss += c.y;
        }
    }
    unsigned long long tr, ts;
    block_excl_scan<unsigned long long, kScanThreads>(sr, &tr);
    block_excl_scan<unsigned long long, kScanThreads>(ss, &ts);
    if (threadIdx.x == 0) {
        bsum[2 * blockIdx.x] = tr;
        bsum[2 * blockIdx.x + 1] = ts;
    }
}

// One block of 1024 threads: exclusive scan of nb (R, S) block sums in place.
__global__ void __launch_bounds__(1024) k_scan_top(unsigned long long *__restrict__ bsum, int nb) {
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    unsigned long long sr = 0, ss = 0;
    for (int k = 0; k < per; k++) {
        int b = b0 + k;
        if (b < nb) {
            sr += bsum[2 * b];
            ss += bsum[2 * b + 1];
        }
    }
    unsigned long long tr, ts;
    unsigned long long er = block_excl_scan<unsigned long long, 1024>(sr, &tr);
    unsigned long long es = block_excl_scan<unsigned long long, 1024>(ss, &ts);
    for (int k = 0; k < per; k++) {
        int b = b0 + k;
        if (b < nb) {
            unsigned long long vr = bsum[2 * b], vs = bsum[2 * b + 1];
            bsum[2 * b] = er;
            bsum[2 * b + 1] = es;
            er += vr;
            es += vs;
        }
    }
}

// Writes off[t] = (R offset, S offset) for t in [0, T], the chunk table
// ts[c] = first tile whose weight prefix W[t] = offR + offS + t reaches
// c * kChunk, the list of large tiles (weight > kChunk), and the totals.
__global__ void __launch_bounds__(kScanThreads) k_scan_down(
    const uint2 *__restrict__ cnt, long long T, const unsigned long long *__restrict__ boff,
    uint2 *__restrict__ off, unsigned *__restrict__ ts, unsigned nch_cap,
    unsigned *__restrict__ large, unsigned nl_cap, Stats *__restrict__ st) {
    const long long tb = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
    uint2 c[kScanPer];
    unsigned long long sr = 0, ss = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        long long t = tb + k;
        c[k] = t < T ? cnt[t] : make_uint2(0, 0);
        sr += c[k].x;
        ss += c[k].y;
    }
    unsigned long long tr, tsum;
    unsigned long long pr = block_excl_scan<unsigned long long, kScanThreads>(sr, &tr);
    unsigned long long ps = block_excl_scan<unsigned long long, kScanThreads>(ss, &tsum);
    pr += boff[2 * blockIdx.x];
    ps += boff[2 * blockIdx.x + 1];
    // weight of the tile before this thread's first tile
    unsigned long long wprev_w = 0;
    if (tb >= 1 && tb < T) {
        uint2 cp = cnt[tb - 1];
        wprev_w = (unsigned long long)cp.x + cp.y + 1;
    }
    int err = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        long long t = tb + k;
        if (t >= T) break;
        if (pr + c[k].x > 0x7fffffffull || ps + c[k].y > 0x7fffffffull) err |= kErrTooMany;
        off[t] = make_uint2((unsigned)pr, (unsigned)ps);
        const unsigned long long W = pr + ps + (unsigned long long)t;
        const unsigned long long w = (unsigned long long)c[k].x + c[k].y + 1;
        if (t == 0) {
            ts[0] = 0;
        } else {
            const unsigned long long Wp = W - wprev_w;
            for (unsigned long long ch = Wp / kChunk + 1; ch <= W / kChunk; ch++) {
                if (ch < nch_cap) ts[ch] = (unsigned)t;
                else err |= kErrChunkCap;
            }
        }
        if (w > (unsigned long long)kChunk) {
            unsigned idx = atomicAdd(&st->nlarge, 1u);
            if (idx < nl_cap) large[idx] = (unsigned)t;
            else err |= kErrLargeCap;
        }
        if (t == T - 1) {
            const unsigned long long er = pr + c[k].x, es = ps + c[k].y;
            off[T] = make_uint2((unsigned)er, (unsigned)es);
            st->e_r = er;
            st->e_s = es;
            st->w_total = W + w;
            const unsigned long long nch = W / kChunk + 1;
            if (nch < nch_cap) {
                ts[nch] = (unsigned)T;
                st->nchunks = (unsigned)nch;
            } else {
                err |= kErrChunkCap;
            }
        }
        wprev_w = w;
        pr += c[k].x;
        ps += c[k].y;
    }
    if (err) atomicOr(&st->err, err);
}

// ---- a4: scatter -----------------------------------------------------------
// Second read of the rectangles.  Each (rectangle, tile) takes a slot of the
// tile's segment by decrementing the tile's count (the count array ends at
// zero).  The id word carries the first-column / first-row flags used by the
// duplicate test.  Coordinates are canonicalised (-0 -> +0).
template <int U>
__global__ void __launch_bounds__(256) k_scatter(const float4 *__restrict__ R, long long nR,
                                                 const float4 *__restrict__ S, long long nS,
                                                 GridDev g, unsigned *__restrict__ cnt,
                                                 const uint2 *__restrict__ off,
                                                 float4 *__restrict__ ent_r, unsigned *__restrict__ id_r,
                                                 unsigned long long cap_r,
                                                 float4 *__restrict__ ent_s, unsigned *__restrict__ id_s,
                                                 unsigned long long cap_s, Stats *__restrict__ st) {
    const long long n = nR + nS;
    const long long step = (long long)gridDim.x * blockDim.x * U;
    int err = 0;
    for (long long base = (long long)blockIdx.x * blockDim.x * U + threadIdx.x; base < n;
         base += step) {
        float4 m[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            long long i = base + (long long)u * blockDim.x;
            if (i < n) m[u] = ld_stream(i < nR ? R + i : S + (i - nR));
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = base + (long long)u * blockDim.x;
            float4 v = m[u];
            const bool valid = i < n && rect_ok(v);
            v.x = __fadd_rn(v.x, 0.0f);
            v.y = __fadd_rn(v.y, 0.0f);
            v.z = __fadd_rn(v.z, 0.0f);
            v.w = __fadd_rn(v.w, 0.0f);
            const unsigned side = i >= nR;
            const unsigned id = (unsigned)(side ? i - nR : i);
            int cx0 = 0, cx1 = -1, cy0 = 0, cy1 = -1;
            if (valid) {
                cx0 = cell_of(v.x, g.x0, g.gx, g.nx), cx1 = cell_of(v.z, g.x0, g.gx, g.nx);
                cy0 = cell_of(v.y, g.y0, g.gy, g.ny), cy1 = cell_of(v.w, g.y0, g.gy, g.ny);
            }
            // slots of the first tile: lanes that hit the same tile take
            // consecutive slots with one atomic on its counter
            const unsigned long long key =
                valid ? 2ull * ((unsigned long long)cy0 * (unsigned)g.nx + (unsigned)cx0) + side : ~0ull;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const int leader = __ffs(peers) - 1;
            unsigned first = 0;
            if (valid && (int)(threadIdx.x & 31) == leader) first = atomicSub(cnt + key, (unsigned)__popc(peers));
            first = __shfl_sync(0xffffffffu, first, leader);
            unsigned lt;
            asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
            const unsigned k0 = first - 1u - (unsigned)__popc(peers & lt);
            float4 *ent = side ? ent_s : ent_r;
            unsigned *idw = side ? id_s : id_r;
            const unsigned long long cap = side ? cap_s : cap_r;
            for (int cy = cy0; cy <= cy1; cy++)
                for (int cx = cx0; cx <= cx1; cx++) {
                    const long long t = (long long)cy * g.nx + cx;
                    const unsigned k = (cy == cy0 && cx == cx0) ? k0 : atomicSub(cnt + 2 * t + side, 1u) - 1u;
                    const unsigned o = side ? off[t].y : off[t].x;
                    const unsigned long long pos = (unsigned long long)o + k;
                    // slot k counts down from the tile's count: within its segment
                    if (!SJ_IN(st, k, (side ? off[t + 1].y : off[t + 1].x) - o)) continue;
                    if (pos < cap) {
                        ent[pos] = v;
                        idw[pos] = id | (cx == cx0 ? kFlagCol : 0u) | (cy == cy0 ? kFlagRow : 0u);
                    } else {
                        err |= kErrEntCap;
                    }
                }
        }
    }
    if (err) atomicOr(&st->err, err);
}

// ---- launchers ---------------------------------------------------------------
cudaError_t launch_count(const float4 *R, long long nR, const float4 *S, long long nS, GridDev g,
                         unsigned *cnt, Stats *st, int grid, cudaStream_t s) {
    if (nR + nS == 0) return cudaSuccess;
    k_count<4><<<grid, 256, 0, s>>>(R, nR, S, nS, g, cnt, st);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint2 *cnt, long long T, unsigned long long *bsum, uint2 *off,
                        unsigned *ts, unsigned nch_cap, unsigned *large, unsigned nl_cap, Stats *st,
                        cudaStream_t s) {
    const long long nb = (T + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(cnt, T, bsum);
    k_scan_top<<<1, 1024, 0, s>>>(bsum, (int)nb);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(cnt, T, bsum, off, ts, nch_cap, large, nl_cap,
                                                      st);
    return cudaGetLastError();
}

long long scan_blocks(long long T) { return (T + kScanTile - 1) / kScanTile; }

cudaError_t launch_scatter(const float4 *R, long long nR, const float4 *S, long long nS, GridDev g,
                           unsigned *cnt, const uint2 *off, float4 *ent_r, unsigned *id_r,
                           unsigned long long cap_r, float4 *ent_s, unsigned *id_s,
                           unsigned long long cap_s, Stats *st, int grid, cudaStream_t s) {
    if (nR + nS == 0) return cudaSuccess;
    k_scatter<4><<<grid, 256, 0, s>>>(R, nR, S, nS, g, cnt, off, ent_r, id_r, cap_r, ent_s, id_s,
                                      cap_s, st);
    return cudaGetLastError();
}

}  // namespace sj
