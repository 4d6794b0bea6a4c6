// blocked.cu -- two-level PBSM on the GPU: the uniform nx x ny grid of the
// method (Sec. 2.2) is grouped into coarse blocks of G x G tiles.
//
//  L1 (global memory): the count -> prefix-sum -> write scheme of Sec. 3.4
//     steps 2-4, applied to blocks: every CTA counts its slice of the input
//     per block in shared memory, a scan turns the (block, CTA) counts into
//     write offsets, and every CTA writes its slice into the blocks
//     (multi-assignment: a rectangle goes to every block it overlaps).  Each
//     entry is one aligned 32-byte sector, so the scattered writes are whole
//     sectors and need no read-modify-write.
//  L2 (shared memory, fused with the join): one CTA takes a block, assigns
//     its entries to the block's tiles (again every tile a rectangle
//     overlaps), sorts every tile by x_l, and runs the forward scan of
//     Algorithm 1 with the y-test and the reference-point test of Eq. 1.  The
//     tile segments never leave shared memory.
//
// The pairs reported are exactly those of single-level PBSM on the same
// nx x ny grid: a pair is reported by the tile that holds its reference
// point, and that tile belongs to exactly one block.
#define SJ_FILE_CODE 1
#include <cstddef>

#include "sj_blocked.h"
#include "sj_learned.h"

namespace sj {

constexpr unsigned kFullMask = 0xffffffffu;

// x / G for x < 2^16 and G <= 32 as a multiply-high by gmul = 2^32 / G + 1
// (exact in that range); G == 1 passes x through.
__device__ __forceinline__ int div_g(int x, const BArgs &a) {
    return a.G == 1 ? x : (int)__umulhi((unsigned)x, a.gmul);
}

__device__ __forceinline__ unsigned lanemask_lt_b() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// L1 count: per-CTA block histograms (shared memory), slice c of the input.
// H is CTA-major: H[c * 2NB + side * NB + b].
// ---------------------------------------------------------------------------
template <int PTS>
__global__ void __launch_bounds__(kL1Threads) k_bcount(BArgs a) {
    extern __shared__ unsigned hist[];   // 2 * NB
    const int NB2 = 2 * a.nb;
    for (int k = threadIdx.x; k < NB2; k += kL1Threads) hist[k] = 0;
    __syncthreads();
    const long long n = a.nR + a.nS;
    const long long q = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * q, i1 = min(n, i0 + q);
    int bad = 0;
    constexpr int U = 8;   // loads in flight per thread
    for (long long base = i0 + threadIdx.x; base < i1; base += (long long)U * kL1Threads) {
        float4 m[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = base + (long long)u * kL1Threads;
            if (i < i1) {
                if constexpr (PTS) m[u] = load_square(i < a.nR ? a.R : a.S, i < a.nR ? i : i - a.nR, a.h);
                else m[u] = ld_stream(i < a.nR ? a.R + i : a.S + (i - a.nR));
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long i = base + (long long)u * kL1Threads;
            if (i >= i1) break;
            if (!rect_ok(m[u])) {
                bad = 1;
                continue;
            }
            const int side = i >= a.nR;
            const int cx0 = cell_of(m[u].x, a.g.x0, a.g.gx, a.g.nx), cx1 = cell_of(m[u].z, a.g.x0, a.g.gx, a.g.nx);
            const int cy0 = cell_of(m[u].y, a.g.y0, a.g.gy, a.g.ny), cy1 = cell_of(m[u].w, a.g.y0, a.g.gy, a.g.ny);
            const int bx0 = div_g(cx0, a), bx1 = div_g(cx1, a), by0 = div_g(cy0, a), by1 = div_g(cy1, a);
            unsigned *h = hist + side * a.nb;
            for (int by = by0; by <= by1; by++)
                for (int bx = bx0; bx <= bx1; bx++)
                    if (SJ_IN(a.st, by * a.bx + bx, a.nb)) atomicAdd(h + by * a.bx + bx, 1u);

        }
    }
    __syncthreads();
    unsigned *row = a.H + (size_t)blockIdx.x * NB2;
    for (int k = threadIdx.x; k < NB2; k += kL1Threads) row[k] = hist[k];
    if (bad) atomicOr(&a.st->err, kErrBadRect);
}

// L1 scan, part 1: for every (side, block), the total per (side, block) and,
// for the CTA-private write ranges (no shared cursors), the exclusive prefix
// over CTAs (in place).
__global__ void __launch_bounds__(256) k_bscan_ctas(BArgs a, int nc) {
    const int NB2 = 2 * a.nb;
    const int sb = blockIdx.x * 256 + threadIdx.x;
    if (sb >= NB2) return;
    unsigned *__restrict__ H = a.H;
    const bool prefix = a.cur == nullptr;
    unsigned run = 0;
    for (int c0 = 0; c0 < nc; c0 += 16) {
        unsigned v[16];
#pragma unroll
        for (int u = 0; u < 16; u++) v[u] = c0 + u < nc ? H[(size_t)(c0 + u) * NB2 + sb] : 0u;
#pragma unroll
        for (int u = 0; u < 16; u++)
            if (c0 + u < nc) {
                if (prefix) H[(size_t)(c0 + u) * NB2 + sb] = run;
                run += v[u];
            }
    }
    a.btot[sb] = run;
}

// L1 scan, part 2 (one block of 1024): exclusive scans of the per-block
// totals of each side -> block starts (and the shared write cursors); the
// work list of blocks that hold both sides, in block order (so the items of
// each join are consecutive), with their ranges, join and each join's first
// item; the totals.  One pass over chunks of 8192 blocks: every thread loads
// 8 consecutive blocks of each side, the chunk is scanned once for the packed
// (R, S) prefix and once for the work-item count, and a carry links chunks.
constexpr int kScanPer = 8;
constexpr int kScanThreads = 256;
constexpr int kScanChunk = kScanThreads * kScanPer;   // blocks per CTA of the block scan
__device__ __forceinline__ void load8(const unsigned *__restrict__ p, int b, int nb, unsigned (&v)[kScanPer]) {
    if (b + kScanPer <= nb && ((reinterpret_cast<uintptr_t>(p + b) & 15) == 0)) {
        const uint4 x = *reinterpret_cast<const uint4 *>(p + b), y = *reinterpret_cast<const uint4 *>(p + b + 4);
        v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w, v[4] = y.x, v[5] = y.y, v[6] = y.z, v[7] = y.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanPer; k++) v[k] = b + k < nb ? p[b + k] : 0u;
    }
}

// p[b .. b+7] = v (two 16-byte stores when aligned and in range).
__device__ __forceinline__ void store8(unsigned *__restrict__ p, int b, int nb, const unsigned (&v)[kScanPer]) {
    if (b + kScanPer <= nb && ((reinterpret_cast<uintptr_t>(p + b) & 15) == 0)) {
        *reinterpret_cast<uint4 *>(p + b) = make_uint4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<uint4 *>(p + b + 4) = make_uint4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanPer; k++)
            if (b + k < nb) p[b + k] = v[k];
    }
}

// Exclusive block scan (1024 threads) of v; *total gets the sum.  Two barriers.
template <typename T>
__device__ __forceinline__ T scan1024(T v, T *s_w, T *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T o = __shfl_up_sync(kFullMask, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const T x = s_w[lane];
        T xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T o = __shfl_up_sync(kFullMask, xi, d);
            if (lane >= d) xi += o;
        }
        s_w[lane] = xi - x;
        if (lane == 31) s_w[32] = xi;
    }
    __syncthreads();
    *total = s_w[32];
    return s_w[wid] + inc - v;
}

// Exclusive block scan (256 threads) of v; *total gets the sum.  Two
// barriers; every warp writes only its own slot of s_w before the first one,
// so consecutive calls may share s_w.
template <typename T>
__device__ __forceinline__ T scan256(T v, T *s_w, T *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T o = __shfl_up_sync(kFullMask, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const T x = lane < kScanThreads / 32 ? s_w[lane] : T(0);
        T xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T o = __shfl_up_sync(kFullMask, xi, d);
            if (lane >= d) xi += o;
        }
        if (lane < kScanThreads / 32) s_w[lane] = xi - x;
        if (lane == kScanThreads / 32 - 1) s_w[kScanThreads / 32] = xi;
    }
    __syncthreads();
    *total = s_w[kScanThreads / 32];
    return s_w[wid] + inc - v;
}

// Part 2a: per chunk of kScanChunk blocks, the entries of each side and the
// blocks that hold both sides -> part[3 c .. 3 c + 2].
__global__ void __launch_bounds__(kScanThreads) k_bscan_part(BArgs a, unsigned long long *__restrict__ part) {
    __shared__ unsigned long long s_w64[kScanThreads / 32 + 1];
    __shared__ unsigned s_w32[kScanThreads / 32 + 1];
    const int nb = a.nbt;
    const int b0 = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    unsigned vr[kScanPer], vs[kScanPer];
    load8(a.btot, b0, nb, vr);
    load8(a.btot + nb, b0, nb, vs);
    unsigned long long sr = 0, ss = 0;
    unsigned sf = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        sr += vr[k];
        ss += vs[k];
        sf += (vr[k] > 0 && vs[k] > 0);
    }
    unsigned long long tr, ts;
    unsigned tf;
    scan256(sr, s_w64, &tr);
    scan256(ss, s_w64, &ts);
    scan256(sf, s_w32, &tf);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = tr;
        part[3 * blockIdx.x + 1] = ts;
        part[3 * blockIdx.x + 2] = tf;
    }
}

// Part 2b (one CTA): exclusive scan of the chunk sums in place; the totals.
__global__ void __launch_bounds__(1024) k_bscan_top(BArgs a, unsigned long long *__restrict__ part, int nch) {
    __shared__ unsigned long long s_w64[33];
    const int nb = a.nbt;
    unsigned long long cr = 0, cs = 0, cf = 0;
    for (int c0 = 0; c0 < nch; c0 += 1024) {
        const int c = c0 + threadIdx.x;
        const unsigned long long r = c < nch ? part[3 * c] : 0ull, sv = c < nch ? part[3 * c + 1] : 0ull,
                                 f = c < nch ? part[3 * c + 2] : 0ull;
        unsigned long long tr, ts, tf;
        const unsigned long long er = cr + scan1024(r, s_w64, &tr);
        const unsigned long long es = cs + scan1024(sv, s_w64, &ts);
        const unsigned long long ef = cf + scan1024(f, s_w64, &tf);
        if (c < nch) {
            part[3 * c] = er;
            part[3 * c + 1] = es;
            part[3 * c + 2] = ef;
        }
        cr += tr;
        cs += ts;
        cf += tf;
    }
    if (threadIdx.x == 0) {
        a.bo_r[nb] = (unsigned)cr;
        a.bo_s[nb] = (unsigned)cs;
        a.st->e_r = cr;
        a.st->e_s = cs;
        if (cr > a.cap_r || cs > a.cap_s) atomicOr(&a.st->err, kErrEntCap);
        a.st->nchunks = (unsigned)cf;
        if (a.jfirst) a.jfirst[a.nj] = (unsigned)cf;
    }
}

// Part 2c: every chunk's blocks -> block starts (and shared cursors), work
// items with their ranges and join, first item of every join.
__global__ void __launch_bounds__(kScanThreads) k_bscan_fill(BArgs a, const unsigned long long *__restrict__ part) {
    __shared__ unsigned long long s_w64[kScanThreads / 32 + 1];
    __shared__ unsigned s_w32[kScanThreads / 32 + 1];
    __shared__ int s_boff[kMaxJoins];
    const int nb = a.nbt;
    if (a.nj > 1)
        for (int j = threadIdx.x; j < a.nj; j += kScanThreads) s_boff[j] = a.jd[j].boff;
    const int b0 = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    unsigned vr[kScanPer], vs[kScanPer];
    load8(a.btot, b0, nb, vr);
    load8(a.btot + nb, b0, nb, vs);
    unsigned long long sr = 0, ss = 0;
    unsigned sf = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        sr += vr[k];
        ss += vs[k];
        sf += (vr[k] > 0 && vs[k] > 0);
    }
    unsigned long long tr, ts;
    unsigned tf;
    unsigned long long pr = part[3 * blockIdx.x] + scan256(sr, s_w64, &tr);
    unsigned long long ps = part[3 * blockIdx.x + 1] + scan256(ss, s_w64, &ts);
    unsigned idx = (unsigned)part[3 * blockIdx.x + 2] + scan256(sf, s_w32, &tf);
    unsigned orr[kScanPer], oss[kScanPer];
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        orr[k] = (unsigned)pr;
        oss[k] = (unsigned)ps;
        pr += vr[k];
        ps += vs[k];
    }
    store8(a.bo_r, b0, nb, orr);
    store8(a.bo_s, b0, nb, oss);
    if (a.cur) {
        store8(a.cur, b0, nb, orr);
        store8(a.cur + nb, b0, nb, oss);
    }
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        const int b = b0 + k;
        if (b >= nb) break;
        int lo = 0;
        if (a.nj > 1) {   // join of block b: the last join whose first block is <= b
            int hi = a.nj;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_boff[mid] <= b) lo = mid;
                else hi = mid;
            }
            if (a.jfirst && s_boff[lo] == b) a.jfirst[lo] = idx;
        } else if (a.jfirst && b == 0) {
            a.jfirst[0] = idx;
        }
        // more entries than every tile of the block could hold in shared
        // memory (fine_cap per tile: the block join's, or the stripe
        // kernel's): some tile exceeds it (each entry covers a tile of its
        // block), and the join needs the single-level path
        {
            const unsigned long long G = (unsigned long long)(a.nj > 1 ? a.jd[lo].G : (a.G > 0 ? a.G : a.jd[0].G));
            if ((unsigned long long)vr[k] + vs[k] > (unsigned long long)a.fine_cap * G * G)
                atomicOr(&a.st->need_direct, 1);
        }
        if (vr[k] > 0 && vs[k] > 0 && SJ_IN(a.st, idx, nb)) {
            a.items[idx] = (unsigned)b;
            a.imeta[idx] = make_uint4((unsigned)b, orr[k], vr[k], oss[k]);
            a.ins[idx] = vs[k];
            if (a.ijoin) a.ijoin[idx] = (unsigned)lo;
            idx++;
        }
    }
}

// Pairs before every join's first item (two-pass offsets), nj + 1 values.
__global__ void k_join_offsets(BArgs a, const unsigned long long *__restrict__ poff,
                               unsigned long long *__restrict__ joff) {
    const unsigned n = a.st->nchunks;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= a.nj; j += gridDim.x * blockDim.x) {
        const unsigned f = a.jfirst[j];
        joff[j] = f < n ? poff[f] : a.st->npairs;
    }
}

// Debug build: slot pos of block key kb (side * nbt + block) lies in that
// block's run of the L1 array, [block start, block start + block total).
__device__ __forceinline__ bool l1_slot_ok(const BArgs &a, unsigned kb, unsigned pos) {
#if SJ_CHECK
    if (!SJ_IN(a.st, kb, 2ull * (unsigned)a.nbt)) return false;
    const unsigned side = kb >= (unsigned)a.nbt, b = kb - side * (unsigned)a.nbt;
    const long long start = side ? a.bo_s[b] : a.bo_r[b];
    return SJ_IN(a.st, (long long)pos - start, a.btot[kb]);
#else
    (void)a;
    (void)kb;
    (void)pos;
    return true;
#endif
}

// L1 write: the same slice per CTA as k_bcount; shared cursors start at
// block start + this CTA's prefix.
template <int PTS>
__global__ void __launch_bounds__(kL1Threads) k_bscatter(BArgs a) {
    extern __shared__ unsigned cur[];   // 2 * NB
    if (block_skip_blocked(a.st)) return;
    const int NB2 = 2 * a.nb;
    const unsigned *row = a.H + (size_t)blockIdx.x * NB2;
    for (int k = threadIdx.x; k < NB2; k += kL1Threads)
        cur[k] = row[k] + (k < a.nb ? a.bo_r[k] : a.bo_s[k - a.nb]);
    __syncthreads();
    const long long n = a.nR + a.nS;
    const long long q = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * q, i1 = min(n, i0 + q);
    for (long long base = i0 + threadIdx.x; base < i1; base += 4ll * kL1Threads) {
        float4 m[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const long long i = base + (long long)u * kL1Threads;
            if (i < i1) {
                if constexpr (PTS) m[u] = load_square(i < a.nR ? a.R : a.S, i < a.nR ? i : i - a.nR, a.h);
                else m[u] = ld_stream(i < a.nR ? a.R + i : a.S + (i - a.nR));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const long long i = base + (long long)u * kL1Threads;
            if (i >= i1) break;
            float4 v = m[u];
            if (!rect_ok(v)) continue;
            v.x = __fadd_rn(v.x, 0.0f);
            v.y = __fadd_rn(v.y, 0.0f);
            v.z = __fadd_rn(v.z, 0.0f);
            v.w = __fadd_rn(v.w, 0.0f);
            const int side = i >= a.nR;
            const unsigned id = (unsigned)(side ? i - a.nR : i);
            const int cx0 = cell_of(v.x, a.g.x0, a.g.gx, a.g.nx), cx1 = cell_of(v.z, a.g.x0, a.g.gx, a.g.nx);
            const int cy0 = cell_of(v.y, a.g.y0, a.g.gy, a.g.ny), cy1 = cell_of(v.w, a.g.y0, a.g.gy, a.g.ny);
            const uint4 tail = make_uint4(id, (unsigned)cx0 | ((unsigned)cx1 << 16),
                                          (unsigned)cy0 | ((unsigned)cy1 << 16), 0u);
            BEnt *dst = side ? a.bent_s : a.bent_r;
            const unsigned long long cap = side ? a.cap_s : a.cap_r;
            unsigned *c = cur + side * a.nb;
            const int bx0 = div_g(cx0, a), bx1 = div_g(cx1, a), by0 = div_g(cy0, a), by1 = div_g(cy1, a);
            for (int by = by0; by <= by1; by++)
                for (int bx = bx0; bx <= bx1; bx++) {
                    const unsigned pos = atomicAdd(c + by * a.bx + bx, 1u);
                    if (pos < cap && l1_slot_ok(a, (unsigned)(side * a.nbt + by * a.bx + bx), pos))
                        store_bent(dst + pos,
                                   make_uint4(__float_as_uint(v.x), __float_as_uint(v.y), __float_as_uint(v.z),
                                              __float_as_uint(v.w)),
                                   tail);
                }
        }
    }
}

// L1 write, shared cursors: every CTA appends to one run per block through a
// global cursor (lanes of a warp that hit the same block take their slots
// with one atomic), so each block's run is filled front to back by all CTAs
// together and L2 merges the 32-byte entries into whole lines before they
// reach DRAM.
// Join of global input index i (binary search over the joins' first
// indices, kept in shared memory).
__device__ __forceinline__ int join_of(const long long *jin, int nj, long long i) {
    int lo = 0, hi = nj;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (jin[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int div_gj(int x, const JoinDesc &d) {
    return d.G == 1 ? x : (int)__umulhi((unsigned)x, d.gmul);
}

// Every thread takes kScatterU rectangles per step in phases: all loads,
// then cells and block keys, then the warp-aggregated cursor atomics of
// the first blocks, then the stores, so that the DRAM loads and the L2
// atomic round trips of the kScatterU rectangles overlap.
constexpr int kScatterU = 4;
template <int PTS>
__global__ void __launch_bounds__(256) k_bscatter_shared(BArgs a) {
    extern __shared__ long long s_jin[];   // nj + 1
    if (block_skip_blocked(a.st)) return;
    for (int j = threadIdx.x; j < a.nj; j += 256) s_jin[j] = a.jd[j].in_off;
    if (threadIdx.x == 0) s_jin[a.nj] = a.jd[a.nj - 1].in_off + a.jd[a.nj - 1].nR + a.jd[a.nj - 1].nS;
    __syncthreads();
    const long long n = s_jin[a.nj];
    const unsigned lane = threadIdx.x & 31;
    for (long long base = blockIdx.x * 256ll * kScatterU + threadIdx.x; base - threadIdx.x < n;
         base += 256ll * kScatterU * gridDim.x) {
        float4 v[kScatterU];
        int jj[kScatterU];
        unsigned idx[kScatterU];   // index in its side | side << 31
        bool ok[kScatterU];
#pragma unroll
        for (int u = 0; u < kScatterU; u++) {   // loads
            const long long i = base + u * 256;
            ok[u] = i < n;
            jj[u] = ok[u] ? (a.nj == 1 ? 0 : join_of(s_jin, a.nj, i)) : 0;
            const JoinDesc &d = a.jd[jj[u]];
            const long long li = i - s_jin[jj[u]];
            const int side = li >= d.nR;
            idx[u] = (unsigned)(side ? li - d.nR : li) | ((unsigned)side << 31);
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok[u]) {
                if constexpr (PTS) v[u] = load_square(side ? d.S : d.R, side ? li - d.nR : li, d.h);
                else v[u] = ld_stream(side ? d.S + (li - d.nR) : d.R + li);
            }
        }
        unsigned cxp[kScatterU], cyp[kScatterU], key[kScatterU], pos0[kScatterU], peers[kScatterU];
#pragma unroll
        for (int u = 0; u < kScatterU; u++) {   // cells, first block, cursor atomic
            const JoinDesc &d = a.jd[jj[u]];
            if (ok[u] && !rect_ok(v[u])) ok[u] = false;
            v[u].x = __fadd_rn(v[u].x, 0.0f);
            v[u].y = __fadd_rn(v[u].y, 0.0f);
            v[u].z = __fadd_rn(v[u].z, 0.0f);
            v[u].w = __fadd_rn(v[u].w, 0.0f);
            int cx0 = 0, cx1 = 0, cy0 = 0, cy1 = 0;
            if (ok[u]) {
                cx0 = cell_of(v[u].x, d.g.x0, d.g.gx, d.g.nx);
                cx1 = cell_of(v[u].z, d.g.x0, d.g.gx, d.g.nx);
                cy0 = cell_of(v[u].y, d.g.y0, d.g.gy, d.g.ny);
                cy1 = cell_of(v[u].w, d.g.y0, d.g.gy, d.g.ny);
            }
            cxp[u] = (unsigned)cx0 | ((unsigned)cx1 << 16);
            cyp[u] = (unsigned)cy0 | ((unsigned)cy1 << 16);
            const unsigned cb = (idx[u] >> 31) * (unsigned)a.nbt + (unsigned)d.boff;
            key[u] = ok[u] ? cb + (unsigned)(div_gj(cy0, d) * d.bx + div_gj(cx0, d)) : 0xffffffffu;
            peers[u] = __match_any_sync(0xffffffffu, key[u]);
            pos0[u] = 0;
            if (ok[u] && (int)lane == __ffs(peers[u]) - 1 && SJ_IN(a.st, key[u], 2ull * (unsigned)a.nbt))
                pos0[u] = atomicAdd(a.cur + key[u], (unsigned)__popc(peers[u]));
        }
#pragma unroll
        for (int u = 0; u < kScatterU; u++) {   // slots, stores (further blocks: one atomic each)
            pos0[u] = __shfl_sync(0xffffffffu, pos0[u], __ffs(peers[u]) - 1) + __popc(peers[u] & ((1u << lane) - 1u));
            if (!ok[u]) continue;
            const JoinDesc &d = a.jd[jj[u]];
            const int side = idx[u] >> 31;
            const int cx0 = cxp[u] & 0xffff, cx1 = cxp[u] >> 16, cy0 = cyp[u] & 0xffff, cy1 = cyp[u] >> 16;
            const uint4 head = make_uint4(__float_as_uint(v[u].x), __float_as_uint(v[u].y), __float_as_uint(v[u].z),
                                          __float_as_uint(v[u].w));
            const uint4 tail = make_uint4(idx[u] & 0x7fffffffu, cxp[u], cyp[u], 0u);
            BEnt *dst = side ? a.bent_s : a.bent_r;
            const unsigned long long cap = side ? a.cap_s : a.cap_r;
            const unsigned cb = (unsigned)side * (unsigned)a.nbt + (unsigned)d.boff;
            const int bx0 = div_gj(cx0, d), bx1 = div_gj(cx1, d), by0 = div_gj(cy0, d), by1 = div_gj(cy1, d);
            for (int by = by0; by <= by1; by++)
                for (int bx = bx0; bx <= bx1; bx++) {
                    const unsigned kb = cb + by * d.bx + bx;
                    const unsigned pos = (by == by0 && bx == bx0) ? pos0[u] : atomicAdd(a.cur + kb, 1u);
                    if (pos >= cap) atomicOr(&a.st->err, kErrEntCap);
                    else if (l1_slot_ok(a, kb, pos)) store_bent(dst + pos, head, tail);
                }
        }
    }
}

// L1 count with global per-block totals (any number of blocks; batches):
// lanes of a warp that hit the same block add with one atomic.
__global__ void __launch_bounds__(256) k_bcount_global(BArgs a) {
    extern __shared__ long long s_jin[];   // nj + 1
    for (int j = threadIdx.x; j < a.nj; j += 256) s_jin[j] = a.jd[j].in_off;
    if (threadIdx.x == 0) s_jin[a.nj] = a.jd[a.nj - 1].in_off + a.jd[a.nj - 1].nR + a.jd[a.nj - 1].nS;
    __syncthreads();
    const long long n = s_jin[a.nj];
    int bad = 0;
    for (long long base = blockIdx.x * 256ll + threadIdx.x; base - threadIdx.x < n; base += 256ll * gridDim.x) {
        const long long i = base;
        bool valid = i < n;
        const int j = valid ? (a.nj == 1 ? 0 : join_of(s_jin, a.nj, i)) : 0;
        const JoinDesc &d = a.jd[j];
        const long long li = i - s_jin[j];
        const int side = li >= d.nR;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) v = ld_stream(side ? d.S + (li - d.nR) : d.R + li);
        if (valid && !rect_ok(v)) {
            valid = false;
            bad = 1;
        }
        int bx0 = 0, bx1 = -1, by0 = 0, by1 = -1;
        if (valid) {
            bx0 = div_gj(cell_of(v.x, d.g.x0, d.g.gx, d.g.nx), d);
            bx1 = div_gj(cell_of(v.z, d.g.x0, d.g.gx, d.g.nx), d);
            by0 = div_gj(cell_of(v.y, d.g.y0, d.g.gy, d.g.ny), d);
            by1 = div_gj(cell_of(v.w, d.g.y0, d.g.gy, d.g.ny), d);
        }
        const unsigned cb = (unsigned)side * (unsigned)a.nbt + (unsigned)d.boff;
        const unsigned key = valid ? cb + (unsigned)(by0 * d.bx + bx0) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (valid && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(a.btot + key, (unsigned)__popc(peers));
        if (!valid) continue;
        for (int by = by0; by <= by1; by++)
            for (int bx = bx0; bx <= bx1; bx++)
                if (by != by0 || bx != bx0) atomicAdd(a.btot + cb + by * d.bx + bx, 1u);
    }
    if (bad) atomicOr(&a.st->err, kErrBadRect);
}

// L1 count of a batch with per-join shared histograms: every CTA takes a
// contiguous slice of the batch's input, so it meets only the joins whose
// input ranges overlap the slice; it counts each join's part of the slice in
// a shared histogram of that join's blocks and then adds the non-zero counts
// to the global totals (one atomic per touched block and CTA instead of one
// per rectangle).  A join with more blocks than the histogram holds counts
// with global atomics.
constexpr int kLocalHist = 16384;   // counters: 2 per block (R, S)
constexpr int kLocalThreads = 512;
constexpr int kLocalU = 4;          // loads in flight per thread
__global__ void __launch_bounds__(kLocalThreads) k_bcount_local(BArgs a) {
    extern __shared__ long long s_dyn[];
    long long *s_jin = s_dyn;                                         // nj + 1
    unsigned *hist = reinterpret_cast<unsigned *>(s_dyn + a.nj + 1);   // kLocalHist
    for (int j = threadIdx.x; j < a.nj; j += kLocalThreads) s_jin[j] = a.jd[j].in_off;
    if (threadIdx.x == 0) s_jin[a.nj] = a.jd[a.nj - 1].in_off + a.jd[a.nj - 1].nR + a.jd[a.nj - 1].nS;
    __syncthreads();
    const long long n = s_jin[a.nj];
    const long long q = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * q, i1 = min(n, i0 + q);
    int bad = 0;
    const int j0 = i0 < i1 ? join_of(s_jin, a.nj, i0) : 0;
    const int j1 = i0 < i1 ? join_of(s_jin, a.nj, i1 - 1) : -1;
    for (int j = j0; j <= j1; j++) {   // block-uniform
        const long long lo = max(i0, s_jin[j]), hi = min(i1, s_jin[j + 1]);
        if (lo >= hi) continue;
        const JoinDesc &d = a.jd[j];
        const long long jin = s_jin[j], nRj = d.nR;
        const float4 *Rj = d.R, *Sj = d.S;
        const GridDev g = d.g;
        const int jbx = d.bx, nbj = d.bx * d.by;
        const bool local = 2 * nbj <= kLocalHist;
        if (local) {
            for (int k = threadIdx.x; k < 2 * nbj; k += kLocalThreads) hist[k] = 0;
            __syncthreads();
        }
        for (long long base = lo + threadIdx.x; base < hi; base += (long long)kLocalU * kLocalThreads) {
            float4 m[kLocalU];
#pragma unroll
            for (int u = 0; u < kLocalU; u++) {
                const long long i = base + (long long)u * kLocalThreads;
                if (i < hi) m[u] = ld_stream(i - jin < nRj ? Rj + (i - jin) : Sj + (i - jin - nRj));
            }
#pragma unroll
            for (int u = 0; u < kLocalU; u++) {
                const long long i = base + (long long)u * kLocalThreads;
                if (i >= hi) break;
                if (!rect_ok(m[u])) {
                    bad = 1;
                    continue;
                }
                const int side = i - jin >= nRj;
                const int bx0 = div_gj(cell_of(m[u].x, g.x0, g.gx, g.nx), d);
                const int bx1 = div_gj(cell_of(m[u].z, g.x0, g.gx, g.nx), d);
                const int by0 = div_gj(cell_of(m[u].y, g.y0, g.gy, g.ny), d);
                const int by1 = div_gj(cell_of(m[u].w, g.y0, g.gy, g.ny), d);
                for (int by = by0; by <= by1; by++)
                    for (int bx = bx0; bx <= bx1; bx++) {
                        const int b = by * jbx + bx;
                        if (!SJ_IN(a.st, b, nbj)) continue;
                        if (local) atomicAdd(hist + side * nbj + b, 1u);
                        else atomicAdd(a.btot + (unsigned)side * (unsigned)a.nbt + (unsigned)d.boff + (unsigned)b, 1u);
                    }
            }
        }
        if (local) {
            __syncthreads();
            for (int k = threadIdx.x; k < 2 * nbj; k += kLocalThreads) {
                const unsigned c = hist[k];
                const int side = k >= nbj;
                if (c) atomicAdd(a.btot + (unsigned)side * (unsigned)a.nbt + (unsigned)d.boff + (unsigned)(k - side * nbj), c);
            }
            __syncthreads();   // the next join clears the histogram
        }
    }
    if (bad) atomicOr(&a.st->err, kErrBadRect);
}

// ---------------------------------------------------------------------------
// L2: fused tile partition + per-tile sort + sweep of one block per CTA step.
// ---------------------------------------------------------------------------
struct BJSmem {
    unsigned cnt[2][kMaxFine];       // entries per tile of the block
    unsigned off[2][kMaxFine + 1];   // band offsets; after the scatter: segment ends
    unsigned key[kFineCap];          // x_l keys; after the ranking: positions in x_l order per segment
    float4 mbr[kFineCap];            // the band's entries, grouped by tile segment
    unsigned id[kFineCap];
    unsigned short tile[kFineCap];   // band-local tile of each position
    unsigned short ord[kFineCap];    // x_l order of every tile segment (positions of its entries)
    unsigned short band[kMaxFine + 2];
    int2 pbuf[kPairBuf];             // one-pass: the block's pairs before its reservation
    unsigned axis[kMaxFine / 32];    // adaptive sweep axis: bit per tile, 1 = y
};

// Adaptive sweep axis (Sec. 3.3, Eq. 2): during the count step, before any
// entry is placed, key[] .. id[] hold the histograms of every tile of the
// block: [tile][side][axis][k = 8 buckets] as 16-bit counters, two to a word
// (16 words per tile).  A tile holds at most kFineCap entries when it is
// joined (a larger one sends the join to the single-level path), so no
// counter of a joined tile can carry into its neighbour.
constexpr int kAxisBuckets = 8;
constexpr int kHistWords = 16;
static_assert(offsetof(BJSmem, id) + sizeof(BJSmem::id) - offsetof(BJSmem, key) >=
                  sizeof(unsigned) * kHistWords * kMaxFine,
              "per-tile histograms must fit in key[] .. id[]");
static_assert(kFineCap < 65536, "16-bit histogram counters");
static_assert(sizeof(BJSmem) <= 111 * 1024, "two block-join CTAs (and their static shared memory) per SM");

// Bucket index at 8x the tile resolution: floor(8 t) for the cell-function
// value t = (v - g0) * ginv (both rounded to float32, as in cell_of; 8 t is
// exact), clamped like the cells to [0, 8 n - 1].  Within tile c the bucket
// is this minus 8 c.
__device__ __forceinline__ int cell8_of(float v, float g0, float ginv, int n) {
    const float t = __fmul_rn(__fsub_rn(v, g0), ginv);
    const float f = floorf(t * 8.0f);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(8 * n - 1)) return 8 * n - 1;
    return (int)f;
}

// Per-row entry lists of a block staged in several bands: entry e (R: e <
// nr1, S: e - nr1) appears in the list of every tile row it covers.  Row y
// has room for the sum of its tile counts (an upper bound on the entries
// covering it), at off[y] of the block's pool slice; pre[] is the exclusive
// prefix of the rows' actual lengths.
struct RowLists {
    unsigned off[kMaxG + 1];
    unsigned pre[kMaxG + 1];
    unsigned cur[kMaxG];
    unsigned *pool;
    int on;
};

struct BlockCtx {
    int cxb, cyb, gw, gh, ntl;
    const unsigned *axis;  // adaptive sweep axis: bit lt set = tile lt swept along y (else nullptr)
    int gbda;              // grouping-based duplicate avoidance instead of the test of Eq. 1
    unsigned r0, nr1, s0, ns1;
    const BEnt *er, *es;   // the block's R and S entries (shared-memory copy or global)
    Stats *st;             // error word of the bounds checks (debug build)
};

// Grouping-based duplicate avoidance (GBDA, the alternative to Eq. 1 that
// follows it in the paper): the entries of a tile fall into four classes by
// the two flag bits, A (first column and first row of the rectangle), B
// (first column only), C (first row only) and D (neither).  A pair is
// reported by this tile exactly when one of the two is in its first column
// and one in its first row, so only the class combinations A-any, any-A, B-C
// and C-B (9 of 16) are joined, with no test per pair.  Segments are sorted
// by (class rank, x_l) with the ranks D = 0, B = 1, A = 2, C = 3: the classes
// a pivot joins are then one contiguous range of ranks, [2, 2] for D, [2, 3]
// for B, [1, 2] for C and [0, 3] for A.  The rank is kept in bits 14-15 of
// the entry's tile field.
__device__ __forceinline__ unsigned gbda_rank(unsigned flags2) { return (0x2310u >> (4 * flags2)) & 3u; }
__device__ __forceinline__ unsigned gbda_lo(unsigned flags2) { return (0x0122u >> (4 * flags2)) & 3u; }
__device__ __forceinline__ unsigned gbda_hi(unsigned flags2) { return (0x3232u >> (4 * flags2)) & 3u; }
constexpr unsigned kTileMask = 0x3FFFu;

// Write an entry of the block (side, MBR words hd, tail words t) into every
// tile of [ta, tb) it overlaps (rows row_a..row_b of the block).  With
// row >= 0 the entry comes from the list of that row and is taken only there
// if it is its first row in the band.  A tile swept along y (adaptive axis)
// gets its MBRs with the axes exchanged: the sort key, the forward scan and
// the test then run along y unchanged, and the intersection test is
// symmetric in the two axes, so the pairs are the same.
__device__ __forceinline__ void place_entry(BJSmem &sm, const BlockCtx &bc, int side, const uint4 &hd,
                                            const uint4 &t, int ta, int tb, int row_a, int row_b, int row,
                                            int nRb, int nb) {
    const int cx0 = t.y & 0xffff, cx1 = t.y >> 16, cy0 = t.z & 0xffff, cy1 = t.z >> 16;
    const int ly0 = max(cy0 - bc.cyb, row_a), ly1 = min(cy1 - bc.cyb, row_b);
    if (ly0 > ly1 || (row >= 0 && ly0 != row)) return;
    const int lx0 = max(cx0 - bc.cxb, 0), lx1 = min(cx1 - bc.cxb, bc.gw - 1);
    const float4 mx = make_float4(__uint_as_float(hd.x), __uint_as_float(hd.y), __uint_as_float(hd.z),
                                  __uint_as_float(hd.w));
    const float4 my = make_float4(mx.y, mx.x, mx.w, mx.z);
    for (int ly = ly0; ly <= ly1; ly++)
        for (int lx = lx0; lx <= lx1; lx++) {
            const int lt = ly * bc.gw + lx;
            if (lt < ta || lt >= tb) continue;
            const int j = lt - ta;
            const unsigned pos = atomicAdd(&sm.off[side][j], 1u);
            // the band's R entries are [0, nRb), its S entries [nRb, nb)
            if (!SJ_IN(bc.st, (int)pos - (side ? nRb : 0), side ? nb - nRb : nRb)) continue;
            const unsigned flags = (lx + bc.cxb == cx0 ? kFlagCol : 0u) | (ly + bc.cyb == cy0 ? kFlagRow : 0u);
            const bool swap = bc.axis && ((bc.axis[lt >> 5] >> (lt & 31)) & 1u);
            const float4 mb = swap ? my : mx;
            sm.key[pos] = xkey(mb.x);
            sm.mbr[pos] = mb;
            sm.id[pos] = t.x | flags;
            sm.tile[pos] = (unsigned short)(bc.gbda ? (unsigned)j | (gbda_rank(flags >> 30) << 14) : (unsigned)j);
        }
}

__device__ __forceinline__ const uint4 *entry_words(const BlockCtx &bc, int e) {
    return reinterpret_cast<const uint4 *>(e >= (int)bc.nr1 ? bc.es + (e - bc.nr1) : bc.er + e);
}

// Offsets of the band [ta, tb): sm.off[0][j] / sm.off[1][j] = start of tile
// ta + j's R / S segment (S segments after all R segments); nRb, nSb = the
// band's entries per side.  Ends with a barrier.
__device__ __forceinline__ void band_offsets(BJSmem &sm, int ta, int tb, int &nRb, int &nSb) {
    const int NT = kBJThreads;
    const int nt = tb - ta;
    // packed exclusive scan of (R count | S count << 32) over the band's tiles
    __shared__ unsigned long long s_warp[kBJThreads / 32];
    __shared__ unsigned long long s_tot;
    const int per = (nt + NT - 1) / NT;
    const int j0 = threadIdx.x * per;
    unsigned long long sum = 0;
    for (int k = 0; k < per; k++) {
        const int j = j0 + k;
        if (j < nt) sum += (unsigned long long)sm.cnt[0][ta + j] | ((unsigned long long)sm.cnt[1][ta + j] << 32);
    }
    unsigned long long inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long o = __shfl_up_sync(kFullMask, inc, d);
        if ((threadIdx.x & 31) >= d) inc += o;
    }
    if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned long long x = threadIdx.x < NT / 32 ? s_warp[threadIdx.x] : 0ull;
        unsigned long long xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long o = __shfl_up_sync(kFullMask, xi, d);
            if (threadIdx.x >= (unsigned)d) xi += o;
        }
        if (threadIdx.x < NT / 32) s_warp[threadIdx.x] = xi - x;
        if (threadIdx.x == NT / 32 - 1) s_tot = xi;
    }
    __syncthreads();
    const unsigned long long tot = s_tot;
    nRb = (int)(tot & 0xffffffffull);
    nSb = (int)(tot >> 32);
    unsigned long long run = s_warp[threadIdx.x >> 5] + inc - sum;
    for (int k = 0; k < per; k++) {
        const int j = j0 + k;
        if (j < nt) {
            sm.off[0][j] = (unsigned)(run & 0xffffffffull);
            sm.off[1][j] = (unsigned)nRb + (unsigned)(run >> 32);
            run += (unsigned long long)sm.cnt[0][ta + j] | ((unsigned long long)sm.cnt[1][ta + j] << 32);
        }
    }
    __syncthreads();
}

// Scatter of the band's entries into its tile segments (entries from the row
// lists when rl is given, else from the block's whole L1 range; every thread
// loads kStageU entries before placing them), then the x_l order of every
// segment.  Needs band_offsets first; results live in sm.
constexpr int kStageU = 1;
__device__ __forceinline__ void band_fill(BJSmem &sm, const BlockCtx &bc, int ta, int tb, int nRb, int nSb,
                                          const RowLists *rl) {
    const int NT = kBJThreads;
    // scatter the block's entries into the band's tile segments
    const int row_a = ta / bc.gw, row_b = (tb - 1) / bc.gw;
    if (rl) {
        const unsigned i0 = rl->pre[row_a], i1 = rl->pre[row_b + 1];
        for (unsigned ib = i0 + threadIdx.x; ib < i1; ib += kStageU * NT) {
            int e[kStageU], row[kStageU];
            uint4 hd[kStageU], t[kStageU];
#pragma unroll
            for (int u = 0; u < kStageU; u++) {
                const unsigned i = ib + u * NT;
                e[u] = -1;
                if (i < i1) {
                    int lo = row_a, hi = row_b;   // the row holding item i: last y with pre[y] <= i
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (rl->pre[mid] <= i) lo = mid;
                        else hi = mid - 1;
                    }
                    row[u] = lo;
                    e[u] = (int)rl->pool[rl->off[lo] + (i - rl->pre[lo])];
                    if (!SJ_IN(bc.st, e[u], bc.nr1 + bc.ns1)) e[u] = -1;
                }
            }
#pragma unroll
            for (int u = 0; u < kStageU; u++)
                if (e[u] >= 0) {
                    load_bent(entry_words(bc, e[u]), hd[u], t[u]);
                }
#pragma unroll
            for (int u = 0; u < kStageU; u++)
                if (e[u] >= 0)
                    place_entry(sm, bc, e[u] >= (int)bc.nr1, hd[u], t[u], ta, tb, row_a, row_b, row[u], nRb,
                                nRb + nSb);
        }
    } else {
        const int n1 = (int)(bc.nr1 + bc.ns1);
        for (int eb = threadIdx.x; eb < n1; eb += kStageU * NT) {
            uint4 hd[kStageU], t[kStageU];
#pragma unroll
            for (int u = 0; u < kStageU; u++)
                if (eb + u * NT < n1) {
                    load_bent(entry_words(bc, eb + u * NT), hd[u], t[u]);
                }
#pragma unroll
            for (int u = 0; u < kStageU; u++)
                if (eb + u * NT < n1)
                    place_entry(sm, bc, eb + u * NT >= (int)bc.nr1, hd[u], t[u], ta, tb, row_a, row_b, -1, nRb,
                                nRb + nSb);
        }
    }
    __syncthreads();
    // sort every tile segment by x_l: the rank of each position among its
    // segment (ties by position) gives ord[segment start + rank] = position,
    // i.e. after this step ord[] holds the x_l order of every segment and
    // the entries themselves stay where the scatter put them
    const int nb = nRb + nSb;
    constexpr int KP = kFineCap / kBJThreads;
#pragma unroll
    for (int q = 0; q < KP; q++) {
        const int pidx = threadIdx.x + q * NT;
        if (pidx < nb) {
            const int side = pidx >= nRb;
            const unsigned tw = sm.tile[pidx];
            const int j = (int)(tw & kTileMask);
            const int s0 = j ? (int)sm.off[side][j - 1] : (side ? nRb : 0);
            const int s1 = (int)sm.off[side][j];
            if (!SJ_IN(bc.st, s1 - 1, nb) || !SJ_IN(bc.st, pidx - s0, s1 - s0)) continue;
            const unsigned k0 = sm.key[pidx];
            int r = 0;
            if (bc.gbda) {   // order by (class rank, x_l)
                const unsigned c0 = tw >> 14;
                for (int qq = s0; qq < s1; qq++) {
                    const unsigned kq = sm.key[qq], cq = (unsigned)sm.tile[qq] >> 14;
                    r += (cq < c0) | ((cq == c0) & ((kq < k0) | ((kq == k0) & (qq < pidx))));
                }
            } else {
                for (int qq = s0; qq < s1; qq++) {
                    const unsigned kq = sm.key[qq];
                    r += (kq < k0) | ((kq == k0) & (qq < pidx));
                }
            }
            sm.ord[s0 + r] = (unsigned short)pidx;
        }
    }
    __syncthreads();
}

// All steps of one band [ta, tb): offsets (unless the band is the whole
// block and they were computed already: entries nR0, nS0), scatter, x_l
// order.
__device__ __forceinline__ void stage_band(BJSmem &sm, const BlockCtx &bc, int ta, int tb, bool have_offsets,
                                        int nR0, int nS0, const RowLists *rl, int &nRb, int &nSb) {
    if (have_offsets) {
        nRb = nR0;
        nSb = nS0;
    } else {
        band_offsets(sm, ta, tb, nRb, nSb);
    }
    band_fill(sm, bc, ta, tb, nRb, nSb, rl);
}

// Candidate range of pivot p (any position) in the other side of its tile:
// ranks k..kend-1 of that segment's x_l order (entry sm.ord[k]).
__device__ __forceinline__ void band_pivot(const BJSmem &sm, int nRb, int p, float4 &pv, unsigned &pid, int &k,
                                           int &kend, bool &isR, Stats *st, int nb) {
    isR = p < nRb;
    const int j = (int)(sm.tile[p] & kTileMask);
    pv = sm.mbr[p];
    pid = sm.id[p];
    const int o = isR ? 1 : 0;
    int lo = j ? (int)sm.off[o][j - 1] : (o ? nRb : 0);
    int hi = (int)sm.off[o][j];
    if (!SJ_IN(st, hi - lo, (o ? nb : nRb) - lo + 1) || !SJ_IN(st, lo, nb + 1)) hi = lo;   // empty on failure
    kend = hi;
    // first x_l > pivot.x_l (R pivot) or >= pivot.x_l (S pivot), in x_l order
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float xm = sm.mbr[sm.ord[mid]].x;
        const bool right = isR ? (xm > pv.x) : (xm >= pv.x);
        if (right) hi = mid;
        else lo = mid + 1;
    }
    k = lo;
}

// Count pairs of the staged band; per-tile counts go to tile_pairs if given.
__device__ __forceinline__ unsigned band_count(const BJSmem &sm, const BlockCtx &bc, int ta, int nRb, int nSb,
                                               unsigned *tile_pairs, int nx) {
    unsigned my = 0;
    const int nb = nRb + nSb;
    if (nRb == 0 || nSb == 0) return 0;
    for (int p = threadIdx.x; p < nb; p += kBJThreads) {
        float4 pv;
        unsigned pid;
        int k, kend;
        bool isR;
        band_pivot(sm, nRb, p, pv, pid, k, kend, isR, bc.st, nb);
        unsigned c = 0;
        for (; k < kend; k++) {
            const unsigned q = SJ_AT(bc.st, sm.ord[k], nb);
            const float4 o = sm.mbr[q];
            if (o.x > pv.z) break;
            if (o.y <= pv.w && pv.y <= o.w && reported_here(pid, sm.id[q])) c++;
        }
        if (tile_pairs && c) {
            const int lt = ta + (int)(sm.tile[p] & kTileMask);
            const int gt = (bc.cyb + lt / bc.gw) * nx + bc.cxb + lt % bc.gw;
            atomicAdd(tile_pairs + gt, c);
        }
        my += c;
    }
    return my;
}

// Write the pairs of the staged band at out[base + cursor ...].
__device__ __forceinline__ void band_write(const BJSmem &sm, int nRb, int nSb, int2 *out, unsigned long long base,
                                           unsigned *s_cursor, Stats *st, unsigned long long cap) {
    const int nb = nRb + nSb;
    if (nRb == 0 || nSb == 0) return;
    const unsigned lane = threadIdx.x & 31;
    for (int pb = 0; pb < nb; pb += kBJThreads) {
        const int p = pb + threadIdx.x;
        const bool active = p < nb;
        float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned pid = 0;
        int k = 0, kend = 0;
        bool isR = true;
        if (active) band_pivot(sm, nRb, p, pv, pid, k, kend, isR, st, nb);
        bool go = active;
        for (;;) {
            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned q = 0;
            bool cand = false;
            if (go && k < kend) {
                q = SJ_AT(st, sm.ord[k], nb);
                o = sm.mbr[q];
                cand = o.x <= pv.z;
            }
            if (!__any_sync(kFullMask, cand)) break;
            go = cand;
            bool hit = false;
            int2 pr = make_int2(0, 0);
            if (cand) {
                if (o.y <= pv.w && pv.y <= o.w) {
                    const unsigned oid = sm.id[q];
                    if (reported_here(pid, oid)) {
                        hit = true;
                        pr = isR ? make_int2((int)(pid & kIdMask), (int)(oid & kIdMask))
                                 : make_int2((int)(oid & kIdMask), (int)(pid & kIdMask));
                    }
                }
                k++;
            }
            const unsigned hm = __ballot_sync(kFullMask, hit);
            if (hm) {
                const int leader = __ffs(hm) - 1;
                unsigned pos = 0;
                if ((int)lane == leader) pos = atomicAdd(s_cursor, (unsigned)__popc(hm));
                pos = __shfl_sync(kFullMask, pos, leader);
                const unsigned long long at = base + pos + __popc(hm & lanemask_lt_b());
                if (hit && SJ_IN(st, at, cap)) out[at] = pr;
            }
        }
    }
}

// Pairs of the staged band into the block's shared buffer (one-pass join):
// every hit takes the next slot of *s_pc (warp-aggregated); slots beyond the
// buffer go to the CTA's spill area (if any), slots beyond both are only
// counted.
__device__ __forceinline__ void band_collect(BJSmem &sm, int nRb, int nSb, unsigned *s_pc, int2 *spill, Stats *st) {
    const int nb = nRb + nSb;
    if (nRb == 0 || nSb == 0) return;
    for (int p = threadIdx.x; p < nb; p += kBJThreads) {
        float4 pv;
        unsigned pid;
        int k, kend;
        bool isR;
        band_pivot(sm, nRb, p, pv, pid, k, kend, isR, st, nb);
        for (; k < kend; k++) {
            const unsigned q = SJ_AT(st, sm.ord[k], nb);
            const float4 o = sm.mbr[q];
            if (o.x > pv.z) break;
            if (o.y <= pv.w && pv.y <= o.w) {
                const unsigned oid = sm.id[q];
                if (reported_here(pid, oid)) {
                    const unsigned m = __activemask();
                    const int leader = __ffs(m) - 1;
                    unsigned pos = 0;
                    if ((int)(threadIdx.x & 31) == leader) pos = atomicAdd(s_pc, (unsigned)__popc(m));
                    pos = __shfl_sync(m, pos, leader) + __popc(m & lanemask_lt_b());
                    const int2 pr = isR ? make_int2((int)(pid & kIdMask), (int)(oid & kIdMask))
                                        : make_int2((int)(oid & kIdMask), (int)(pid & kIdMask));
                    if (pos < (unsigned)kPairBuf) sm.pbuf[pos] = pr;
                    else if (spill && pos < (unsigned)(kPairBuf + kPairSpill)) spill[pos - kPairBuf] = pr;
                }
            }
        }
    }
}

// GBDA sweep of the staged band: every pivot scans, for each class of the
// other side it is joined with (a contiguous range of ranks), the entries of
// that class with x_l in (x_l, x_u] (R pivot) or [x_l, x_u] (S pivot), as in
// the pivot-parallel Algorithm 1, and reports every y-intersecting one with
// no duplicate test.  OUT: 0 = count (returns this thread's pairs, per-tile
// counts to tile_pairs if given), 1 = collect into the block's shared buffer
// and spill area (slot counter *ctr), 2 = write at out[base + *ctr ...].
template <int OUT>
__device__ __forceinline__ unsigned gbda_sweep(BJSmem &sm, const BlockCtx &bc, int ta, int nRb, int nSb,
                                               unsigned *ctr, int2 *spill, int2 *out, unsigned long long base,
                                               unsigned *tile_pairs, int nx, unsigned long long cap = ~0ull) {
    unsigned my = 0;
    const int nb = nRb + nSb;
    if (nRb == 0 || nSb == 0) return 0;
    for (int p = threadIdx.x; p < nb; p += kBJThreads) {
        const bool isR = p < nRb;
        const unsigned tw = sm.tile[p];
        const int j = (int)(tw & kTileMask);
        const float4 pv = sm.mbr[p];
        const unsigned pid = sm.id[p];
        const unsigned f = pid >> 30;
        const int o = isR ? 1 : 0;
        const int s0 = j ? (int)sm.off[o][j - 1] : (o ? nRb : 0);
        const int s1 = (int)sm.off[o][j];
        if (!SJ_IN(bc.st, s1 - s0, (o ? nb : nRb) - s0 + 1)) continue;
        unsigned c = 0;
        for (unsigned cl = gbda_lo(f); cl <= gbda_hi(f); cl++) {
            // first sorted position of class > cl, or of class cl with x_l
            // past the pivot's start
            int lo = s0, hi = s1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const unsigned q = sm.ord[mid];
                const unsigned cq = (unsigned)sm.tile[q] >> 14;
                const float xm = sm.mbr[q].x;
                const bool right = cq > cl || (cq == cl && (isR ? (xm > pv.x) : (xm >= pv.x)));
                if (right) hi = mid;
                else lo = mid + 1;
            }
            for (int k = lo; k < s1; k++) {
                const unsigned q = SJ_AT(bc.st, sm.ord[k], nb);
                if (((unsigned)sm.tile[q] >> 14) != cl) break;
                const float4 ov = sm.mbr[q];
                if (ov.x > pv.z) break;
                if (ov.y <= pv.w && pv.y <= ov.w) {
                    if (OUT == 0) {
                        c++;
                    } else {
                        const unsigned oid = sm.id[q];
                        const int2 pr = isR ? make_int2((int)(pid & kIdMask), (int)(oid & kIdMask))
                                            : make_int2((int)(oid & kIdMask), (int)(pid & kIdMask));
                        const unsigned m = __activemask();
                        const int leader = __ffs(m) - 1;
                        unsigned pos = 0;
                        if ((int)(threadIdx.x & 31) == leader) pos = atomicAdd(ctr, (unsigned)__popc(m));
                        pos = __shfl_sync(m, pos, leader) + __popc(m & lanemask_lt_b());
                        if (OUT == 1) {
                            if (pos < (unsigned)kPairBuf) sm.pbuf[pos] = pr;
                            else if (spill && pos < (unsigned)(kPairBuf + kPairSpill)) spill[pos - kPairBuf] = pr;
                        } else if (SJ_IN(bc.st, base + pos, cap)) {
                            out[base + pos] = pr;
                        }
                    }
                }
            }
        }
        if (OUT == 0) {
            if (tile_pairs && c) {
                const int lt = ta + j;
                atomicAdd(tile_pairs + (bc.cyb + lt / bc.gw) * nx + bc.cxb + lt % bc.gw, c);
            }
            my += c;
        }
    }
    return my;
}

// Row lists of a block that needs several bands (see RowLists).  The slice
// comes from the pool cursor of this launch; rl.on = 0 when the pool is
// exhausted (the bands then read the whole L1 range).  Ends with a barrier.
__device__ void build_row_lists(BJSmem &sm, const BlockCtx &bc, RowLists &rl, unsigned *pool,
                                unsigned long long pool_cap, unsigned long long *cursor) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < bc.gh; y += kBJThreads / 32) {
        unsigned c = lane < bc.gw ? sm.cnt[0][y * bc.gw + lane] + sm.cnt[1][y * bc.gw + lane] : 0u;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFullMask, c, d);
        if (lane == 0) rl.pre[y] = c;   // room of row y
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned c = lane < bc.gh ? rl.pre[lane] : 0u;
        unsigned inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(kFullMask, inc, d);
            if (lane >= d) inc += o;
        }
        const unsigned total = __shfl_sync(kFullMask, inc, 31);
        rl.off[lane] = inc - c;
        rl.cur[lane] = 0;
        if (lane == 0) {
            rl.off[kMaxG] = total;
            const unsigned long long b = atomicAdd(cursor, (unsigned long long)total);
            rl.on = b + total <= pool_cap;
            rl.pool = pool + b;
        }
    }
    __syncthreads();
    if (!rl.on) return;
    const int n1 = (int)(bc.nr1 + bc.ns1);
    for (int e = threadIdx.x; e < n1; e += kBJThreads) {
        const int side = e >= (int)bc.nr1;
        const uint4 t = reinterpret_cast<const uint4 *>(side ? bc.es + (e - bc.nr1) : bc.er + e)[1];
        const int ly0 = max((int)(t.z & 0xffff) - bc.cyb, 0), ly1 = min((int)(t.z >> 16) - bc.cyb, bc.gh - 1);
        const int lx0 = max((int)(t.y & 0xffff) - bc.cxb, 0), lx1 = min((int)(t.y >> 16) - bc.cxb, bc.gw - 1);
        if (lx0 > lx1) continue;   // counted in no tile of the block (never for a written entry)
        for (int y = ly0; y <= ly1; y++) {
            const unsigned k = atomicAdd(&rl.cur[y], 1u);   // within the row's room
            if (SJ_IN(bc.st, k, rl.off[y + 1] - rl.off[y])) rl.pool[rl.off[y] + k] = (unsigned)e;
        }
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned c = lane < bc.gh ? rl.cur[lane] : 0u;
        unsigned inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(kFullMask, inc, d);
            if (lane >= d) inc += o;
        }
        rl.pre[lane] = inc - c;
        if (lane == 31) rl.pre[kMaxG] = inc;
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned *s_red) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFullMask, v, d);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned t = 0;
    for (int w = 0; w < kBJThreads / 32; w++) t += s_red[w];
    return t;
}

// Parallel band split of the block's ntl tiles (see step 2 of k_bjoin).
// Uses sm.off as scratch; writes sm.band[0..nbands] and the flags.
__device__ void band_split(BJSmem &sm, int ntl, unsigned *s_nbands, int *s_huge) {
    constexpr unsigned h = kFineCap / 2;
    __shared__ unsigned s_w[kBJThreads / 32];
    __shared__ unsigned s_t;
    __shared__ int s_hg;
    if (threadIdx.x == 0) s_hg = 0;
    // exclusive prefix of per-tile entries -> sm.off[0][lt]
    const int per = (ntl + kBJThreads - 1) / kBJThreads;
    const int l0 = threadIdx.x * per;
    unsigned sum = 0;
    for (int k = 0; k < per; k++)
        if (l0 + k < ntl) sum += sm.cnt[0][l0 + k] + sm.cnt[1][l0 + k];
    unsigned inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(kFullMask, inc, d);
        if ((threadIdx.x & 31) >= d) inc += o;
    }
    if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned x = threadIdx.x < kBJThreads / 32 ? s_w[threadIdx.x] : 0u;
        unsigned xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(kFullMask, xi, d);
            if (threadIdx.x >= (unsigned)d) xi += o;
        }
        if (threadIdx.x < kBJThreads / 32) s_w[threadIdx.x] = xi - x;
    }
    __syncthreads();
    unsigned run = s_w[threadIdx.x >> 5] + inc - sum;
    for (int k = 0; k < per; k++)
        if (l0 + k < ntl) {
            sm.off[0][l0 + k] = run;
            run += sm.cnt[0][l0 + k] + sm.cnt[1][l0 + k];
            if (l0 + k == ntl - 1) sm.off[0][ntl] = run;
        }
    __syncthreads();
    // band-start flags -> sm.off[1][lt]
    for (int lt = threadIdx.x; lt < ntl; lt += kBJThreads) {
        const unsigned c = sm.cnt[0][lt] + sm.cnt[1][lt];
        if (c > (unsigned)kFineCap) s_hg = 1;
        unsigned f = lt == 0;
        if (lt > 0) {
            const unsigned cp = sm.cnt[0][lt - 1] + sm.cnt[1][lt - 1];
            f |= (c > h) | (cp > h) | (sm.off[0][lt] / h != sm.off[0][lt - 1] / h);
        }
        sm.off[1][lt] = f;
    }
    __syncthreads();
    // compaction of the flags (exclusive scan) -> band starts
    sum = 0;
    for (int k = 0; k < per; k++)
        if (l0 + k < ntl) sum += sm.off[1][l0 + k];
    inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(kFullMask, inc, d);
        if ((threadIdx.x & 31) >= d) inc += o;
    }
    if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned x = threadIdx.x < kBJThreads / 32 ? s_w[threadIdx.x] : 0u;
        unsigned xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(kFullMask, xi, d);
            if (threadIdx.x >= (unsigned)d) xi += o;
        }
        if (threadIdx.x < kBJThreads / 32) s_w[threadIdx.x] = xi - x;
        if (threadIdx.x == kBJThreads / 32 - 1) s_t = xi;
    }
    __syncthreads();
    run = s_w[threadIdx.x >> 5] + inc - sum;
    for (int k = 0; k < per; k++)
        if (l0 + k < ntl) {
            if (sm.off[1][l0 + k]) sm.band[run] = (unsigned short)(l0 + k);
            run += sm.off[1][l0 + k];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        sm.band[s_t] = (unsigned short)ntl;
        // the rule above leaves bands of h to 2h entries: merge neighbours
        // greedily while the merged band still fits (sm.off[0] = prefix)
        unsigned k = s_t;
        if (!s_hg) {
            k = 0;
            for (unsigned i = 1; i < s_t; i++)
                if (sm.off[0][sm.band[i + 1]] - sm.off[0][sm.band[k]] > (unsigned)kFineCap) sm.band[++k] = sm.band[i];
            sm.band[++k] = (unsigned short)ntl;
        }
        *s_nbands = k;
        *s_huge = s_hg;
    }
    __syncthreads();
}

template <int MODE, int VARIANT>   // VARIANT: 0 plain, 1 adaptive sweep axis, 2 GBDA
__global__ void __launch_bounds__(kBJThreads, 2) k_bjoin(BArgs a, BJoinOut o) {
    constexpr int ADAPT = VARIANT == 1;
    constexpr int GBDA = VARIANT == 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BJSmem &sm = *reinterpret_cast<BJSmem *>(smem_raw);
    __shared__ unsigned s_meta[2][16];  // current / next item: item, block, r0, nr, s0, ns, join geometry
    __shared__ unsigned s_nbands, s_cursor, s_pc;
    __shared__ RowLists s_rows;
    __shared__ int s_ok, s_huge;
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_red[kBJThreads / 32];
    if (block_skip_blocked(a.st)) return;
    const unsigned nlist = o.list ? *o.list_n : a.st->nchunks;
    // Thread 0 runs two steps ahead: the work counter is read for item k+2
    // and the (single-load) metadata of item k+1 is gathered while item k is
    // joined, so neither round trip stalls the block.
    unsigned raw_next = 0;   // thread 0: work index of the item after the current one
    auto load_meta = [&](unsigned raw, unsigned *m) {
        if (raw < nlist) {
            const unsigned it = o.list ? o.list[raw] : raw;
            const uint4 q = a.imeta[it];
            const unsigned ns = a.ins[it];
            const JoinDesc &d = a.jd[a.nj == 1 ? 0 : a.ijoin[it]];
            m[0] = it;
            m[1] = q.x - (unsigned)d.boff;   // block inside its join
            m[2] = q.y;
            m[3] = q.z;
            m[4] = q.w;
            m[5] = ns;
            m[6] = (unsigned)d.G;
            m[7] = (unsigned)d.bx;
            m[8] = (unsigned)d.g.nx;
            m[9] = (unsigned)d.g.ny;
            m[10] = __float_as_uint(d.g.x0);   // the join's grid (adaptive axis: the Eq. 2 buckets)
            m[11] = __float_as_uint(d.g.gx);
            m[12] = __float_as_uint(d.g.y0);
            m[13] = __float_as_uint(d.g.gy);
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.bent_r + q.y),
                         "r"(q.z * (unsigned)sizeof(BEnt)) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.bent_s + q.w),
                         "r"(ns * (unsigned)sizeof(BEnt)) : "memory");
        } else {
            m[0] = 0xffffffffu;
        }
    };
    if (threadIdx.x == 0) {
        const unsigned r0_ = atomicAdd(&a.st->work[o.work_slot], 1u);
        raw_next = atomicAdd(&a.st->work[o.work_slot], 1u);
        load_meta(r0_, s_meta[0]);
    }
    // per-tile counters start cleared; each block clears the ones it used
    // when it ends (the adaptive variant clears them, with its histograms, as
    // each block starts)
    if (!ADAPT)
        for (int k = threadIdx.x; k < 2 * kMaxFine; k += kBJThreads) (&sm.cnt[0][0])[k] = 0;
    __syncthreads();
    for (int step = 0;; step++) {
        const int cur = step & 1;
        if (s_meta[cur][0] == 0xffffffffu) break;
        unsigned raw_after = 0;
        if (threadIdx.x == 0) raw_after = atomicAdd(&a.st->work[o.work_slot], 1u);   // value used next step
        const unsigned *m = s_meta[cur];
        const unsigned it = m[0], b = m[1];
        const int jG = (int)m[6], jbx = (int)m[7], jnx = (int)m[8], jny = (int)m[9];
        BlockCtx bc;
        const int bxi = (int)(b % (unsigned)jbx), byi = (int)(b / (unsigned)jbx);
        bc.cxb = bxi * jG;
        bc.cyb = byi * jG;
        bc.gw = min(jG, jnx - bc.cxb);
        bc.gh = min(jG, jny - bc.cyb);
        bc.ntl = bc.gw * bc.gh;
        bc.r0 = m[2];
        bc.nr1 = m[3];
        bc.s0 = m[4];
        bc.ns1 = m[5];
        bc.er = a.bent_r + bc.r0;
        bc.es = a.bent_s + bc.s0;
        bc.st = a.st;

        // step 1: entries per tile of the block (and, for the adaptive sweep
        // axis, the Eq. 2 histograms of every tile: k = 8 buckets per axis)
        unsigned *hist = reinterpret_cast<unsigned *>(sm.key);
        if (ADAPT) {
            for (int k = threadIdx.x; k < bc.ntl; k += kBJThreads) {
                sm.cnt[0][k] = 0;
                sm.cnt[1][k] = 0;
            }
            for (int k = threadIdx.x; k < bc.ntl * kHistWords; k += kBJThreads) hist[k] = 0;
            __syncthreads();
        }
        const int n1 = (int)(bc.nr1 + bc.ns1);
        constexpr int kCountU = 2;   // entries a thread loads before counting them
        for (int eb = threadIdx.x; eb < n1; eb += kCountU * kBJThreads) {
            uint4 t[kCountU], hd[kCountU];
#pragma unroll
            for (int u = 0; u < kCountU; u++)
                if (eb + u * kBJThreads < n1) {
                    const uint4 *w = entry_words(bc, eb + u * kBJThreads);
                    t[u] = w[1];
                    if (ADAPT) hd[u] = w[0];
                }
#pragma unroll
            for (int u = 0; u < kCountU; u++) {
                const int e = eb + u * kBJThreads;
                if (e >= n1) break;
                const int side = e >= (int)bc.nr1;
                const int cx0 = (int)(t[u].y & 0xffff), cx1 = (int)(t[u].y >> 16);
                const int cy0 = (int)(t[u].z & 0xffff), cy1 = (int)(t[u].z >> 16);
                const int lx0 = max(cx0 - bc.cxb, 0), lx1 = min(cx1 - bc.cxb, bc.gw - 1);
                const int ly0 = max(cy0 - bc.cyb, 0), ly1 = min(cy1 - bc.cyb, bc.gh - 1);
                int fx0 = 0, fx1 = 0, fy0 = 0, fy1 = 0;
                if (ADAPT) {
                    const float gx0 = __uint_as_float(m[10]), ggx = __uint_as_float(m[11]);
                    const float gy0 = __uint_as_float(m[12]), ggy = __uint_as_float(m[13]);
                    fx0 = cell8_of(__uint_as_float(hd[u].x), gx0, ggx, jnx);
                    fx1 = cell8_of(__uint_as_float(hd[u].z), gx0, ggx, jnx);
                    fy0 = cell8_of(__uint_as_float(hd[u].y), gy0, ggy, jny);
                    fy1 = cell8_of(__uint_as_float(hd[u].w), gy0, ggy, jny);
                }
                for (int ly = ly0; ly <= ly1; ly++)
                    for (int lx = lx0; lx <= lx1; lx++) {
                        const int lt = ly * bc.gw + lx;
                        if (!SJ_IN(a.st, lt, bc.ntl)) continue;
                        atomicAdd(&sm.cnt[side][lt], 1u);
                        if (ADAPT) {
                            // buckets of the projections inside this tile
                            const int col = bc.cxb + lx, row = bc.cyb + ly;
                            const int bx0 = col == cx0 ? fx0 - 8 * col : 0, bx1 = col == cx1 ? fx1 - 8 * col : 7;
                            const int by0 = row == cy0 ? fy0 - 8 * row : 0, by1 = row == cy1 ? fy1 - 8 * row : 7;
                            unsigned *hx = hist + lt * kHistWords + side * 8, *hy = hx + 4;
                            for (int b = bx0; b <= bx1; b++) atomicAdd(hx + (b >> 1), 1u << ((b & 1) << 4));
                            for (int b = by0; b <= by1; b++) atomicAdd(hy + (b >> 1), 1u << ((b & 1) << 4));
                        }
                    }
            }
        }
        __syncthreads();
        bc.axis = nullptr;
        bc.gbda = GBDA;
        if (ADAPT) {
            // Eq. 2: I = sum_i H_R[i] H_S[i] per axis; sweep along y when
            // I_y < I_x (ties and tiles missing a side keep x)
            for (int l0 = 0; l0 < bc.ntl; l0 += kBJThreads) {
                const int lt = l0 + threadIdx.x;
                bool y = false;
                if (lt < bc.ntl && sm.cnt[0][lt] && sm.cnt[1][lt]) {
                    const unsigned *h = hist + lt * kHistWords;
                    unsigned long long ix = 0, iy = 0;
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const unsigned rx = h[q], ry = h[4 + q], sx = h[8 + q], sy = h[12 + q];
                        ix += (unsigned long long)(rx & 0xffffu) * (sx & 0xffffu) +
                              (unsigned long long)(rx >> 16) * (sx >> 16);
                        iy += (unsigned long long)(ry & 0xffffu) * (sy & 0xffffu) +
                              (unsigned long long)(ry >> 16) * (sy >> 16);
                    }
                    y = iy < ix;
                }
                const unsigned bits = __ballot_sync(kFullMask, y);
                if ((threadIdx.x & 31) == 0 && lt < bc.ntl) {
                    sm.axis[lt >> 5] = bits;
                    if ((MODE == MODE_COUNT || MODE == MODE_RESERVE) && bits)
                        atomicAdd(&a.st->naxis_y, (unsigned)__popc(bits));
                }
                if (MODE == MODE_COUNT && o.tile_axis && lt < bc.ntl)
                    o.tile_axis[(size_t)(bc.cyb + lt / bc.gw) * jnx + bc.cxb + lt % bc.gw] = y ? 1 : 0;
            }
            bc.axis = sm.axis;   // read in the placement, after the barriers of step 2
        }
        // step 2: bands of consecutive tiles that fit in shared memory.
        // Usually the whole block fits (one band): the offsets of the whole
        // block computed here are then its band's.  Otherwise, with h = half
        // the capacity, a band starts at every tile whose exclusive prefix
        // of entries enters a new multiple of h, and around every tile
        // heavier than h (each band then holds fewer than 2h entries), and
        // neighbouring bands are merged while they fit.
        int nR0, nS0;
        band_offsets(sm, 0, bc.ntl, nR0, nS0);   // ends with a barrier: every thread knows the total
        const bool single = nR0 + nS0 <= kFineCap;
        if (single) {
            // the usual case decides without a barrier: the cursors are first
            // used after the barrier of the band's scatter
            if (threadIdx.x == 0) {
                s_cursor = 0;
                s_pc = 0;
            }
        } else {
            band_split(sm, bc.ntl, &s_nbands, &s_huge);
            if (threadIdx.x == 0) {
                s_cursor = 0;
                s_pc = 0;
            }
            __syncthreads();
        }
        // tiles of band bi
        auto band_lo = [&](int bi) { return single ? 0 : (int)sm.band[bi]; };
        auto band_hi = [&](int bi) { return single ? bc.ntl : (int)sm.band[bi + 1]; };
        if (!single && s_huge) {   // a single tile exceeds shared memory: the caller reruns on the direct path
            if (threadIdx.x == 0) {
                atomicOr(&a.st->need_direct, 1);
                if (MODE == MODE_COUNT) o.cnt_out[it] = 0;
            }
        } else {
            const int nbands = single ? 1 : (int)s_nbands;
            // a block staged in several bands first lists its entries per tile
            // row, so that every band reads only the entries of its rows
            const RowLists *rl = nullptr;
            if (nbands > 1 && a.lpool) {
                build_row_lists(sm, bc, s_rows, a.lpool, a.lpool_cap, &a.st->lpool[o.work_slot & 3]);
                if (s_rows.on) rl = &s_rows;
            }
            // band bi into shared memory (a single band has its offsets already)
            auto stage = [&](int bi, int &nRb, int &nSb) {
                stage_band(sm, bc, band_lo(bi), band_hi(bi), nbands == 1, nR0, nS0, rl, nRb, nSb);
            };
            // pairs of the staged band at out[base + s_cursor ...]
            auto write = [&](int nRb, int nSb, unsigned long long base) {
                if (GBDA) gbda_sweep<2>(sm, bc, 0, nRb, nSb, &s_cursor, nullptr, o.out, base, nullptr, 0, o.cap);
                else band_write(sm, nRb, nSb, o.out, base, &s_cursor, a.st, o.cap);
            };
            if (MODE == MODE_WRITE) {
                const unsigned long long base = o.off_in[it];
                for (int bi = 0; bi < nbands; bi++) {
                    int nRb, nSb;
                    stage(bi, nRb, nSb);
                    write(nRb, nSb, base);
                    __syncthreads();
                }
            } else {
                unsigned tot = 0;
                int nRb = 0, nSb = 0;
                for (int bi = 0; bi < nbands; bi++) {
                    stage(bi, nRb, nSb);
                    if (MODE == MODE_RESERVE) {
                        int2 *sp = o.spill ? o.spill + (size_t)blockIdx.x * kPairSpill : nullptr;
                        if (GBDA) gbda_sweep<1>(sm, bc, 0, nRb, nSb, &s_pc, sp, nullptr, 0, nullptr, 0);
                        else band_collect(sm, nRb, nSb, &s_pc, sp, a.st);
                        __syncthreads();
                    } else {
                        unsigned *tp = MODE == MODE_TILES ? o.tile_pairs : nullptr;
                        const unsigned c = GBDA ? gbda_sweep<0>(sm, bc, band_lo(bi), nRb, nSb, nullptr, nullptr,
                                                                nullptr, 0, tp, jnx)
                                                : band_count(sm, bc, band_lo(bi), nRb, nSb, tp, jnx);
                        tot += block_sum(c, s_red);
                    }
                }
                if (MODE == MODE_RESERVE) tot = s_pc;
                if (MODE == MODE_COUNT || MODE == MODE_RESERVE) {
                    if (threadIdx.x == 0) {
                        if (MODE == MODE_COUNT) {
                            o.cnt_out[it] = tot;
                        } else {
                            const unsigned long long bs = atomicAdd(&a.st->npairs, (unsigned long long)tot);
                            o.resv[it] = bs;
                            if (o.cnt_out) o.cnt_out[it] = tot;
                            const bool ok = tot == 0 || bs + tot <= o.cap;
                            s_ok = ok;
                            s_base = bs;
                            if (!ok) {
                                const unsigned f = atomicAdd(o.nfail, 1u);
                                o.fail[f] = it;
                            }
                        }
                    }
                    __syncthreads();
                    if (MODE == MODE_RESERVE && s_ok) {
                        const unsigned kept = o.spill ? kPairBuf + kPairSpill : kPairBuf;
                        if (tot <= kept) {   // the usual case: copy the collected pairs
                            const int2 *sp = o.spill + (size_t)blockIdx.x * kPairSpill;
                            for (unsigned i = threadIdx.x; i < tot; i += kBJThreads)
                                o.out[s_base + i] = i < (unsigned)kPairBuf ? sm.pbuf[i] : sp[i - kPairBuf];
                        } else if (nbands == 1) {
                            write(nRb, nSb, s_base);
                        } else {
                            for (int bi = 0; bi < nbands; bi++) {
                                stage(bi, nRb, nSb);
                                write(nRb, nSb, s_base);
                                __syncthreads();
                            }
                        }
                    }
                }
            }
        }
        // clear the counters this block used (every reader of them is behind
        // one of the barriers above) for the next block's count
        if (!ADAPT)
            for (int k = threadIdx.x; k < bc.ntl; k += kBJThreads) {
                sm.cnt[0][k] = 0;
                sm.cnt[1][k] = 0;
            }
        if (threadIdx.x == 0) {
            load_meta(raw_next, s_meta[cur ^ 1]);
            raw_next = raw_after;
        }
        __syncthreads();
    }
}

// Feature sampling for the learned sizing: rectangles 0, kPhi, 2 kPhi, ... of
// each side add their bucket ranges to every block they overlap.
template <int PTS>
__global__ void __launch_bounds__(256) k_bfeat_sample(BArgs a) {
    // the one-pass join leaves for the single-level path when the block scan
    // found a tile beyond shared memory: its sample would go unused
    if (a.stop_direct && block_skip_blocked(a.st)) return;
    const long long mr = (a.nR + kPhi - 1) / kPhi, ms = (a.nS + kPhi - 1) / kPhi;
    for (long long k = blockIdx.x * 256ll + threadIdx.x; k < mr + ms; k += 256ll * gridDim.x) {
        const int side = k >= mr;
        const long long i = (side ? k - mr : k) * kPhi;
        float4 v;
        if constexpr (PTS) v = load_square(side ? a.S : a.R, i, a.h);
        else v = ld_stream(side ? a.S + i : a.R + i);
        if (!rect_ok(v)) continue;
        const int cx0 = cell_of(v.x, a.g.x0, a.g.gx, a.g.nx), cx1 = cell_of(v.z, a.g.x0, a.g.gx, a.g.nx);
        const int cy0 = cell_of(v.y, a.g.y0, a.g.gy, a.g.ny), cy1 = cell_of(v.w, a.g.y0, a.g.gy, a.g.ny);
        feat_add(a.feat_raw, a.G, a.bx, side, cx0, cx1, cy0, cy1, div_g(cx0, a), div_g(cx1, a), div_g(cy0, a),
                 div_g(cy1, a));
    }
}

// Feature sampling of a batch: sample k of the batch is rectangle
// kPhi * (k - samp_off of its join) of the join's R, then of its S (the same
// systematic sample per side as a single join); its buckets go to the join's
// blocks in the global block index space.
__global__ void __launch_bounds__(256) k_bfeat_sample_batch(BArgs a, long long nsamp) {
    extern __shared__ long long s_soff[];   // nj + 1
    for (int j = threadIdx.x; j < a.nj; j += 256) s_soff[j] = a.jd[j].samp_off;
    if (threadIdx.x == 0) s_soff[a.nj] = nsamp;
    __syncthreads();
    for (long long k = blockIdx.x * 256ll + threadIdx.x; k < nsamp; k += 256ll * gridDim.x) {
        const int j = a.nj == 1 ? 0 : join_of(s_soff, a.nj, k);
        const JoinDesc &d = a.jd[j];
        const long long loc = k - s_soff[j], mr = (d.nR + kPhi - 1) / kPhi;
        const int side = loc >= mr;
        const long long i = (side ? loc - mr : loc) * kPhi;
        const float4 v = ld_stream(side ? d.S + i : d.R + i);
        if (!rect_ok(v)) continue;
        const int cx0 = cell_of(v.x, d.g.x0, d.g.gx, d.g.nx), cx1 = cell_of(v.z, d.g.x0, d.g.gx, d.g.nx);
        const int cy0 = cell_of(v.y, d.g.y0, d.g.gy, d.g.ny), cy1 = cell_of(v.w, d.g.y0, d.g.gy, d.g.ny);
        feat_add(a.feat_raw + (size_t)d.boff * kRawPerBlock, d.G, d.bx, side, cx0, cx1, cy0, cy1,
                 div_gj(cx0, d), div_gj(cx1, d), div_gj(cy0, d), div_gj(cy1, d));
    }
}

// One warp per work item: its cnt pairs from src[resv ...] to dst[poff ...].
__global__ void __launch_bounds__(256) k_regroup(const unsigned *__restrict__ cnt,
                                                 const unsigned long long *__restrict__ resv,
                                                 const unsigned long long *__restrict__ poff,
                                                 const unsigned *__restrict__ n_dev, const int2 *__restrict__ src,
                                                 int2 *__restrict__ dst) {
    const unsigned n = *n_dev;
    const unsigned lane = threadIdx.x & 31;
    for (unsigned it = (blockIdx.x * 256u + threadIdx.x) >> 5; it < n; it += gridDim.x * 8u) {
        const unsigned c = cnt[it];
        const int2 *s = src + resv[it];
        int2 *d = dst + poff[it];
        for (unsigned i = lane; i < c; i += 32) d[i] = s[i];
    }
}

// Sums of widths and heights of every join's rectangles (for the grid rule),
// out[4 j + 0..3] = sum w_R, sum h_R, sum w_S, sum h_S (float64).  Every
// lane walks a contiguous run of rectangles, accumulates in registers and
// adds to the totals only when its run crosses into another join or side.
__global__ void __launch_bounds__(256) k_extent_stats(BArgs a, double *__restrict__ out) {
    extern __shared__ long long s_jin[];
    for (int j = threadIdx.x; j < a.nj; j += 256) s_jin[j] = a.jd[j].in_off;
    if (threadIdx.x == 0) s_jin[a.nj] = a.jd[a.nj - 1].in_off + a.jd[a.nj - 1].nR + a.jd[a.nj - 1].nS;
    __syncthreads();
    const long long n = s_jin[a.nj];
    const long long nthreads = (long long)gridDim.x * 256;
    const long long per = (n + nthreads - 1) / nthreads;
    const long long i0 = ((long long)blockIdx.x * 256 + threadIdx.x) * per;
    const long long i1 = min(n, i0 + per);
    int cur = -1;
    double sw = 0.0, sh = 0.0;
    for (long long i = i0; i < i1; i++) {
        const int j = a.nj == 1 ? 0 : join_of(s_jin, a.nj, i);
        const JoinDesc &d = a.jd[j];
        const long long li = i - s_jin[j];
        const int side = li >= d.nR;
        const int key = 2 * j + side;
        if (key != cur) {
            if (cur >= 0 && (sw != 0.0 || sh != 0.0)) {
                atomicAdd(out + 2 * cur, sw);
                atomicAdd(out + 2 * cur + 1, sh);
            }
            cur = key;
            sw = sh = 0.0;
        }
        const float4 v = ld_stream(side ? d.S + (li - d.nR) : d.R + li);
        if (!rect_ok(v)) continue;
        sw += (double)(v.z - v.x);
        sh += (double)(v.w - v.y);
    }
    if (cur >= 0 && (sw != 0.0 || sh != 0.0)) {
        atomicAdd(out + 2 * cur, sw);
        atomicAdd(out + 2 * cur + 1, sh);
    }
}

// ---- launchers -------------------------------------------------------------
cudaError_t launch_bfeat_sample(const BArgs &a, int grid, cudaStream_t s) {
    if (a.pts) k_bfeat_sample<1><<<grid, 256, 0, s>>>(a);
    else k_bfeat_sample<0><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bfeat_sample_batch(const BArgs &a, long long nsamp, int grid, cudaStream_t s) {
    k_bfeat_sample_batch<<<grid, 256, 8ull * (a.nj + 1), s>>>(a, nsamp);
    return cudaGetLastError();
}

cudaError_t launch_regroup(const unsigned *cnt, const unsigned long long *resv, const unsigned long long *poff,
                           const unsigned *n_dev, const int2 *src, int2 *dst, int grid, cudaStream_t s) {
    k_regroup<<<grid, 256, 0, s>>>(cnt, resv, poff, n_dev, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_extent_stats(const BArgs &a, double *out, int grid, cudaStream_t s) {
    k_extent_stats<<<grid, 256, 8ull * (a.nj + 1), s>>>(a, out);
    return cudaGetLastError();
}

size_t bjoin_smem_bytes() { return sizeof(BJSmem); }

cudaError_t blocked_setup() {
    cudaError_t e;
    const int sm = (int)sizeof(BJSmem);
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_COUNT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_WRITE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_RESERVE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_TILES, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_COUNT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_WRITE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_RESERVE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_COUNT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_WRITE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bjoin<MODE_RESERVE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(k_bcount_local, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(8 * (kMaxJoins + 1) + 4 * kLocalHist))))
        return e;
    const int l1 = 8 * kMaxBlocks;
    if ((e = cudaFuncSetAttribute(k_bcount<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, l1))) return e;
    if ((e = cudaFuncSetAttribute(k_bcount<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, l1))) return e;
    if ((e = cudaFuncSetAttribute(k_bscatter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, l1))) return e;
    if ((e = cudaFuncSetAttribute(k_bscatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, l1))) return e;
    return cudaSuccess;
}

int bjoin_blocks_per_sm() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bjoin<MODE_WRITE, 0>, kBJThreads, sizeof(BJSmem));
    return nb > 0 ? nb : 1;
}

int l1_blocks_per_sm(int nb_blocks) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bscatter<0>, kL1Threads, 8ull * nb_blocks);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_bcount(const BArgs &a, int nc, cudaStream_t s) {
    if (a.pts) k_bcount<1><<<nc, kL1Threads, 8ull * a.nb, s>>>(a);
    else k_bcount<0><<<nc, kL1Threads, 8ull * a.nb, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bscan_blocks_only(const BArgs &a, cudaStream_t s) {
    const int nch = (a.nbt + kScanChunk - 1) / kScanChunk;
    k_bscan_part<<<nch, kScanThreads, 0, s>>>(a, a.scan_part);
    k_bscan_top<<<1, 1024, 0, s>>>(a, a.scan_part, nch);
    k_bscan_fill<<<nch, kScanThreads, 0, s>>>(a, a.scan_part);
    return cudaGetLastError();
}

int bscan_chunks(int nb) { return (nb + kScanChunk - 1) / kScanChunk; }

cudaError_t launch_bscan(const BArgs &a, int nc, cudaStream_t s) {
    k_bscan_ctas<<<(2 * a.nb + 255) / 256, 256, 0, s>>>(a, nc);
    return launch_bscan_blocks_only(a, s);
}

cudaError_t launch_bcount_global(const BArgs &a, int grid, cudaStream_t s) {
    k_bcount_global<<<grid, 256, 8ull * (a.nj + 1), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bcount_local(const BArgs &a, int grid, cudaStream_t s) {
    k_bcount_local<<<grid, kLocalThreads, 8ull * (a.nj + 1) + 4ull * kLocalHist, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_join_offsets(const BArgs &a, const unsigned long long *poff, unsigned long long *joff,
                                cudaStream_t s) {
    k_join_offsets<<<(a.nj + 256) / 256, 256, 0, s>>>(a, poff, joff);
    return cudaGetLastError();
}

cudaError_t launch_bscatter(const BArgs &a, int nc, cudaStream_t s) {
    if (a.cur) {
        if (a.pts) k_bscatter_shared<1><<<nc * 8, 256, 8ull * (a.nj + 1), s>>>(a);
        else k_bscatter_shared<0><<<nc * 8, 256, 8ull * (a.nj + 1), s>>>(a);
    } else {
        if (a.pts) k_bscatter<1><<<nc, kL1Threads, 8ull * a.nb, s>>>(a);
        else k_bscatter<0><<<nc, kL1Threads, 8ull * a.nb, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_bjoin(int mode, const BArgs &a, const BJoinOut &o, int grid, cudaStream_t s) {
    const size_t sm = sizeof(BJSmem);
    if (a.gbda) {
        switch (mode) {
            case MODE_COUNT: k_bjoin<MODE_COUNT, 2><<<grid, kBJThreads, sm, s>>>(a, o); break;
            case MODE_WRITE: k_bjoin<MODE_WRITE, 2><<<grid, kBJThreads, sm, s>>>(a, o); break;
            case MODE_RESERVE: k_bjoin<MODE_RESERVE, 2><<<grid, kBJThreads, sm, s>>>(a, o); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    if (a.adaptive) {
        switch (mode) {
            case MODE_COUNT: k_bjoin<MODE_COUNT, 1><<<grid, kBJThreads, sm, s>>>(a, o); break;
            case MODE_WRITE: k_bjoin<MODE_WRITE, 1><<<grid, kBJThreads, sm, s>>>(a, o); break;
            case MODE_RESERVE: k_bjoin<MODE_RESERVE, 1><<<grid, kBJThreads, sm, s>>>(a, o); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (mode) {
        case MODE_COUNT: k_bjoin<MODE_COUNT, 0><<<grid, kBJThreads, sm, s>>>(a, o); break;
        case MODE_WRITE: k_bjoin<MODE_WRITE, 0><<<grid, kBJThreads, sm, s>>>(a, o); break;
        case MODE_RESERVE: k_bjoin<MODE_RESERVE, 0><<<grid, kBJThreads, sm, s>>>(a, o); break;
        default: k_bjoin<MODE_TILES, 0><<<grid, kBJThreads, sm, s>>>(a, o); break;
    }
    return cudaGetLastError();
}

}  // namespace sj
