// sweep.cu -- joining phase of PBSM on the GPU (Sec. 3.4 steps 5-6):
// per tile, sort both sides by x_l and run the forward-scan plane sweep of
// Algorithm 1 with a y-overlap test and the reference-point duplicate test of
// Eq. 1.
//
// Pivot-parallel form of Algorithm 1.  Algorithm 1 walks the merged x_l order;
// when r comes first (r.x_l < s.x_l) r scans S forward while s.x_l <= r.x_u,
// otherwise (ties included) s scans R forward while r.x_l <= s.x_u.  So a
// pair (r, s) that x-overlaps is examined exactly once: by r when
// s.x_l in (r.x_l, r.x_u], by s when r.x_l in [s.x_l, s.x_u].  Every entry is
// therefore an independent pivot: it locates its start in the other side's
// sorted segment by binary search and scans forward.  The set of examined
// candidates and reported pairs is the same as Algorithm 1's.
#define SJ_FILE_CODE 2
#include "sj_common.cuh"
#include "sj_kernels.h"

namespace sj {

constexpr unsigned kFull = 0xffffffffu;

// first index k in [lo, hi) with x[k] > v (strict) or >= v (!strict)
template <bool STRICT, typename Get>
__device__ __forceinline__ int lower_pos(int lo, int hi, float v, Get get) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        float xm = get(mid);
        bool right = STRICT ? (xm > v) : (xm >= v);
        if (right) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// ----------------------------------------------------------------------------
// Small tiles: one chunk of consecutive tiles per CTA iteration, staged in
// shared memory.  Persistent CTAs take chunks from a device counter.
//   MODE_COUNT : pairs per chunk -> cnt_out[c]
//   MODE_WRITE : pairs written at out[off_in[c] ...]
//   MODE_RESERVE : count, reserve a range with one atomic on st->npairs,
//                  write if it fits below cap, else record the chunk
//   MODE_TILES : pairs per tile -> tile_pairs[t] (statistics / labels)
// ----------------------------------------------------------------------------
struct SmemChunk {
    uint2 off[kChunk + 1];          // absolute (R, S) offsets of the chunk's tiles
    float4 mbr[kChunkEnt];          // sorted entries: R segment, then S segment
    unsigned id[kChunkEnt];
    unsigned key[kChunkEnt];        // x_l keys, load order
    unsigned short tile[kChunkEnt]; // chunk-local tile of each position
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int MODE>
__global__ void __launch_bounds__(kSweepThreads, 3) k_sweep_chunks(SweepArgs a) {
    if (block_skip(a.st)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemChunk &sm = *reinterpret_cast<SmemChunk *>(smem_raw);
    __shared__ unsigned s_chunk;
    __shared__ unsigned s_cursor;
    __shared__ unsigned long long s_base;
    __shared__ int s_ok;
    __shared__ unsigned s_red[kSweepThreads / 32];

    const int tid = threadIdx.x;
    const unsigned lane = tid & 31;
    const unsigned nlist = a.list ? *a.list_n : a.st->nchunks;

    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(&a.st->work[a.work_slot], 1u);
        __syncthreads();
        const unsigned item = s_chunk;
        if (item >= nlist) break;
        const unsigned c = a.list ? a.list[item] : item;
        unsigned t0 = a.ts[c], t1 = a.ts[c + 1];
        if (t1 > t0) {
            const uint2 lo = a.off[t1 - 1], hi = a.off[t1];
            if ((hi.x - lo.x) + (hi.y - lo.y) + 1u > (unsigned)kChunk) t1--;   // large tile
        }
        const int nt = (int)(t1 - t0);
        const uint2 b0 = a.off[t0], b1 = a.off[t1];
        const int nR = (int)(b1.x - b0.x), nS = (int)(b1.y - b0.y);
        const int nc = nR + nS;
        if (nt > kChunk || nc > kChunkEnt) {   // cannot happen by construction
            if (tid == 0) atomicOr(&a.st->err, kErrChunkCap);
            __syncthreads();
            continue;
        }
        for (int k = tid; k <= nt; k += kSweepThreads) sm.off[k] = a.off[t0 + k];
        __syncthreads();

        // Phase 1: load entries, keys and chunk-local tile of every position.
        float4 m[kItems];
        unsigned idv[kItems], key[kItems];
        int tl[kItems];
#pragma unroll
        for (int it = 0; it < kItems; it++) {
            const int e = it * kSweepThreads + tid;
            tl[it] = -1;
            if (e < nc) {
                const bool isS = e >= nR;
                const unsigned loc = isS ? (unsigned)(e - nR) : (unsigned)e;
                const unsigned gi = (isS ? b0.y : b0.x) + loc;
                m[it] = isS ? a.ent_s[gi] : a.ent_r[gi];
                idv[it] = isS ? a.id_s[gi] : a.id_r[gi];
                key[it] = xkey(m[it].x);
                // largest j with rel_off(j) <= loc
                int lo = 0, hi = nt;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    const unsigned o = isS ? sm.off[mid].y - b0.y : sm.off[mid].x - b0.x;
                    if (o <= loc) lo = mid;
                    else hi = mid;
                }
                tl[it] = lo;
                sm.key[e] = key[it];
                sm.tile[e] = (unsigned short)lo;
            }
        }
        __syncthreads();

        // Phase 2: rank of every entry inside its tile segment (ties by
        // position) -> write it to its sorted place.
#pragma unroll
        for (int it = 0; it < kItems; it++) {
            const int e = it * kSweepThreads + tid;
            if (e < nc) {
                const bool isS = e >= nR;
                const int j = tl[it];
                const int s0 = isS ? nR + (int)(sm.off[j].y - b0.y) : (int)(sm.off[j].x - b0.x);
                const int s1 = isS ? nR + (int)(sm.off[j + 1].y - b0.y) : (int)(sm.off[j + 1].x - b0.x);
                const unsigned k0 = key[it];
                int r = 0;
                for (int q = s0; q < s1; q++) {
                    const unsigned kq = sm.key[q];
                    r += (kq < k0) | ((kq == k0) & (q < e));
                }
                if (!SJ_IN(a.st, r, s1 - s0) || !SJ_IN(a.st, s1 - 1, nc)) continue;
                sm.mbr[s0 + r] = m[it];
                sm.id[s0 + r] = idv[it];
            }
        }
        if (tid == 0) s_cursor = 0;
        __syncthreads();

        // Phase 3: sweep.  Pivot p scans the other side of its tile.
        unsigned my = 0;
        auto pivot_setup = [&](int p, float4 &pv, unsigned &pid, int &k, int &kend, bool &isR) {
            isR = p < nR;
            const int j = sm.tile[p];
            pv = sm.mbr[p];
            pid = sm.id[p];
            if (isR) {
                const int o0 = nR + (int)(sm.off[j].y - b0.y), o1 = nR + (int)(sm.off[j + 1].y - b0.y);
                k = lower_pos<true>(o0, o1, pv.x, [&](int q) { return sm.mbr[q].x; });
                kend = o1;
            } else {
                const int o0 = (int)(sm.off[j].x - b0.x), o1 = (int)(sm.off[j + 1].x - b0.x);
                k = lower_pos<false>(o0, o1, pv.x, [&](int q) { return sm.mbr[q].x; });
                kend = o1;
            }
        };

        if (MODE == MODE_COUNT || MODE == MODE_RESERVE || MODE == MODE_TILES) {
            for (int p = tid; p < nc; p += kSweepThreads) {
                float4 pv;
                unsigned pid;
                int k, kend;
                bool isR;
                pivot_setup(p, pv, pid, k, kend, isR);
                unsigned cnt = 0;
                for (; k < kend; k++) {
                    const float4 o = sm.mbr[k];
                    if (o.x > pv.z) break;
                    if (o.y <= pv.w && pv.y <= o.w && reported_here(pid, sm.id[k])) cnt++;
                }
                if (MODE == MODE_TILES) {
                    if (cnt) atomicAdd(a.tile_pairs + t0 + sm.tile[p], cnt);
                }
                my += cnt;
            }
            if (MODE == MODE_TILES) {
                __syncthreads();
                continue;
            }
            // block reduction
            unsigned v = my;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
            if (lane == 0) s_red[tid >> 5] = v;
            __syncthreads();
            if (tid == 0) {
                unsigned tot = 0;
                for (int w = 0; w < kSweepThreads / 32; w++) tot += s_red[w];
                if (MODE == MODE_COUNT) {
                    a.cnt_out[c] = tot;
                } else {
                    const unsigned long long base = atomicAdd(&a.st->npairs, (unsigned long long)tot);
                    a.resv[c] = base;
                    const bool ok = tot == 0 || base + tot <= a.cap;
                    s_ok = ok;
                    s_base = base;
                    if (!ok) {
                        const unsigned f = atomicAdd(a.nfail, 1u);
                        a.fail[f] = c;
                    }
                }
            }
            __syncthreads();
            if (MODE == MODE_COUNT || !s_ok) continue;
        }

        // Write pass: warp-synchronous scan; hits are compacted with a ballot
        // and appended to the chunk's range with one shared atomic per warp.
        {
            const unsigned long long base = MODE == MODE_WRITE ? a.off_in[c] : s_base;
            for (int pb = 0; pb < nc; pb += kSweepThreads) {
                const int p = pb + tid;
                const bool active = p < nc;
                float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
                unsigned pid = 0;
                int k = 0, kend = 0;
                bool isR = true;
                if (active) pivot_setup(p, pv, pid, k, kend, isR);
                bool go = active;
                for (;;) {
                    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
                    bool cand = false;
                    if (go && k < kend) {
                        o = sm.mbr[k];
                        cand = o.x <= pv.z;
                    }
                    if (!__any_sync(kFull, cand)) break;
                    go = cand;
                    bool hit = false;
                    int2 pr = make_int2(0, 0);
                    if (cand) {
                        if (o.y <= pv.w && pv.y <= o.w) {
                            const unsigned oid = sm.id[k];
                            if (reported_here(pid, oid)) {
                                hit = true;
                                pr = isR ? make_int2((int)(pid & kIdMask), (int)(oid & kIdMask))
                                         : make_int2((int)(oid & kIdMask), (int)(pid & kIdMask));
                            }
                        }
                        k++;
                    }
                    const unsigned hm = __ballot_sync(kFull, hit);
                    if (hm) {
                        const int leader = __ffs(hm) - 1;
                        unsigned pos = 0;
                        if ((int)lane == leader) pos = atomicAdd(&s_cursor, (unsigned)__popc(hm));
                        pos = __shfl_sync(kFull, pos, leader);
                        const unsigned long long at = base + pos + __popc(hm & lanemask_lt());
                        if (hit && SJ_IN(a.st, at, a.cap)) a.out[at] = pr;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Large tiles: segmented LSD radix sort (8-bit digits) of every large tile's
// R and S segments by x_l, then a pivot-parallel sweep over global memory.
// Segment 2*i / 2*i+1 = R / S entries of large tile large[i].  Every segment
// is cut into virtual blocks of kRadixBlock items; all kernels loop over
// virtual blocks (their number is read on the device).
// ----------------------------------------------------------------------------

// Segment sizes, item offsets and virtual-block offsets of the large tiles.
__global__ void __launch_bounds__(1024) k_large_prep(LargeArgs a) {
    if (block_skip(a.st)) return;
    const unsigned nl = a.st->nlarge;   // <= capacity, else the fatal bit is set
    const unsigned nseg = 2 * nl;
    const unsigned per = (nseg + 1023) / 1024;
    const unsigned s0 = threadIdx.x * per;
    unsigned long long items = 0, vbs = 0;
    for (unsigned k = 0; k < per; k++) {
        const unsigned sg = s0 + k;
        if (sg < nseg) {
            const unsigned t = a.large[sg >> 1];
            const uint2 lo = a.off[t], hi = a.off[t + 1];
            const unsigned n = (hi.x == lo.x || hi.y == lo.y) ? 0u : ((sg & 1) ? hi.y - lo.y : hi.x - lo.x);
            items += n;
            vbs += (n + kRadixBlock - 1) / kRadixBlock;
        }
    }
    // block exclusive scans (inline: two 64-bit values)
    __shared__ unsigned long long sh_i[1024], sh_v[1024];
    sh_i[threadIdx.x] = items;
    sh_v[threadIdx.x] = vbs;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        unsigned long long xi = threadIdx.x >= (unsigned)d ? sh_i[threadIdx.x - d] : 0;
        unsigned long long xv = threadIdx.x >= (unsigned)d ? sh_v[threadIdx.x - d] : 0;
        __syncthreads();
        sh_i[threadIdx.x] += xi;
        sh_v[threadIdx.x] += xv;
        __syncthreads();
    }
    unsigned long long pi = sh_i[threadIdx.x] - items, pv = sh_v[threadIdx.x] - vbs;
    for (unsigned k = 0; k < per; k++) {
        const unsigned sg = s0 + k;
        if (sg < nseg) {
            const unsigned t = a.large[sg >> 1];
            const uint2 lo = a.off[t], hi = a.off[t + 1];
            const unsigned n = (hi.x == lo.x || hi.y == lo.y) ? 0u : ((sg & 1) ? hi.y - lo.y : hi.x - lo.x);
            a.seg_off[sg] = (unsigned)pi;
            a.seg_src[sg] = (sg & 1) ? lo.y : lo.x;
            a.seg_vb[sg] = (unsigned)pv;
            pi += n;
            pv += (n + kRadixBlock - 1) / kRadixBlock;
        }
    }
    if (threadIdx.x == 1023) {
        a.seg_off[nseg] = (unsigned)sh_i[1023];
        a.seg_vb[nseg] = (unsigned)sh_v[1023];
        a.st->large_items = sh_i[1023];
        a.st->nvb = (unsigned)sh_v[1023];
        if (sh_i[1023] > a.items_cap || sh_v[1023] > a.vb_cap) atomicOr(&a.st->err, kErrLargeCap);
    }
}

// segment of virtual block vb: largest sg with seg_vb[sg] <= vb
__device__ __forceinline__ unsigned seg_of_vb(const unsigned *seg_vb, unsigned nseg, unsigned vb) {
    unsigned lo = 0, hi = nseg;
    while (hi - lo > 1) {
        unsigned mid = (lo + hi) >> 1;
        if (seg_vb[mid] <= vb) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Key and value of item q of virtual block vb (pass 0 reads the entries).
__device__ __forceinline__ void radix_item(const LargeArgs &a, int pass, unsigned sg, unsigned q,
                                           unsigned &key, unsigned &val) {
    if (pass == 0) {
        const unsigned src = a.seg_src[sg] + q;
        const float4 *ent = (sg & 1) ? a.ent_s : a.ent_r;
        key = xkey(ent[src].x);
        val = src;
    } else {
        const unsigned gi = a.seg_off[sg] + q;
        key = a.key_in[gi];
        val = a.val_in[gi];
    }
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(LargeArgs a, int pass) {
    if (block_skip(a.st)) return;
    __shared__ unsigned h[256];
    const unsigned nvb = a.st->nvb, nseg = 2 * a.st->nlarge;
    const int shift = 8 * pass;
    const unsigned lane = threadIdx.x & 31;
    for (unsigned vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const unsigned sg = seg_of_vb(a.seg_vb, nseg, vb);
        const unsigned q0 = (vb - a.seg_vb[sg]) * kRadixBlock;
        const unsigned n = a.seg_off[sg + 1] - a.seg_off[sg];
        const unsigned q1 = min(n, q0 + kRadixBlock);
        // lanes with equal digits add with one atomic (skewed tiles: long runs
        // of equal high digits)
        for (unsigned qb = q0; qb < q1; qb += kRadixThreads) {
            const unsigned q = qb + threadIdx.x;
            const bool ok = q < q1;
            unsigned key = 0, val = 0;
            if (ok) radix_item(a, pass, sg, q, key, val);
            const unsigned dg = ok ? (key >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(kFull, dg);
            if (ok && (int)lane == __ffs(peers) - 1) atomicAdd(&h[dg], (unsigned)__popc(peers));
        }
        __syncthreads();
        a.hist[(unsigned long long)vb * 256 + threadIdx.x] = h[threadIdx.x];
        __syncthreads();
    }
}

// Per segment: hist[vb][d] -> absolute destination of the first item of
// digit d of virtual block vb (digit-major order inside the segment).
__global__ void __launch_bounds__(256) k_radix_offsets(LargeArgs a) {
    if (block_skip(a.st)) return;
    constexpr int B = 8;   // virtual blocks loaded per step (independent loads in flight)
    __shared__ unsigned s_w[8];
    const unsigned nseg = 2 * a.st->nlarge;
    const unsigned d = threadIdx.x, lane = d & 31, warp = d >> 5;
    for (unsigned sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const unsigned v0 = a.seg_vb[sg], v1 = a.seg_vb[sg + 1];
        unsigned *col = a.hist + d;
        // exclusive prefix over the segment's virtual blocks, per digit
        unsigned run = 0;
        for (unsigned vb = v0; vb < v1; vb += B) {
            unsigned x[B];
#pragma unroll
            for (int k = 0; k < B; k++) x[k] = vb + k < v1 ? col[(unsigned long long)(vb + k) * 256] : 0u;
#pragma unroll
            for (int k = 0; k < B; k++)
                if (vb + k < v1) {
                    col[(unsigned long long)(vb + k) * 256] = run;
                    run += x[k];
                }
        }
        // exclusive scan of the digit totals (digit-major order in the segment)
        unsigned inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, inc, o);
            if ((int)lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        unsigned wpre = 0;
        for (unsigned k = 0; k < warp; k++) wpre += s_w[k];
        const unsigned add = wpre + inc - run + a.seg_off[sg];
        for (unsigned vb = v0; vb < v1; vb += B) {
            unsigned x[B];
#pragma unroll
            for (int k = 0; k < B; k++) x[k] = vb + k < v1 ? col[(unsigned long long)(vb + k) * 256] : 0u;
#pragma unroll
            for (int k = 0; k < B; k++)
                if (vb + k < v1) col[(unsigned long long)(vb + k) * 256] = x[k] + add;
        }
        __syncthreads();   // s_w is reused by the next segment
    }
}

// Stable scatter of a virtual block: warp w owns the block's items
// [w * 512, (w + 1) * 512) and walks them 32 at a time in order.  The warps'
// digit counts give every (warp, digit) its first destination (after the
// same digit's items of the warps before it); inside a warp, equal digits
// are ranked by lane with match_any.  Two barriers per virtual block.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(LargeArgs a, int pass) {
    if (block_skip(a.st)) return;
    constexpr int NW = kRadixThreads / 32;
    constexpr int PER = kRadixBlock / kRadixThreads;   // items per lane
    constexpr int WITEMS = kRadixBlock / NW;           // items per warp
    __shared__ unsigned s_w[NW][256];   // per-warp digit counts, then next destinations
    const unsigned nvb = a.st->nvb, nseg = 2 * a.st->nlarge;
    const int shift = 8 * pass;
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    for (unsigned vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        for (int d = lane; d < 256; d += 32) s_w[w][d] = 0;
        __syncwarp();
        const unsigned sg = seg_of_vb(a.seg_vb, nseg, vb);
        const unsigned q0 = (vb - a.seg_vb[sg]) * kRadixBlock + w * WITEMS;
        const unsigned n = a.seg_off[sg + 1] - a.seg_off[sg];
        const unsigned q1 = min(n, (vb - a.seg_vb[sg]) * kRadixBlock + kRadixBlock);
        unsigned key[PER], val[PER];
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const unsigned q = q0 + r * 32 + lane;
            key[r] = 0;
            val[r] = 0;
            if (q < q1) radix_item(a, pass, sg, q, key[r], val[r]);
        }
#pragma unroll
        for (int r = 0; r < PER; r++) {   // digit counts of this warp
            const bool ok = q0 + r * 32 + lane < q1;
            const unsigned dg = ok ? (key[r] >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(kFull, dg);
            if (ok && (int)lane == __ffs(peers) - 1) s_w[w][dg] += (unsigned)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {   // thread d: first destination of digit d for every warp
            const unsigned d = threadIdx.x;
            unsigned run = a.hist[(unsigned long long)vb * 256 + d];
            for (int ww = 0; ww < NW; ww++) {
                const unsigned c = s_w[ww][d];
                s_w[ww][d] = run;
                run += c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; r++) {   // stable placement
            const bool ok = q0 + r * 32 + lane < q1;
            const unsigned dg = ok ? (key[r] >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(kFull, dg);
            const unsigned base = ok ? s_w[w][dg] : 0u;
            __syncwarp();
            if (ok) {
                const unsigned dst = base + (unsigned)__popc(peers & lt);
                if (SJ_IN(a.st, dst, a.items_cap)) {
                    a.key_out[dst] = key[r];
                    a.val_out[dst] = val[r];
                }
                if ((int)lane == __ffs(peers) - 1) s_w[w][dg] = base + (unsigned)__popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();   // the rows are cleared for the next virtual block
    }
}

// Sorted entries of the large tiles: mbr/id gathered through the sorted values.
__global__ void __launch_bounds__(256) k_large_gather(LargeArgs a) {
    if (block_skip(a.st)) return;
    const unsigned long long n = a.st->large_items;
    const unsigned nseg = 2 * a.st->nlarge;
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n; i += 256ull * gridDim.x) {
        // segment of item i
        unsigned lo = 0, hi = nseg;
        while (hi - lo > 1) {
            unsigned mid = (lo + hi) >> 1;
            if (a.seg_off[mid] <= i) lo = mid;
            else hi = mid;
        }
        const unsigned v = a.val_in[i];
        const float4 m = (lo & 1) ? a.ent_s[v] : a.ent_r[v];
        a.lmbr[i] = m;
        a.lid[i] = (lo & 1) ? a.id_s[v] : a.id_r[v];
        if (a.ly) a.ly[i] = make_float2(m.y, m.w);
    }
}

// Sweep of the large tiles: every entry is a pivot; virtual blocks of
// kRadixBlock pivots are taken from a device counter.
template <int MODE>
__global__ void __launch_bounds__(256) k_sweep_large(LargeArgs a, SweepArgs o) {
    if (block_skip(o.st)) return;
    __shared__ unsigned s_vb;
    __shared__ unsigned s_cursor;
    __shared__ unsigned long long s_base;
    __shared__ int s_ok;
    __shared__ unsigned s_red[8];
    const unsigned nvb_all = a.st->nvb;
    const unsigned nlist = o.list ? *o.list_n : nvb_all;
    const unsigned nseg = 2 * a.st->nlarge;
    const unsigned lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            s_vb = atomicAdd(&o.st->work[o.work_slot], 1u);
            s_cursor = 0;
        }
        __syncthreads();
        const unsigned item = s_vb;
        if (item >= nlist) break;
        const unsigned vb = o.list ? o.list[item] : item;
        const unsigned sg = seg_of_vb(a.seg_vb, nseg, vb);
        const bool isR = (sg & 1) == 0;
        const unsigned og = sg ^ 1u;
        const int o0 = (int)a.seg_off[og], o1 = (int)a.seg_off[og + 1];
        const unsigned q0 = a.seg_off[sg] + (vb - a.seg_vb[sg]) * kRadixBlock;
        const unsigned q1 = min(a.seg_off[sg + 1], q0 + kRadixBlock);
        const unsigned tile = a.large[sg >> 1];
        auto setup = [&](unsigned p, float4 &pv, unsigned &pid, int &k) {
            pv = a.lmbr[p];
            pid = a.lid[p];
            if (isR) k = lower_pos<true>(o0, o1, pv.x, [&](int q) { return a.lmbr[q].x; });
            else k = lower_pos<false>(o0, o1, pv.x, [&](int q) { return a.lmbr[q].x; });
        };
        unsigned long long base = 0;
        bool do_write = MODE == MODE_WRITE;
        if (MODE != MODE_WRITE) {
            unsigned my = 0;
            for (unsigned p = q0 + threadIdx.x; p < q1; p += 256) {
                float4 pv;
                unsigned pid;
                int k;
                setup(p, pv, pid, k);
                unsigned cnt = 0;
                for (; k < o1; k++) {
                    const float4 ob = a.lmbr[k];
                    if (ob.x > pv.z) break;
                    if (ob.y <= pv.w && pv.y <= ob.w && reported_here(pid, a.lid[k])) cnt++;
                }
                my += cnt;
            }
            if (MODE == MODE_TILES) {
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) my += __shfl_xor_sync(kFull, my, d);
                if (lane == 0 && my) atomicAdd(o.tile_pairs + tile, my);
                __syncthreads();
                continue;
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) my += __shfl_xor_sync(kFull, my, d);
            if (lane == 0) s_red[threadIdx.x >> 5] = my;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned tot = 0;
                for (int w = 0; w < 8; w++) tot += s_red[w];
                if (MODE == MODE_COUNT) {
                    o.cnt_out[o.cnt_base + vb] = tot;
                } else {
                    const unsigned long long b = atomicAdd(&o.st->npairs, (unsigned long long)tot);
                    o.resv[o.cnt_base + vb] = b;
                    const bool ok = tot == 0 || b + tot <= o.cap;
                    s_ok = ok;
                    s_base = b;
                    if (!ok) {
                        const unsigned f = atomicAdd(o.nfail, 1u);
                        o.fail[f] = vb;
                    }
                }
            }
            __syncthreads();
            if (MODE == MODE_COUNT) continue;
            do_write = s_ok;
            base = s_base;
        } else {
            base = o.off_in[o.cnt_base + vb];
        }
        if (!do_write) {
            __syncthreads();
            continue;
        }
        for (unsigned pb = q0; pb < q1; pb += 256) {
            const unsigned p = pb + threadIdx.x;
            const bool active = p < q1;
            float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned pid = 0;
            int k = 0;
            if (active) setup(p, pv, pid, k);
            bool go = active;
            for (;;) {
                float4 ob = make_float4(0.f, 0.f, 0.f, 0.f);
                bool cand = false;
                if (go && k < o1) {
                    ob = a.lmbr[k];
                    cand = ob.x <= pv.z;
                }
                if (!__any_sync(kFull, cand)) break;
                go = cand;
                bool hit = false;
                int2 pr = make_int2(0, 0);
                if (cand) {
                    if (ob.y <= pv.w && pv.y <= ob.w) {
                        const unsigned oid = a.lid[k];
                        if (reported_here(pid, oid)) {
                            hit = true;
                            pr = isR ? make_int2((int)(pid & kIdMask), (int)(oid & kIdMask))
                                     : make_int2((int)(oid & kIdMask), (int)(pid & kIdMask));
                        }
                    }
                    k++;
                }
                const unsigned hm = __ballot_sync(kFull, hit);
                if (hm) {
                    const int leader = __ffs(hm) - 1;
                    unsigned pos = 0;
                    if ((int)lane == leader) pos = atomicAdd(&s_cursor, (unsigned)__popc(hm));
                    pos = __shfl_sync(kFull, pos, leader);
                    const unsigned long long at = base + pos + __popc(hm & lanemask_lt());
                if (hit && SJ_IN(o.st, at, o.cap)) o.out[at] = pr;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Candidate-parallel sweep of the large tiles.  A pivot of a large tile can
// have millions of candidates (a wide rectangle over a dense tile), so the
// work is divided by candidates, not by pivots:
//  1. k_large_ranges (one CTA per virtual block): every pivot's candidate
//     range [start, end) in the other segment -- the positions the forward
//     scan of Algorithm 1 visits: x_l in (x_l, x_u] of an R pivot, in
//     [x_l, x_u] of an S pivot -- and the exclusive prefix of the range
//     sizes within the virtual block;
//  2. k_large_plan (one CTA): kCandChunk candidates per chunk, the chunks of
//     every virtual block and their prefix;
//  3. k_large_cand: persistent CTAs take chunks; every thread tests its
//     candidates (y-test, reference-point test of Eq. 1); a chunk's pairs
//     are counted per virtual block, or collected in shared memory and
//     written with one atomic on the virtual block's cursor, at the block's
//     offset from the count pass;
//  4. k_large_finish (count pass): the per-block counts as 32-bit work-item
//     counts of the pair scan.
// ---------------------------------------------------------------------------
constexpr int kCandChunk = kLargeCandChunk;
constexpr int kCandThreads = 256;

// Exclusive scan over the NT threads of a block; *total = sum.  Every warp
// writes only its own slot of s_w before the first barrier, so consecutive
// calls may share s_w.
template <int NT, typename T>
__device__ __forceinline__ T block_scan_ex(T v, T *s_w, T *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T o = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const T x = lane < NT / 32 ? s_w[lane] : T(0);
        T xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T o = __shfl_up_sync(kFull, xi, d);
            if (lane >= d) xi += o;
        }
        if (lane < NT / 32) s_w[lane] = xi - x;
        if (lane == NT / 32 - 1) s_w[NT / 32] = xi;
    }
    __syncthreads();
    *total = s_w[NT / 32];
    return s_w[wid] + inc - v;
}

// Pivots [q0, q1) of virtual block vb, its segment sg and the other segment's range.
struct VbRange {
    unsigned sg, q0, q1;
    int o0, o1;
};
__device__ __forceinline__ VbRange vb_range(const LargeArgs &a, unsigned nseg, unsigned vb) {
    VbRange r;
    r.sg = seg_of_vb(a.seg_vb, nseg, vb);
    const unsigned og = r.sg ^ 1u;
    r.o0 = (int)a.seg_off[og];
    r.o1 = (int)a.seg_off[og + 1];
    r.q0 = a.seg_off[r.sg] + (vb - a.seg_vb[r.sg]) * kRadixBlock;
    r.q1 = min(a.seg_off[r.sg + 1], r.q0 + kRadixBlock);
    return r;
}

__global__ void __launch_bounds__(kCandThreads) k_large_ranges(LargeArgs a) {
    __shared__ unsigned long long s_w[kCandThreads / 32 + 1];
    if (block_skip(a.st)) return;
    const unsigned nvb = min(a.st->nvb, a.vb_cap), nseg = 2 * a.st->nlarge;
    auto getx = [&](int q) { return a.lmbr[q].x; };
    for (unsigned vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        const VbRange v = vb_range(a, nseg, vb);
        const bool isR = (v.sg & 1) == 0;
        unsigned long long carry = 0;
        for (unsigned pb = v.q0; pb < v.q1; pb += kCandThreads) {
            const unsigned p = pb + threadIdx.x;
            unsigned long long num = 0;
            if (p < v.q1) {
                const float4 pv = a.lmbr[p];
                const int k = isR ? lower_pos<true>(v.o0, v.o1, pv.x, getx) : lower_pos<false>(v.o0, v.o1, pv.x, getx);
                // end = first x_l > x_u: gallop from k (the range [lo, lo + len) is
                // known to lie at or below x_u while its last element does), then
                // search the last interval
                int lo = k, len = 1;
                while (lo + len - 1 < v.o1 && getx(lo + len - 1) <= pv.z) {
                    lo += len;
                    len <<= 1;
                }
                const int e = lower_pos<true>(lo, min(v.o1, lo + len - 1), pv.z, getx);
                a.lstart[p] = (unsigned)k;
                num = (unsigned long long)(e - k);
            }
            unsigned long long tot;
            const unsigned long long ex = carry + block_scan_ex<kCandThreads>(num, s_w, &tot);
            if (p < v.q1) a.lcoff[p] = ex;
            carry += tot;
        }
        if (threadIdx.x == 0) a.vbc[vb] = carry;
    }
}

__global__ void __launch_bounds__(1024) k_large_plan(LargeArgs a) {
    __shared__ unsigned long long s_w[33];
    if (block_skip(a.st)) return;
    const unsigned nvb = min(a.st->nvb, a.vb_cap);
    unsigned long long carry = 0;
    for (unsigned b0 = 0; b0 < nvb; b0 += 1024) {
        const unsigned vb = b0 + threadIdx.x;
        unsigned long long ch = 0;
        if (vb < nvb) {
            ch = (a.vbc[vb] + kCandChunk - 1) / kCandChunk;
            a.vbpairs[vb] = 0;
            a.vbcur[vb] = 0;
        }
        unsigned long long tot;
        const unsigned long long ex = carry + block_scan_ex<1024>(ch, s_w, &tot);
        if (vb < nvb) a.vbch[vb] = (unsigned)ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        a.vbch[nvb] = (unsigned)carry;
        a.st->nlch = (unsigned)carry;
        if (carry > 0xffffffffull) atomicOr(&a.st->err, kErrLargeCap);
    }
}

// Last p in [lo, hi] with lcoff[p] <= c (lcoff[lo] <= c).
__device__ __forceinline__ unsigned cand_owner(const unsigned long long *lcoff, unsigned lo, unsigned hi,
                                               unsigned long long c) {
    hi += 1;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (lcoff[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Same, knowing lcoff[lo] <= c and that the answer is usually near lo:
// gallop up from lo, then search the last interval.
__device__ __forceinline__ unsigned cand_owner_from(const unsigned long long *lcoff, unsigned lo, unsigned hi,
                                                    unsigned long long c) {
    unsigned step = 1;
    while (lo < hi) {
        const unsigned b = min(hi, lo + step);
        if (lcoff[b] <= c) {
            lo = b;
            step <<= 1;
        } else {
            return cand_owner(lcoff, lo, b - 1, c);
        }
    }
    return lo;
}

// CTAs take groups of kCandGroup consecutive chunks from a counter; inside
// a group, thread 0 walks the virtual blocks and the pivots forward from
// one chunk to the next instead of searching them anew.
template <int MODE>
__global__ void __launch_bounds__(kCandThreads) k_large_cand(LargeArgs a, SweepArgs o) {
    __shared__ int2 s_pairs[kCandChunk];   // MODE_WRITE: the chunk's pairs
    __shared__ unsigned s_vb, s_sg, s_pa, s_pb, s_n, s_q0;
    __shared__ unsigned long long s_c0, s_c1, s_base;
    __shared__ float2 s_pv;
    __shared__ unsigned s_pid;
    __shared__ unsigned s_red[kCandThreads / 32];
    if (block_skip(o.st)) return;
    const unsigned nch = a.st->nlch, nvb = min(a.st->nvb, a.vb_cap), nseg = 2 * a.st->nlarge;
    const unsigned lane = threadIdx.x & 31;
    constexpr int kU = 4;   // candidates a thread loads before testing them
    constexpr unsigned kCandGroup = 8;
    __shared__ unsigned s_w0;
    unsigned t_vb = 0xffffffffu, t_q1 = 0, t_sg = 0, t_prev = 0;   // thread 0's walk
    for (;;) {
        if (threadIdx.x == 0) {
            s_w0 = atomicAdd(&o.st->work[o.work_slot], 1u) * kCandGroup;
            t_vb = 0xffffffffu;
        }
        __syncthreads();
        const unsigned w0 = s_w0;
        if (w0 >= nch) break;
        const unsigned w1 = min(nch, w0 + kCandGroup);
        for (unsigned w = w0; w < w1; w++) {
            if (threadIdx.x == 0) {
                s_n = 0;
                if (t_vb == 0xffffffffu || w >= a.vbch[t_vb + 1]) {   // the next virtual block with chunk w
                    if (t_vb == 0xffffffffu) {
                        unsigned lo = 0, hi = nvb;   // last vb with vbch[vb] <= w
                        while (hi - lo > 1) {
                            const unsigned mid = (lo + hi) >> 1;
                            if (a.vbch[mid] <= w) lo = mid;
                            else hi = mid;
                        }
                        t_vb = lo;
                    } else {
                        do t_vb++;
                        while (a.vbch[t_vb + 1] <= w);
                    }
                    const VbRange v = vb_range(a, nseg, t_vb);
                    t_q1 = v.q1;
                    t_sg = v.sg;
                    t_prev = v.q0;
                }
                const unsigned long long c0 = (unsigned long long)(w - a.vbch[t_vb]) * kCandChunk;
                const unsigned long long c1 = min(c0 + (unsigned long long)kCandChunk, a.vbc[t_vb]);
                const unsigned pa = cand_owner_from(a.lcoff, t_prev, t_q1 - 1, c0);
                const unsigned pb = cand_owner_from(a.lcoff, pa, t_q1 - 1, c1 - 1);
                t_prev = pb;
                s_vb = t_vb;
                s_sg = t_sg;
                s_c0 = c0;
                s_c1 = c1;
                s_pa = pa;
                s_pb = pb;
                if (pa == pb) {   // one pivot owns the whole chunk (a heavy pivot): its data once
                    s_pv = a.ly[pa];
                    s_pid = a.lid[pa];
                    s_q0 = a.lstart[pa] + (unsigned)(c0 - a.lcoff[pa]);
                }
            }
            __syncthreads();
            const unsigned vb = s_vb, pa = s_pa, pb = s_pb;
            const bool isR = (s_sg & 1) == 0;
            const unsigned long long c0 = s_c0, c1 = s_c1;
            const unsigned nc = (unsigned)(c1 - c0);   // <= kCandChunk
            const bool single = pa == pb;
            unsigned my = 0;
            for (unsigned jb = 0; jb < nc; jb += kCandThreads * kU) {
                // the candidates lie in the pivot's x range by construction: the
                // test reads only the y extents (8 bytes) and ids of both
                float2 pv[kU], ob[kU];
                unsigned pid[kU], oid[kU];
                bool ok[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) {   // loads of kU candidates
                    const unsigned j = jb + u * kCandThreads + threadIdx.x;
                    ok[u] = j < nc;
                    if (!ok[u]) continue;
                    unsigned q;
                    if (single) {
                        pv[u] = s_pv;
                        pid[u] = s_pid;
                        q = s_q0 + j;
                    } else {
                        const unsigned long long c = c0 + j;
                        const unsigned p = cand_owner(a.lcoff, pa, pb, c);
                        q = a.lstart[p] + (unsigned)(c - a.lcoff[p]);
                        pv[u] = a.ly[p];
                        pid[u] = a.lid[p];
                    }
                    ob[u] = a.ly[q];
                    oid[u] = a.lid[q];
                }
#pragma unroll
                for (int u = 0; u < kU; u++) {   // y-test, reference-point test, emission
                    const bool hit = ok[u] && ob[u].x <= pv[u].y && pv[u].x <= ob[u].y && reported_here(pid[u], oid[u]);
                    if (MODE == MODE_WRITE || MODE == MODE_APPEND) {
                        const unsigned hm = __ballot_sync(kFull, hit);
                        if (hm) {
                            unsigned pos = 0;
                            if (lane == (unsigned)(__ffs(hm) - 1)) pos = atomicAdd(&s_n, (unsigned)__popc(hm));
                            pos = __shfl_sync(kFull, pos, __ffs(hm) - 1) + __popc(hm & lanemask_lt());
                            if (hit && SJ_IN(o.st, pos, kCandChunk))
                                s_pairs[pos] = isR ? make_int2((int)(pid[u] & kIdMask), (int)(oid[u] & kIdMask))
                                                   : make_int2((int)(oid[u] & kIdMask), (int)(pid[u] & kIdMask));
                        }
                    } else {
                        my += hit;
                    }
                }
            }
            if (MODE == MODE_WRITE || MODE == MODE_APPEND) {
                __syncthreads();
                if (threadIdx.x == 0 && s_n) {
                    if (MODE == MODE_APPEND) {   // one pass: the chunk's range from one atomic
                        s_base = o.base + atomicAdd(o.append, (unsigned long long)s_n);
                        if (s_base + s_n > o.cap) atomicOr(&o.st->err, kErrOutCap);
                    } else {
                        s_base = o.off_in[o.cnt_base + vb] + atomicAdd(&a.vbcur[vb], (unsigned long long)s_n);
                    }
                }
                __syncthreads();
                const unsigned n = (MODE == MODE_APPEND && s_base + s_n > o.cap) ? 0u : s_n;
                for (unsigned i = threadIdx.x; i < n; i += kCandThreads)
                    if (SJ_IN(o.st, s_base + i, o.cap)) o.out[s_base + i] = s_pairs[i];
            } else {
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) my += __shfl_xor_sync(kFull, my, d);
                if (lane == 0) s_red[threadIdx.x >> 5] = my;
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned tot = 0;
                    for (int w = 0; w < kCandThreads / 32; w++) tot += s_red[w];
                    if (tot) {
                        if (MODE == MODE_TILES) atomicAdd(o.tile_pairs + a.large[s_sg >> 1], tot);
                        else atomicAdd(&a.vbpairs[vb], (unsigned long long)tot);
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void k_large_finish(LargeArgs a, SweepArgs o) {
    const unsigned nvb = min(a.st->nvb, a.vb_cap);
    for (unsigned vb = blockIdx.x * blockDim.x + threadIdx.x; vb < nvb; vb += gridDim.x * blockDim.x) {
        const unsigned long long v = a.vbpairs[vb];
        if (v > 0xffffffffull) atomicOr(&a.st->err, kErrLargeCap);   // one work item over 2^32 pairs
        o.cnt_out[o.cnt_base + vb] = (unsigned)v;
    }
}

// Exclusive scan of n uint32 pair counts into uint64 offsets; the total goes
// to st->npairs.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_pairs(const unsigned *__restrict__ cnt, unsigned n,
                                                     unsigned long long *__restrict__ off,
                                                     Stats *__restrict__ st) {
    __shared__ unsigned long long sh[1024];
    const unsigned per = (n + 1023) / 1024;
    const unsigned i0 = threadIdx.x * per;
    unsigned long long sum = 0;
    for (unsigned k = 0; k < per; k++)
        if (i0 + k < n) sum += cnt[i0 + k];
    sh[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        unsigned long long x = threadIdx.x >= (unsigned)d ? sh[threadIdx.x - d] : 0;
        __syncthreads();
        sh[threadIdx.x] += x;
        __syncthreads();
    }
    unsigned long long run = sh[threadIdx.x] - sum;
    for (unsigned k = 0; k < per; k++)
        if (i0 + k < n) {
            off[i0 + k] = run;
            run += cnt[i0 + k];
        }
    if (threadIdx.x == 1023) st->npairs = sh[1023];
}

// ---- launchers ---------------------------------------------------------------
size_t sweep_smem_bytes() { return sizeof(SmemChunk); }

cudaError_t sweep_setup() {
    cudaError_t e;
    const int sm = (int)sizeof(SmemChunk);
    if ((e = cudaFuncSetAttribute(k_sweep_chunks<MODE_COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_sweep_chunks<MODE_WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_sweep_chunks<MODE_RESERVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_sweep_chunks<MODE_TILES>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    return cudaSuccess;
}

int sweep_blocks_per_sm() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_chunks<MODE_WRITE>, kSweepThreads,
                                                  sizeof(SmemChunk));
    return nb > 0 ? nb : 1;
}

cudaError_t launch_sweep_chunks(int mode, const SweepArgs &a, int grid, cudaStream_t s) {
    const size_t sm = sizeof(SmemChunk);
    switch (mode) {
        case MODE_COUNT: k_sweep_chunks<MODE_COUNT><<<grid, kSweepThreads, sm, s>>>(a); break;
        case MODE_WRITE: k_sweep_chunks<MODE_WRITE><<<grid, kSweepThreads, sm, s>>>(a); break;
        case MODE_RESERVE: k_sweep_chunks<MODE_RESERVE><<<grid, kSweepThreads, sm, s>>>(a); break;
        default: k_sweep_chunks<MODE_TILES><<<grid, kSweepThreads, sm, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_large_sort(LargeArgs a, int grid, cudaStream_t s) {
    k_large_prep<<<1, 1024, 0, s>>>(a);
    for (int pass = 0; pass < 4; pass++) {
        k_radix_hist<<<grid, kRadixThreads, 0, s>>>(a, pass);
        k_radix_offsets<<<grid, 256, 0, s>>>(a);
        k_radix_scatter<<<grid, kRadixThreads, 0, s>>>(a, pass);
        // ping-pong
        unsigned *tk = a.key_in;
        a.key_in = a.key_out;
        a.key_out = tk;
        unsigned *tv = a.val_in;
        a.val_in = a.val_out;
        a.val_out = tv;
        if (pass == 0) {
            // pass 0 read the entries; later passes read key_in/val_in, which
            // now hold pass 0's output.  Nothing else to do.
        }
    }
    k_large_gather<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_large(int mode, const LargeArgs &a, const SweepArgs &o, int grid,
                               cudaStream_t s) {
    if (a.lcoff && !o.list && mode != MODE_RESERVE) {   // candidate-parallel
        k_large_ranges<<<grid, kCandThreads, 0, s>>>(a);
        k_large_plan<<<1, 1024, 0, s>>>(a);
        switch (mode) {
            case MODE_COUNT: k_large_cand<MODE_COUNT><<<grid, kCandThreads, 0, s>>>(a, o); break;
            case MODE_WRITE: k_large_cand<MODE_WRITE><<<grid, kCandThreads, 0, s>>>(a, o); break;
            default: k_large_cand<MODE_TILES><<<grid, kCandThreads, 0, s>>>(a, o); break;
        }
        if (mode == MODE_COUNT) k_large_finish<<<grid, 256, 0, s>>>(a, o);
        return cudaGetLastError();
    }
    switch (mode) {
        case MODE_COUNT: k_sweep_large<MODE_COUNT><<<grid, 256, 0, s>>>(a, o); break;
        case MODE_WRITE: k_sweep_large<MODE_WRITE><<<grid, 256, 0, s>>>(a, o); break;
        case MODE_RESERVE: k_sweep_large<MODE_RESERVE><<<grid, 256, 0, s>>>(a, o); break;
        default: k_sweep_large<MODE_TILES><<<grid, 256, 0, s>>>(a, o); break;
    }
    return cudaGetLastError();
}

// One-pass large tiles: the candidate ranges and chunks (before the count is
// known), then the candidate sweep appending each chunk's pairs.
cudaError_t launch_large_plan(const LargeArgs &a, int grid, cudaStream_t s) {
    k_large_ranges<<<grid, kCandThreads, 0, s>>>(a);
    k_large_plan<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_large_append(const LargeArgs &a, const SweepArgs &o, int grid, cudaStream_t s) {
    k_large_cand<MODE_APPEND><<<grid, kCandThreads, 0, s>>>(a, o);
    return cudaGetLastError();
}

cudaError_t launch_scan_pairs(const unsigned *cnt, unsigned n, unsigned long long *off, Stats *st,
                              cudaStream_t s) {
    k_scan_pairs<<<1, 1024, 0, s>>>(cnt, n, off, st);
    return cudaGetLastError();
}

}  // namespace sj
