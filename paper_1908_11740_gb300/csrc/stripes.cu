// stripes.cu -- 1D partitioning (Sec. 3.1): vertical stripes (an nx x 1
// grid) swept along y, or horizontal stripes (1 x ny) swept along x -- the
// axis along the stripe, which the paper finds to be the better sweep axis
// for stripes in every case (Sec. 3.3) -- with the duplicate test of one
// comparison (Sec. 3.2: a pair is reported in the stripe where its
// max(r.x_l, s.x_l) falls, for vertical stripes).
//
//  1. The L1 partition of the two-level path with blocks of a single tile:
//     every rectangle is written into every stripe it overlaps (k_bcount,
//     the block scan and k_bscatter_shared with G = 1).  Each stripe's R and
//     S entries are then contiguous runs of 32-byte L1 entries.
//  2. k_stripe_join: persistent, one CTA of 1024 threads per stripe (taken
//     from a counter).  The stripe's keys -- the order-preserving image of
//     the lower coordinate along the stripe -- of its S entries, then its R
//     entries, are sorted together in shared memory by a stable LSD radix
//     sort (4 passes of 8-bit digits, per-warp digit counts, a digit-major
//     exclusive scan, and a stable scatter in which every warp walks its
//     items 32 at a time in order, ranking equal digits by lane).  S before
//     R on equal keys is Algorithm 1's tie rule, so the candidates of every
//     entry follow it in the merged order: each entry is a pivot of the
//     forward scan along the stripe, from its own sorted position, over the
//     other side's entries whose lower coordinate is at most its upper one.
//     Such a candidate intersects along the stripe by construction, so only
//     the other axis is tested, and the pair is reported when the stripe is
//     the one that holds its reference point.  Candidates are read from their
//     L1 entries.
//  3. Two passes: count (pairs per stripe), scan, exact allocation, write.
//     The count pass stores every stripe's sorted keys and order (6 bytes an
//     entry, at the stripe's R start + S start, which are disjoint ranges);
//     the write pass loads them instead of sorting again.
// A stripe with more entries than shared memory holds sends the join to the
// general path.
#define SJ_FILE_CODE 4
#include <string.h>

#include <algorithm>

#include "sj_blocked.h"
#include "sj_internal.h"

namespace sj {

constexpr int kStThreads = 1024;
constexpr int kStWarps = kStThreads / 32;
constexpr int kStCap = 16384;   // R + S entries of one stripe joined in shared memory

struct StSmem {
    unsigned key[kStCap];            // sorted keys of the stripe's S and R entries (merged)
    unsigned short val[kStCap];      // merged index of each key's entry: S in [0, ns), R in [ns, n)
    unsigned tkey[kStCap];           // radix ping-pong
    unsigned short tval[kStCap];     // radix ping-pong; then the sorted position of every entry
    unsigned hist[kStWarps * 256];   // per-warp digit counts, then running offsets
};

__device__ __forceinline__ unsigned st_lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan over the 1024 threads of v (in thread order); two barriers.
__device__ __forceinline__ unsigned st_scan(unsigned v, unsigned *s_w) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
        if ((int)lane >= d) inc += o;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned x = s_w[lane];
        unsigned xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(0xffffffffu, xi, d);
            if ((int)lane >= d) xi += o;
        }
        s_w[lane] = xi - x;
    }
    __syncthreads();
    return s_w[warp] + inc - v;
}

// Stable LSD radix sort of (ka, va)[0, n) by the 32-bit keys; (kb, vb) is
// scratch of n items.  The result is back in (ka, va) (4 passes).
__device__ void st_sort(unsigned *ka, unsigned short *va, unsigned *kb, unsigned short *vb, int n, unsigned *hist,
                        unsigned *s_w) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = st_lanemask_lt();
    const int m = (n + kStWarps - 1) / kStWarps;   // items of each warp, contiguous
    const int w0 = min(n, (int)warp * m), w1 = min(n, w0 + m);
    unsigned *hw = hist + warp * 256;
    for (int pass = 0; pass < 4; pass++) {
        const int sh = 8 * pass;
        const unsigned *sk = (pass & 1) ? kb : ka;
        const unsigned short *sv = (pass & 1) ? vb : va;
        unsigned *dk = (pass & 1) ? ka : kb;
        unsigned short *dv = (pass & 1) ? va : vb;
        for (int d = lane; d < 256; d += 32) hw[d] = 0;
        __syncwarp();
        // digit counts of this warp's items
        for (int i = w0 + (int)lane; i - (int)lane < w1; i += 32) {
            const bool ok = i < w1;
            const unsigned d = ok ? (sk[i] >> sh) & 0xffu : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (ok && (int)lane == __ffs(peers) - 1) hw[d] += (unsigned)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // digit-major exclusive scan: thread t holds digit t / 4 of warps
        // 8 (t % 4) .. 8 (t % 4) + 7
        {
            const int d = threadIdx.x >> 2, q = threadIdx.x & 3;
            unsigned v[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                v[j] = hist[(q * 8 + j) * 256 + d];
                sum += v[j];
            }
            unsigned ex = st_scan(sum, s_w);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                hist[(q * 8 + j) * 256 + d] = ex;
                ex += v[j];
            }
        }
        __syncthreads();
        // stable scatter: chunks of 32 in order, equal digits ranked by lane
        for (int i = w0 + (int)lane; i - (int)lane < w1; i += 32) {
            const bool ok = i < w1;
            const unsigned k = ok ? sk[i] : 0u;
            const unsigned short v = ok ? sv[i] : (unsigned short)0;
            const unsigned d = ok ? (k >> sh) & 0xffu : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const unsigned base = ok ? hw[d] : 0u;
            __syncwarp();
            if (ok) {
                const unsigned pos = base + (unsigned)__popc(peers & lt);
                dk[pos] = k;
                dv[pos] = v;
                if ((int)lane == __ffs(peers) - 1) hw[d] = base + (unsigned)__popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

struct StArgs {
    const BEnt *bent_r, *bent_s;
    const uint4 *imeta;        // per work item: block, R start, R count, S start
    const unsigned *ins;       // per work item: S count
    int bx;                    // stripes per row of the block grid (G = 1: blocks are tiles)
    int vert;                  // 1: vertical stripes (nx x 1), swept along y; 0: along x
    unsigned *skey;            // sorted keys of every stripe (count pass writes, write pass reads)
    unsigned short *sval;      // ... and the merged index of each sorted position
    unsigned long long scap;   // entries skey / sval hold
    Stats *st;
};

template <int MODE>
__global__ void __launch_bounds__(kStThreads, 1) k_stripe_join(StArgs a, BJoinOut o) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    StSmem &sm = *reinterpret_cast<StSmem *>(smem_raw);
    __shared__ unsigned s_w[32];
    __shared__ unsigned s_item, s_cnt;
    // a stripe beyond shared memory (flagged by the block scan) sends the
    // join to the general path, whose L1 write then did not run: stop here
    if (block_skip_blocked(a.st)) return;
    const unsigned nitems = a.st->nchunks;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(&a.st->work[o.work_slot], 1u);
            s_cnt = 0;
        }
        __syncthreads();
        const unsigned it = s_item;
        if (it >= nitems) break;
        const uint4 mt = a.imeta[it];
        const int nr = (int)mt.z, ns = (int)a.ins[it], n = nr + ns;
        const int col = (int)(mt.x % (unsigned)a.bx), row = (int)(mt.x / (unsigned)a.bx);
        const BEnt *er = a.bent_r + mt.y, *es = a.bent_s + mt.w;
        if (n > kStCap) {   // beyond shared memory: the general path joins this input
            if (threadIdx.x == 0) {
                atomicOr(&a.st->need_direct, 1);
                if (MODE == MODE_COUNT) o.cnt_out[it] = 0;
            }
            __syncthreads();
            continue;
        }
        const unsigned long long sbase = (unsigned long long)mt.y + mt.w;   // this stripe's sorted order
        const bool keep = a.skey && sbase + (unsigned long long)n <= a.scap;   // room for the stored order
        if (MODE == MODE_WRITE && keep) {   // the count pass's order
            for (int k = threadIdx.x; k < n; k += kStThreads) {
                sm.key[k] = a.skey[sbase + k];
                sm.val[k] = a.sval[sbase + k];
            }
            __syncthreads();
        } else {
            // keys of the lower coordinate along the stripe, S first, then R:
            // the stable sort then puts S before R on equal keys, which is
            // Algorithm 1's tie rule (on r.x_l == s.x_l, s is the pivot), so
            // every pivot's candidates follow it in the merged order
            for (int e = threadIdx.x; e < n; e += kStThreads) {
                const bool isS = e < ns;
                const float4 m = (isS ? es[e] : er[e - ns]).mbr;
                sm.key[e] = xkey(a.vert ? m.y : m.x);
                sm.val[e] = (unsigned short)e;
            }
            __syncthreads();
            st_sort(sm.key, sm.val, sm.tkey, sm.tval, n, sm.hist, s_w);
            if (MODE == MODE_COUNT && keep)
                for (int k = threadIdx.x; k < n; k += kStThreads) {
                    a.skey[sbase + k] = sm.key[k];
                    a.sval[sbase + k] = sm.val[k];
                }
        }
        // position of every entry in the merged order (tval is free now)
        for (int k = threadIdx.x; k < n; k += kStThreads)
            if (SJ_IN(a.st, sm.val[k], n)) sm.tval[sm.val[k]] = (unsigned short)k;
        __syncthreads();
        // every entry is a pivot of the forward scan along the stripe: the
        // other side's entries after it, while their lower coordinate is at
        // most its upper one (for an R pivot those have a key above its own;
        // for an S pivot, at least its own)
        unsigned my = 0;
        for (int e = threadIdx.x; e < n; e += kStThreads) {
            const bool isS = e < ns;
            uint4 mh, mt2;   // the pivot's entry: MBR, then id, columns, rows
            load_bent(reinterpret_cast<const uint4 *>(isS ? es + e : er + (e - ns)), mh, mt2);
            const float4 m = make_float4(__uint_as_float(mh.x), __uint_as_float(mh.y), __uint_as_float(mh.z),
                                         __uint_as_float(mh.w));
            const unsigned pid = mt2.x;
            const int cx0 = (int)(mt2.y & 0xffffu), cy0 = (int)(mt2.z & 0xffffu);
            const float hi = a.vert ? m.w : m.z;
            const float olo = a.vert ? m.x : m.y, ohi = a.vert ? m.z : m.w;
            const unsigned khi = xkey(hi);
            for (int k = (int)sm.tval[e] + 1; k < n && sm.key[k] <= khi; k++) {
                const unsigned c = SJ_AT(a.st, sm.val[k], n);
                const bool cS = c < (unsigned)ns;
                if (cS == isS) continue;   // same side
                uint4 ch, ct;   // the candidate's entry
                load_bent(reinterpret_cast<const uint4 *>(cS ? es + c : er + (c - ns)), ch, ct);
                const float clo = __uint_as_float(a.vert ? ch.x : ch.y), chi = __uint_as_float(a.vert ? ch.z : ch.w);
                if (!(clo <= ohi && olo <= chi)) continue;
                // Eq. 1 in 1D: the pair's reference point lies in this stripe
                const int ccx0 = (int)(ct.y & 0xffffu), ccy0 = (int)(ct.z & 0xffffu);
                if (max(cx0, ccx0) != col || max(cy0, ccy0) != row) continue;
                if (MODE == MODE_COUNT) {
                    my++;
                } else {
                    const unsigned oid = ct.x;
                    const int2 pr = isS ? make_int2((int)oid, (int)pid) : make_int2((int)pid, (int)oid);
                    const unsigned msk = __activemask();
                    const int leader = __ffs(msk) - 1;
                    unsigned pos = 0;
                    if ((int)(threadIdx.x & 31) == leader) pos = atomicAdd(&s_cnt, (unsigned)__popc(msk));
                    pos = __shfl_sync(msk, pos, leader) + (unsigned)__popc(msk & st_lanemask_lt());
                    if (SJ_IN(a.st, o.off_in[it] + pos, o.cap)) o.out[o.off_in[it] + pos] = pr;
                }
            }
        }
        if (MODE == MODE_COUNT) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) my += __shfl_xor_sync(0xffffffffu, my, d);
            if ((threadIdx.x & 31) == 0 && my) atomicAdd(&s_cnt, my);
            __syncthreads();
            if (threadIdx.x == 0) o.cnt_out[it] = s_cnt;
        }
        __syncthreads();
    }
}

size_t stripe_smem_bytes() { return sizeof(StSmem); }

cudaError_t stripe_setup() {
    cudaError_t e;
    const int sm = (int)sizeof(StSmem);
    if ((e = cudaFuncSetAttribute(k_stripe_join<MODE_COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    return cudaFuncSetAttribute(k_stripe_join<MODE_WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t launch_stripe_join(int mode, const BArgs &b, int vert, unsigned *skey, unsigned short *sval,
                               unsigned long long scap, const BJoinOut &o, int grid, cudaStream_t s) {
    StArgs a;
    a.bent_r = b.bent_r;
    a.bent_s = b.bent_s;
    a.imeta = b.imeta;
    a.ins = b.ins;
    a.bx = b.bx;
    a.vert = vert;
    a.skey = skey;
    a.sval = sval;
    a.scap = scap;
    a.st = b.st;
    if (mode == MODE_COUNT) k_stripe_join<MODE_COUNT><<<grid, kStThreads, sizeof(StSmem), s>>>(a, o);
    else k_stripe_join<MODE_WRITE><<<grid, kStThreads, sizeof(StSmem), s>>>(a, o);
    return cudaGetLastError();
}

}  // namespace sj

using namespace sj;

// The join on a 1D grid through the stripe kernel (two passes); returns
// STRIPES_UNSUITED when the grid is not 1D or a stripe exceeds shared memory
// (the caller then runs the general path).
int sj::join_stripes(sj_ctx *ctx, Workspace &w, const float4 *R, long long nR, const float4 *S, long long nS,
                     const GridDev &gd, const sj_opts *o, OutSpec &os, int64_t *npairs) {
    if (!ctx->use_stripes || !(gd.nx == 1 || gd.ny == 1) || (long long)gd.nx * gd.ny > kMaxBlocks)
        return STRIPES_UNSUITED;
    BPlan p;
    p.G = 1;
    p.bx = gd.nx;
    p.by = gd.ny;
    p.nb = gd.nx * gd.ny;
    p.nc = ctx->num_sms * l1_blocks_per_sm(p.nb);
    const int vert = gd.ny == 1 ? 1 : 0;
    w.bcap_r = std::max<unsigned long long>(w.bcap_r, (unsigned long long)nR + nR / 8 + 1024);
    w.bcap_s = std::max<unsigned long long>(w.bcap_s, (unsigned long long)nS + nS / 8 + 1024);
    cudaStream_t s = ctx->stream;
    for (int attempt = 0; attempt < 3; attempt++) {
        int st;
        if ((st = size_blocked(ctx, w, p))) return st;
        // the stripes' sorted orders: keys, then merged indexes, one slot per L1 entry
        const unsigned long long scap = w.bcap_r + w.bcap_s;
        if ((st = ensure(ctx, w.st_order, 6ull * scap + 16))) return st;
        unsigned *skey = (unsigned *)w.st_order.p;
        unsigned short *sval = (unsigned short *)(skey + scap);
        BArgs a = blocked_args(w, p, R, nR, S, nS, gd);
        if (ctx->shared_cursors) a.cur = (unsigned *)w.bCur.p;
        a.fine_cap = kStCap;   // a stripe beyond the stripe kernel's capacity needs the general path
        if ((st = enqueue_blocked_partition(ctx, w, p, a))) return st;
        cudaError_t e;
        {
            PhaseScope ph(ctx, PH_SWEEP_COUNT, 1);
            if ((e = launch_stripe_join(MODE_COUNT, a, vert, skey, sval, scap, bjoin_out(w, 0), ctx->num_sms, s)))
                return cuda_fail(ctx, e, "stripe join kernel");
        }
        {
            PhaseScope ph(ctx, PH_PAIRSCAN, 1);
            if ((e = launch_scan_pairs((const unsigned *)w.bPc.p, (unsigned)p.nb, (unsigned long long *)w.bPoff.p,
                                       a.st, s)))
                return cuda_fail(ctx, e, "pair-count scan");
        }
        Stats stats;
        if ((st = read_stats(ctx, w, &stats))) return st;
        if (stats.err & kErrBadRect)
            return fail(ctx, SJ_EINVAL, "invalid rectangle: NaN/Inf coordinate or xl > xu / yl > yu");
        if (stats.err & kErrEntCap) {
            w.bcap_r = std::max<unsigned long long>(w.bcap_r, stats.e_r + stats.e_r / 8 + 1024);
            w.bcap_s = std::max<unsigned long long>(w.bcap_s, stats.e_s + stats.e_s / 8 + 1024);
            continue;
        }
        if (stats.err) return fail(ctx, SJ_EINTERNAL, "device error bits 0x%x", stats.err);
        if (stats.need_direct) return STRIPES_UNSUITED;
        const unsigned long long P = stats.npairs;
        *npairs = (int64_t)P;
        memset(&ctx->last, 0, sizeof ctx->last);
        ctx->last.path = 2;
        ctx->last.block_side = 1;
        ctx->last.blocks = p.nb;
        ctx->last.work_items = stats.nchunks;
        ctx->last.l1_entries_r = (int64_t)stats.e_r;
        ctx->last.l1_entries_s = (int64_t)stats.e_s;
        ctx->last.npairs = (int64_t)P;
        if ((st = out_acquire(ctx, w, os, P))) return st;
        if (P == 0) return SJ_OK;
        BJoinOut wo = bjoin_out(w, 1);
        wo.out = os.got;
        wo.cap = P;
        {
            PhaseScope ph(ctx, PH_SWEEP_WRITE, 1);
            if ((e = launch_stripe_join(MODE_WRITE, a, vert, skey, sval, scap, wo, ctx->num_sms, s))) {
                out_abandon(ctx, os);
                return cuda_fail(ctx, e, "stripe join kernel");
            }
        }
        if (o && o->sort_output && (st = sort_pairs(ctx, w, os.got, P))) {
            out_abandon(ctx, os);
            return st;
        }
        return SJ_OK;
    }
    return fail(ctx, SJ_EINTERNAL, "stripe workspace did not converge");
}
