// learned.cu -- the learned result-count predictor of the one-pass join.
//
// Unit: a block of the two-level partition (G x G tiles; the unit of work
// and of output reservation of the join).  Features of a block follow the
// histograms of Sec. 3.3 (Eq. 2): for each side (R, S) and axis (x, y), k = 8
// buckets over the block's extent, bucket i counting the rectangles whose
// projection overlaps it; as in the paper, only a sample (one rectangle of
// every kPhi of each side) feeds the histograms, and each histogram is then
// scaled to the block's exact entry count.  The 32 inputs are log1p of those
// scaled counts.  Buckets are ranges of tile columns (rows), so the features
// depend only on integer tile indices.
//
// Model: 32 -> 64 (ReLU) -> 64 (ReLU) -> 1, weights stored as bf16, every
// product accumulated in fp32; output = predicted log1p(pairs of the block).
// Training (forward, backward, Adam) runs in the kernels below.
#include <cuda_bf16.h>

#include "sj_learned.h"

namespace sj {

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// feat[it][32] of every work item (block with both sides), scaled to the
// exact entry counts btot.  A block side without a sample gets its entries
// spread evenly over the 8 buckets.  One warp per item, lane q = feature q
// (side q / 16), so reads and writes are coalesced.
__global__ void k_features(const unsigned *__restrict__ raw, const unsigned *__restrict__ items,
                           const unsigned *__restrict__ btot, int nb, const Stats *__restrict__ st,
                           float *__restrict__ feat) {
    const unsigned n = st->nchunks;
    const unsigned q = threadIdx.x & 31, side = q >> 4;
    const unsigned nwarps = gridDim.x * (blockDim.x >> 5);
    for (unsigned it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n; it += nwarps) {
        const unsigned b = items[it];
        const unsigned *r = raw + (size_t)b * kRawPerBlock;
        const float nt = (float)btot[side * nb + b];
        const unsigned samp = r[32 + side];
        const float h = samp ? (float)r[q] * nt / (float)samp : nt * 0.125f;
        feat[(size_t)it * kFeat + q] = log1pf(h);
    }
}

// ---------------------------------------------------------------------------
// MLP forward (inference): one warp per sample, bf16 weights in shared memory
// ---------------------------------------------------------------------------
// Weights are kept input-major (w1t[k][j] = W1[j][k], w2t[k][j] = W2[j][k]):
// in the forward pass the 32 lanes of a warp compute 32 consecutive units j
// and read 32 consecutive values; the backward pass (lane = k) walks j from
// a lane-dependent start, so the lanes again fall in different banks.
struct __align__(16) MlpSmem {
    __nv_bfloat16 w1t[kFeat * kH1];
    __nv_bfloat16 w2t[kH1 * kH2];
    __nv_bfloat16 w3[kH2];
    float b1[kH1], b2[kH2], b3;
};

__device__ __forceinline__ void mlp_load(MlpSmem &m, const MlpWeights &w) {
    // the published weights are input-major already: straight 16-byte copies
    {
        const uint4 *s1 = reinterpret_cast<const uint4 *>(w.w1), *s2 = reinterpret_cast<const uint4 *>(w.w2);
        uint4 *d1 = reinterpret_cast<uint4 *>(m.w1t), *d2 = reinterpret_cast<uint4 *>(m.w2t);
        for (int k = threadIdx.x; k < kH1 * kFeat / 8; k += blockDim.x) d1[k] = s1[k];
        for (int k = threadIdx.x; k < kH2 * kH1 / 8; k += blockDim.x) d2[k] = s2[k];
    }
    for (int k = threadIdx.x; k < kH2; k += blockDim.x) {
        m.w3[k] = w.w3[k];
        m.b2[k] = w.b2[k];
    }
    for (int k = threadIdx.x; k < kH1; k += blockDim.x) m.b1[k] = w.b1[k];
    if (threadIdx.x == 0) m.b3 = w.b3[0];
    __syncthreads();
}

// lane computes hidden units lane and lane + 32 of both layers; x and h1
// live in shared memory per warp.  Returns the output on every lane; when
// act is given, stores z1, z2 (pre-activations) for the backward pass.
__device__ __forceinline__ float mlp_warp_forward(const MlpSmem &m, const float *x, float *h1s, float *z1o,
                                                  float *z2o) {
    const int lane = threadIdx.x & 31;
    float z1[2], z2[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int j = lane + 32 * u;
        float acc = m.b1[j];
#pragma unroll 8
        for (int k = 0; k < kFeat; k++) acc = fmaf(__bfloat162float(m.w1t[k * kH1 + j]), x[k], acc);
        z1[u] = acc;
        h1s[j] = fmaxf(acc, 0.0f);
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int j = lane + 32 * u;
        float acc = m.b2[j];
#pragma unroll 8
        for (int k = 0; k < kH1; k++) acc = fmaf(__bfloat162float(m.w2t[k * kH2 + j]), h1s[k], acc);
        z2[u] = acc;
    }
    float part = 0.0f;
#pragma unroll
    for (int u = 0; u < 2; u++) part = fmaf(__bfloat162float(m.w3[lane + 32 * u]), fmaxf(z2[u], 0.0f), part);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    if (z1o) {
        z1o[lane] = z1[0];
        z1o[lane + 32] = z1[1];
        z2o[lane] = z2[0];
        z2o[lane + 32] = z2[1];
    }
    __syncwarp();
    return part + m.b3;
}

constexpr int kMlpThreads = 256;
constexpr int kMlpWarps = kMlpThreads / 32;

// y[i] = f(X[i]) for i < n (n read from *n_dev when given).  One thread per
// sample; every warp reads the same weights at the same time (shared-memory
// broadcasts, 8 bf16 weights per 16-byte load; a bf16 is the high half of
// the float with the same bits).  The sums run in the order of mlp_warp_forward (k ascending
// from the bias; the output's partials per lane l = w3[l] h2[l] + w3[l+32]
// h2[l+32], then halved pairwise like the butterfly), so inference and the
// training forward give the same bits.
constexpr int kMlpInfThreads = 64;
__global__ void __launch_bounds__(kMlpInfThreads) k_mlp_forward(MlpWeights w, const float *__restrict__ X,
                                                                long long n, const unsigned *n_dev,
                                                                float *__restrict__ y) {
    __shared__ __align__(16) MlpSmem m;
    // this thread's input and hidden layer (rows padded: no bank conflicts)
    __shared__ float xs[kMlpInfThreads][kFeat + 1];
    __shared__ float h1s[kMlpInfThreads][kH1 + 1];
    mlp_load(m, w);
    const long long nn = n_dev ? (long long)*n_dev : n;
    float *x = xs[threadIdx.x];
    float *h1 = h1s[threadIdx.x];
    for (long long i = (long long)blockIdx.x * kMlpInfThreads + threadIdx.x; i < nn;
         i += (long long)gridDim.x * kMlpInfThreads) {
        const float4 *xv = reinterpret_cast<const float4 *>(X + i * kFeat);
#pragma unroll
        for (int q = 0; q < kFeat / 4; q++) {
            const float4 t = xv[q];
            x[4 * q] = t.x;
            x[4 * q + 1] = t.y;
            x[4 * q + 2] = t.z;
            x[4 * q + 3] = t.w;
        }
        {
            float acc[kH1];
#pragma unroll
            for (int j = 0; j < kH1; j++) acc[j] = m.b1[j];
#pragma unroll 2
            for (int k = 0; k < kFeat; k++) {
                const float xk = x[k];
                const uint4 *row = reinterpret_cast<const uint4 *>(m.w1t + k * kH1);   // 8 weights per load
#pragma unroll
                for (int q = 0; q < kH1 / 8; q++) {
                    const uint4 u = row[q];
                    const unsigned wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const int j = 8 * q + 2 * t;
                        acc[j] = fmaf(__uint_as_float(wd[t] << 16), xk, acc[j]);
                        acc[j + 1] = fmaf(__uint_as_float(wd[t] & 0xffff0000u), xk, acc[j + 1]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kH1; j++) h1[j] = fmaxf(acc[j], 0.0f);
        }
        float part[32];
#pragma unroll
        for (int c = 0; c < kH2 / 16; c++) {
            float acc[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) acc[jj] = m.b2[c * 16 + jj];
#pragma unroll 4
            for (int k = 0; k < kH1; k++) {
                const float hk = h1[k];
                const uint4 *row = reinterpret_cast<const uint4 *>(m.w2t + k * kH2 + c * 16);
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const uint4 u = row[q];
                    const unsigned wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const int jj = 8 * q + 2 * t;
                        acc[jj] = fmaf(__uint_as_float(wd[t] << 16), hk, acc[jj]);
                        acc[jj + 1] = fmaf(__uint_as_float(wd[t] & 0xffff0000u), hk, acc[jj + 1]);
                    }
                }
            }
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int j = c * 16 + jj;
                const float t = fmaxf(acc[jj], 0.0f);
                if (j < 32) part[j] = fmaf(__bfloat162float(m.w3[j]), t, 0.0f);
                else part[j - 32] = fmaf(__bfloat162float(m.w3[j]), t, part[j - 32]);
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
#pragma unroll
            for (int l = 0; l < d; l++) part[l] += part[l + d];
        y[i] = part[0] + m.b3;
    }
}

// ---------------------------------------------------------------------------
// training: forward + backward of the mean squared error, gradients summed
// per CTA in shared memory, then added to the global gradient buffer.
// Parameter layout (fp32, kParams): W1[64x32], b1[64], W2[64x64], b2[64],
// W3[64], b3[1].  The forward uses the bf16 weights (what inference uses);
// gradients are with respect to those values.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMlpThreads) k_mlp_grad(MlpWeights w, const float *__restrict__ X,
                                                          const float *__restrict__ Y, long long n,
                                                          float *__restrict__ grad, float *__restrict__ loss) {
    __shared__ MlpSmem m;
    __shared__ float g[kParams];
    __shared__ float xs[kMlpWarps][kFeat];
    __shared__ float hs[kMlpWarps][kH1];
    __shared__ float z1s[kMlpWarps][kH1];
    __shared__ float z2s[kMlpWarps][kH2];
    __shared__ float d2s[kMlpWarps][kH2];
    __shared__ float s_loss;
    mlp_load(m, w);
    for (int k = threadIdx.x; k < kParams; k += blockDim.x) g[k] = 0.0f;
    if (threadIdx.x == 0) s_loss = 0.0f;
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float inv_n = 1.0f / (float)(n > 0 ? n : 1);
    for (long long i = (long long)blockIdx.x * kMlpWarps + wid; i < n; i += (long long)gridDim.x * kMlpWarps) {
        xs[wid][lane] = X[i * kFeat + lane];
        __syncwarp();
        const float out = mlp_warp_forward(m, xs[wid], hs[wid], z1s[wid], z2s[wid]);
        const float err = out - Y[i];
        if (lane == 0) atomicAdd(&s_loss, err * err * inv_n);
        const float dout = 2.0f * err * inv_n;          // d loss / d out
        // layer 3
        float d2[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int j = lane + 32 * u;
            const float z = z2s[wid][j];
            atomicAdd(&g[kOffW3 + j], dout * fmaxf(z, 0.0f));
            d2[u] = z > 0.0f ? dout * __bfloat162float(m.w3[j]) : 0.0f;   // d loss / d z2_j
            d2s[wid][j] = d2[u];
        }
        if (lane == 0) atomicAdd(&g[kOffB3], dout);
        __syncwarp();
        // layer 2: dW2[j][k] = d2_j * h1_k ; d h1_k = sum_j d2_j W2[j][k]
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int j = lane + 32 * u;
            atomicAdd(&g[kOffB2 + j], d2[u]);
            if (d2[u] != 0.0f)
                for (int kk = 0; kk < kH1; kk++) {   // rotated so the 32 lanes hit 32 banks
                    const int k = (kk + lane) & (kH1 - 1);
                    atomicAdd(&g[kOffW2 + j * kH1 + k], d2[u] * hs[wid][k]);
                }
        }
        float d1[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int k = lane + 32 * u;
            float acc = 0.0f;
            for (int jj = 0; jj < kH2; jj++) {
                const int j = (jj + lane) & (kH2 - 1);
                acc = fmaf(d2s[wid][j], __bfloat162float(m.w2t[k * kH2 + j]), acc);
            }
            d1[u] = z1s[wid][k] > 0.0f ? acc : 0.0f;          // d loss / d z1_k
        }
        // layer 1
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int j = lane + 32 * u;
            atomicAdd(&g[kOffB1 + j], d1[u]);
            if (d1[u] != 0.0f)
                for (int kk = 0; kk < kFeat; kk++) {
                    const int k = (kk + lane) & (kFeat - 1);
                    atomicAdd(&g[kOffW1 + j * kFeat + k], d1[u] * xs[wid][k]);
                }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kParams; k += blockDim.x)
        if (g[k] != 0.0f) atomicAdd(grad + k, g[k]);
    if (threadIdx.x == 0) atomicAdd(loss, s_loss);
}

// Adam step on the fp32 master parameters, then the bf16 copies.
__global__ void k_adam(MlpParams p, const float *__restrict__ grad, float lr, float b1, float b2, float eps,
                       int step) {
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kParams; k += gridDim.x * blockDim.x) {
        const float gk = grad[k];
        const float mk = b1 * p.m[k] + (1.0f - b1) * gk;
        const float vk = b2 * p.v[k] + (1.0f - b2) * gk * gk;
        p.m[k] = mk;
        p.v[k] = vk;
        p.master[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// bf16 weights and fp32 biases of the inference copy from the fp32 master.
__global__ void k_mlp_publish(MlpParams p, MlpWeights w) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kParams; k += gridDim.x * blockDim.x) {
        const float v = p.master[k];
        // W1[j][k] (master, row-major) -> w1[k][j] (input-major), W2 alike
        if (k < kOffB1) w.w1[((k - kOffW1) % kFeat) * kH1 + (k - kOffW1) / kFeat] = __float2bfloat16_rn(v);
        else if (k < kOffW2) w.b1[k - kOffB1] = v;
        else if (k < kOffB2) w.w2[((k - kOffW2) % kH1) * kH2 + (k - kOffW2) / kH1] = __float2bfloat16_rn(v);
        else if (k < kOffW3) w.b2[k - kOffB2] = v;
        else if (k < kOffB3) w.w3[k - kOffW3] = __float2bfloat16_rn(v);
        else w.b3[0] = v;
    }
}

// ---------------------------------------------------------------------------
// one-pass plan: capacity of every work item from the predicted log1p(pairs),
// the total, and a heaviest-first order of the items (LPT).
// ---------------------------------------------------------------------------
// The non-learned estimate from the same histograms (Eq. 2): I_x = sum_i
// H_R^x[i] H_S^x[i] estimates the pairs that share an x bucket, I_y alike;
// assuming x and y independent, pairs ~ I_x I_y / (n_R n_S).
__global__ void k_heur_pred(const float *__restrict__ feat, const unsigned *__restrict__ items,
                            const unsigned *__restrict__ btot, int nb, const Stats *__restrict__ st,
                            float *__restrict__ pred) {
    const unsigned n = st->nchunks;
    for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
        const float *f = feat + (size_t)it * kFeat;
        float ix = 0.0f, iy = 0.0f;
        for (int q = 0; q < 8; q++) {
            ix = fmaf(expm1f(f[q]), expm1f(f[16 + q]), ix);
            iy = fmaf(expm1f(f[8 + q]), expm1f(f[24 + q]), iy);
        }
        const unsigned b = items[it];
        const float nn = (float)btot[b] * (float)btot[nb + b];
        // log1p(ix * iy / nn) computed as log(ix) + log(iy) - log(nn) to stay in range
        pred[it] = nn > 0.0f && ix > 0.0f && iy > 0.0f ? log1pf(expf(logf(ix) + logf(iy) - logf(nn))) : 0.0f;
    }
}

// cap[it] = ceil(expm1(pred) * (1 + margin)) + slack (at least 0), summed
// into the total; order = items sorted by predicted cost (L1 entries +
// predicted pairs) into 32 log2 classes, heaviest first.  Two launches over
// all items: class histogram and total, then the slots.  scratch (zeroed by
// the launcher) holds hist[32], cursor[32].
__device__ __forceinline__ int cost_class(float cost) {
    return cost >= 1.0f ? min(31, (int)log2f(cost)) : 0;
}

__device__ __forceinline__ int plan_class(const float *__restrict__ pred, const uint4 *__restrict__ imeta,
                                          const unsigned *__restrict__ ins, unsigned it, float &e) {
    e = expm1f(fminf(fmaxf(pred[it], 0.0f), 21.0f));   // at most ~1.3e9 pairs a block
    return 31 - cost_class((float)imeta[it].z + (float)ins[it] + e);
}

__global__ void __launch_bounds__(256) k_plan_count(const float *__restrict__ pred, const uint4 *__restrict__ imeta,
                                                    const unsigned *__restrict__ ins, const Stats *__restrict__ st,
                                                    float margin, unsigned slack, unsigned long long *cap_total,
                                                    unsigned *__restrict__ scratch) {
    __shared__ unsigned hist[32];
    __shared__ unsigned long long s_tot;
    const unsigned n = st->nchunks;
    if (threadIdx.x < 32) hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    const unsigned lanelt = (1u << (threadIdx.x & 31)) - 1u;
    unsigned long long my = 0;
    for (unsigned b = blockIdx.x * 256; b < n; b += 256 * gridDim.x) {   // whole warps per step
        const unsigned it = b + threadIdx.x;
        int c = -1;
        if (it < n) {
            float e;
            c = plan_class(pred, imeta, ins, it, e);
            my += (unsigned long long)ceilf(e * (1.0f + margin)) + slack;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && (peers & lanelt) == 0) atomicAdd(&hist[c], (unsigned)__popc(peers));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) my += __shfl_xor_sync(0xffffffffu, my, d);
    if ((threadIdx.x & 31) == 0 && my) atomicAdd(&s_tot, my);
    __syncthreads();
    if (threadIdx.x < 32 && hist[threadIdx.x]) atomicAdd(scratch + threadIdx.x, hist[threadIdx.x]);
    if (threadIdx.x == 0 && s_tot) atomicAdd(cap_total, s_tot);
}

__global__ void __launch_bounds__(256) k_plan_order(const float *__restrict__ pred, const uint4 *__restrict__ imeta,
                                                    const unsigned *__restrict__ ins, const Stats *__restrict__ st,
                                                    unsigned *__restrict__ scratch, unsigned *__restrict__ order) {
    __shared__ unsigned base[32];
    const unsigned n = st->nchunks;
    if (threadIdx.x < 32) {   // exclusive scan of the class histogram
        const unsigned h = scratch[threadIdx.x];
        unsigned inc = h;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
            if ((int)threadIdx.x >= d) inc += o;
        }
        base[threadIdx.x] = inc - h;
    }
    __syncthreads();
    const unsigned lanelt = (1u << (threadIdx.x & 31)) - 1u;
    unsigned *cursor = scratch + 32;
    for (unsigned b = blockIdx.x * 256; b < n; b += 256 * gridDim.x) {
        const unsigned it = b + threadIdx.x;
        int c = -1;
        if (it < n) {
            float e;
            c = plan_class(pred, imeta, ins, it, e);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(peers) - 1;
        unsigned pos = 0;
        if (c >= 0 && (int)(threadIdx.x & 31) == leader) pos = atomicAdd(cursor + c, (unsigned)__popc(peers));
        pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & lanelt);
        if (c >= 0) order[base[c] + pos] = it;
    }
}

// label[it] = log1p(pairs of work item it) from the count pass.
__global__ void k_labels(const unsigned *__restrict__ cnt, const Stats *__restrict__ st, float *__restrict__ label) {
    const unsigned n = st->nchunks;
    for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x)
        label[it] = log1pf((float)cnt[it]);
}

// Labels of the work items from per-tile pair counts (for blocks whose tiles
// exceed shared memory, counted by the single-level path): item_of[b] =
// work item of block b (all ones: none), then every tile's pairs are added to
// its block's item, then log1p.  cnt64 must start at zero.
__global__ void k_item_of_block(const unsigned *__restrict__ items, unsigned n, unsigned *__restrict__ item_of) {
    for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x)
        item_of[items[it]] = it;
}

__global__ void k_tile_pairs_to_items(const unsigned *__restrict__ tile_pairs, int nx, long long T, int G, int bx,
                                      const unsigned *__restrict__ item_of,
                                      unsigned long long *__restrict__ cnt64) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x) {
        const unsigned p = tile_pairs[t];
        if (!p) continue;
        const int row = (int)(t / nx), col = (int)(t % nx);
        const unsigned it = item_of[(row / G) * bx + col / G];
        if (it != 0xffffffffu) atomicAdd(cnt64 + it, (unsigned long long)p);
    }
}

__global__ void k_labels64(const unsigned long long *__restrict__ cnt64, unsigned n, float *__restrict__ label) {
    for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x)
        label[it] = log1pf((float)cnt64[it]);
}

// ---- launchers -------------------------------------------------------------
cudaError_t launch_labels_from_tiles(const unsigned *items, unsigned n, unsigned *item_of, const unsigned *tile_pairs,
                                     int nx, long long T, int G, int bx, unsigned long long *cnt64, float *label,
                                     int grid, cudaStream_t s) {
    k_item_of_block<<<grid, 256, 0, s>>>(items, n, item_of);
    k_tile_pairs_to_items<<<grid, 256, 0, s>>>(tile_pairs, nx, T, G, bx, item_of, cnt64);
    k_labels64<<<grid, 256, 0, s>>>(cnt64, n, label);
    return cudaGetLastError();
}

cudaError_t launch_labels(const unsigned *cnt, const Stats *st, float *label, int grid, cudaStream_t s) {
    k_labels<<<grid, 256, 0, s>>>(cnt, st, label);
    return cudaGetLastError();
}

cudaError_t launch_features(const unsigned *raw, const unsigned *items, const unsigned *btot, int nb,
                            const Stats *st, float *feat, int grid, cudaStream_t s) {
    k_features<<<grid, 256, 0, s>>>(raw, items, btot, nb, st, feat);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const MlpWeights &w, const float *X, long long n, const unsigned *n_dev, float *y,
                               int grid, cudaStream_t s) {
    k_mlp_forward<<<grid, kMlpInfThreads, 0, s>>>(w, X, n, n_dev, y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const MlpWeights &w, const float *X, const float *Y, long long n, float *grad,
                            float *loss, int grid, cudaStream_t s) {
    k_mlp_grad<<<grid, kMlpThreads, 0, s>>>(w, X, Y, n, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(const MlpParams &p, const float *grad, float lr, float b1, float b2, float eps, int step,
                        cudaStream_t s) {
    k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(p, grad, lr, b1, b2, eps, step);
    return cudaGetLastError();
}

cudaError_t launch_mlp_publish(const MlpParams &p, const MlpWeights &w, cudaStream_t s) {
    k_mlp_publish<<<(kParams + 255) / 256, 256, 0, s>>>(p, w);
    return cudaGetLastError();
}

cudaError_t launch_heur_pred(const float *feat, const unsigned *items, const unsigned *btot, int nb,
                             const Stats *st, float *pred, int grid, cudaStream_t s) {
    k_heur_pred<<<grid, 256, 0, s>>>(feat, items, btot, nb, st, pred);
    return cudaGetLastError();
}

// cap_total points to kPlanScratch bytes, zeroed by the caller: the total,
// then the class histogram and cursors.  grid: CTAs of 256 over the items.
cudaError_t launch_plan(const float *pred, const uint4 *imeta, const unsigned *ins, const Stats *st, float margin,
                        unsigned slack, unsigned long long *cap_total, unsigned *order, int grid, cudaStream_t s) {
    unsigned *scratch = reinterpret_cast<unsigned *>(cap_total + 1);
    k_plan_count<<<grid, 256, 0, s>>>(pred, imeta, ins, st, margin, slack, cap_total, scratch);
    k_plan_order<<<grid, 256, 0, s>>>(pred, imeta, ins, st, scratch, order);
    return cudaGetLastError();
}

}  // namespace sj
