// sj_learned.h -- the per-block result-count predictor (features, MLP,
// training, one-pass plan).  Internal to the library.
#pragma once
#include <cuda_bf16.h>

#include "sj_common.cuh"

namespace sj {

constexpr int kFeat = 32;          // inputs: [R x | R y | S x | S y] x 8 buckets
constexpr int kBins = 8;           // buckets per histogram (Eq. 2 with k = 8)
constexpr int kPhi = 16;           // one rectangle of every kPhi feeds the histograms
constexpr int kRawPerBlock = 34;   // 32 bucket counts + sampled count per side
constexpr int kH1 = 64, kH2 = 64;  // hidden units
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH1 * kFeat;
constexpr int kOffW2 = kOffB1 + kH1;
constexpr int kOffB2 = kOffW2 + kH2 * kH1;
constexpr int kOffW3 = kOffB2 + kH2;
constexpr int kOffB3 = kOffW3 + kH2;
constexpr int kParams = kOffB3 + 1;   // 6337

struct MlpWeights {               // inference copy: bf16 weights (w1, w2 input-major), fp32 biases
    __nv_bfloat16 *w1, *w2, *w3;
    float *b1, *b2, *b3;
};

struct MlpParams {                // fp32 master parameters and Adam moments
    float *master, *m, *v;
};

// Buckets overlapped by local columns (rows) [l0, l1] of a block G tiles
// wide: column c spans [8c/G, 8(c+1)/G) in bucket units, so the range is
// floor(8 l0 / G) .. floor((8 (l1 + 1) - 1) / G).
__device__ __forceinline__ int bucket_lo(int l0, int G) { return l0 * kBins / G; }
__device__ __forceinline__ int bucket_hi(int l1, int G) { return ((l1 + 1) * kBins - 1) / G; }

// Called by the L1 count kernel for sampled rectangles: adds the rectangle's
// bucket ranges to every block it overlaps.  raw layout per block:
// [side][axis][bucket] (32 counts), then the sampled count of each side.
__device__ __forceinline__ void feat_add(unsigned *raw, int G, int bxn, int side, int cx0, int cx1, int cy0,
                                         int cy1, int bx0, int bx1, int by0, int by1) {
    for (int by = by0; by <= by1; by++)
        for (int bx = bx0; bx <= bx1; bx++) {
            unsigned *r = raw + (size_t)(by * bxn + bx) * kRawPerBlock;
            const int c0 = bx * G, r0 = by * G;
            const int lx0 = max(cx0 - c0, 0), lx1 = min(cx1 - c0, G - 1);
            const int ly0 = max(cy0 - r0, 0), ly1 = min(cy1 - r0, G - 1);
            const int ix0 = bucket_lo(lx0, G), ix1 = bucket_hi(lx1, G);
            const int iy0 = bucket_lo(ly0, G), iy1 = bucket_hi(ly1, G);
            unsigned *hx = r + side * 16, *hy = r + side * 16 + 8;
            for (int i = ix0; i <= ix1; i++) atomicAdd(hx + i, 1u);
            for (int i = iy0; i <= iy1; i++) atomicAdd(hy + i, 1u);
            atomicAdd(r + 32 + side, 1u);
        }
}

cudaError_t launch_features(const unsigned *raw, const unsigned *items, const unsigned *btot, int nb,
                            const Stats *st, float *feat, int grid, cudaStream_t s);
cudaError_t launch_mlp_forward(const MlpWeights &w, const float *X, long long n, const unsigned *n_dev, float *y,
                               int grid, cudaStream_t s);
cudaError_t launch_mlp_grad(const MlpWeights &w, const float *X, const float *Y, long long n, float *grad,
                            float *loss, int grid, cudaStream_t s);
cudaError_t launch_adam(const MlpParams &p, const float *grad, float lr, float b1, float b2, float eps, int step,
                        cudaStream_t s);
cudaError_t launch_mlp_publish(const MlpParams &p, const MlpWeights &w, cudaStream_t s);
cudaError_t launch_heur_pred(const float *feat, const unsigned *items, const unsigned *btot, int nb,
                             const Stats *st, float *pred, int grid, cudaStream_t s);
cudaError_t launch_labels(const unsigned *cnt, const Stats *st, float *label, int grid, cudaStream_t s);
cudaError_t launch_labels_from_tiles(const unsigned *items, unsigned n, unsigned *item_of, const unsigned *tile_pairs,
                                     int nx, long long T, int G, int bx, unsigned long long *cnt64, float *label,
                                     int grid, cudaStream_t s);
constexpr int kPlanScratch = 512;   // capacity total + class histogram + class cursors
cudaError_t launch_plan(const float *pred, const uint4 *imeta, const unsigned *ins, const Stats *st, float margin,
                        unsigned slack, unsigned long long *cap_total, unsigned *order, int grid, cudaStream_t s);

}  // namespace sj
