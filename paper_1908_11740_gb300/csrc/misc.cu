// misc.cu -- small helper kernels of the host runtime.
#include "sj_internal.h"

namespace sj {

// cnt_r[t], cnt_s[t] = replicated entries of tile t (differences of the
// exclusive prefix sums written by the partitioning scan).
__global__ void k_tile_counts(const uint2 *__restrict__ off, long long T, unsigned *__restrict__ cr,
                              unsigned *__restrict__ cs) {
    for (long long t = blockIdx.x * 256ll + threadIdx.x; t < T; t += 256ll * gridDim.x) {
        const uint2 a = off[t], b = off[t + 1];
        if (cr) cr[t] = b.x - a.x;
        if (cs) cs[t] = b.y - a.y;
    }
}

cudaError_t launch_tile_counts(const uint2 *off, long long T, unsigned *cnt_r, unsigned *cnt_s,
                               cudaStream_t s) {
    long long nb = (T + 255) / 256;
    if (nb > 65535) nb = 65535;
    k_tile_counts<<<(unsigned)nb, 256, 0, s>>>(off, T, cnt_r, cnt_s);
    return cudaGetLastError();
}

__global__ void k_zero_words(unsigned *__restrict__ p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

__global__ void k_copy_words(const unsigned *__restrict__ src, unsigned *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

static unsigned words_grid(size_t n) {
    const size_t g = (n + 255) / 256;
    return (unsigned)(g < 1024 ? (g ? g : 1) : 1024);
}

static_assert(sizeof(Stats) % 4 == 0 && sizeof(JoinDesc) % 4 == 0, "word-wise copies");

cudaError_t zero_words_async(void *p, size_t bytes, cudaStream_t s) {
    const size_t n = bytes / 4;
    if (!n) return cudaSuccess;
    k_zero_words<<<words_grid(n), 256, 0, s>>>((unsigned *)p, n);
    return cudaGetLastError();
}

cudaError_t copy_words_async(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    const size_t n = bytes / 4;
    if (!n) return cudaSuccess;
    k_copy_words<<<words_grid(n), 256, 0, s>>>((const unsigned *)src, (unsigned *)dst, n);
    return cudaGetLastError();
}

// Clear the per-call counters of a partition's stats, keep its totals.
__global__ void k_reset_counters(Stats *st) {
    if (threadIdx.x == 0) {
        st->npairs = 0;
        st->nfail = 0;
        st->nfail_large = 0;
        st->err = 0;
        st->check = 0;
    }
    if (threadIdx.x < 8) st->work[threadIdx.x] = 0;
}

cudaError_t launch_reset_counters(Stats *st, cudaStream_t s) {
    k_reset_counters<<<1, 32, 0, s>>>(st);
    return cudaGetLastError();
}

// Models belong to their creator (sj_mlp_free); the context only forgets its reference.
void mlp_release(sj_ctx *ctx) {
    ctx->model = nullptr;
    ctx->mlp_loaded = false;
}

}  // namespace sj
