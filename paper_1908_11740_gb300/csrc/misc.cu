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

// Clear the per-call counters of a partition's stats, keep its totals.
__global__ void k_reset_counters(Stats *st) {
    if (threadIdx.x == 0) {
        st->npairs = 0;
        st->nfail = 0;
        st->nfail_large = 0;
        st->err = 0;
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
