// Cohen's probabilistic output-size estimator (Section V, "Probabilistic
// memory requirement estimation"): the product A A is a three-layer graph
// (rows i of A -> columns k of A = rows of the right factor -> columns j);
// every first-layer vertex gets r keys drawn from Exp(1), each layer keeps
// the minimum key over its in-neighbours, and nnz((AA)_*j) is estimated by
// (r - 1) / sum_l (minimum key l reaching j).  Each layer costs O(r nnz(A)).
//
// Random numbers: the keys come from splitmix64 (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", 2014) evaluated at the
// counter seed + (i * r + l) * golden; the top 53 bits give u in (0, 1] and
// the key is -ln(u), evaluated in FP32.
#include <cuda_runtime.h>

#include <cstdint>

#include "mcl.h"
#include "mcl_device.cuh"
#include "mcl_internal.h"

namespace mcl {

constexpr int COHEN_MAX_R = 16;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// key l of first-layer vertex i: -ln(u), u = (t + 1) / 2^53 with t the top 53
// bits of the hash, u in (0, 1].  FP32 keeps full relative precision on both
// halves: ln(u) from u itself when u <= 1/2, ln1p(-(1 - u)) from the exact
// complement 1 - u = (2^53 - 1 - t) / 2^53 otherwise (small keys, which are
// the minima of large reach sets, would otherwise lose their digits).
__device__ __forceinline__ float cohen_key(uint64_t seed, int64_t i, int l, int r) {
    const uint64_t z = splitmix64(seed + (uint64_t)(i * r + l) * 0x9E3779B97F4A7C15ull);
    const uint64_t t = z >> 11;
    if (t < (1ull << 52)) return -logf((float)(t + 1ull) * 0x1p-53f);
    const uint64_t w = (1ull << 53) - 1ull - t;
    return -log1pf(-((float)w * 0x1p-53f));
}

// layer 2: m[k][l] = min over i in inds(A_*k) of key(i, l); +inf if empty
__global__ void k_cohen_layer2(CscView A, int r, uint64_t seed, float* m) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = gw; k < A.n; k += nw) {
        float mn[COHEN_MAX_R];
#pragma unroll
        for (int l = 0; l < COHEN_MAX_R; ++l) mn[l] = INFINITY;
        for (int64_t p = A.colptr[k] + lane; p < A.colptr[k + 1]; p += 32) {
            const int i = A.rowidx[p];
#pragma unroll
            for (int l = 0; l < COHEN_MAX_R; ++l)
                if (l < r) mn[l] = fminf(mn[l], cohen_key(seed, i, l, r));
        }
#pragma unroll
        for (int l = 0; l < COHEN_MAX_R; ++l) {
            if (l < r) {
                const float v = warp_min(mn[l]);
                if (lane == 0) m[k * r + l] = v;
            }
        }
    }
}

// layer 3 and the estimate: est_j = (r - 1) / sum_l min over k in inds(A_*j) of m[k][l]
__global__ void k_cohen_layer3(CscView A, int r, const float* m, float* est) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < A.n; j += nw) {
        float mn[COHEN_MAX_R];
#pragma unroll
        for (int l = 0; l < COHEN_MAX_R; ++l) mn[l] = INFINITY;
        for (int64_t p = A.colptr[j] + lane; p < A.colptr[j + 1]; p += 32) {
            const int k = A.rowidx[p];
#pragma unroll
            for (int l = 0; l < COHEN_MAX_R; ++l)
                if (l < r) mn[l] = fminf(mn[l], m[(int64_t)k * r + l]);
        }
        float sum = 0.0f;
#pragma unroll
        for (int l = 0; l < COHEN_MAX_R; ++l)
            if (l < r) sum += warp_min(mn[l]);
        if (lane == 0) est[j] = (sum < INFINITY && sum > 0.0f) ? (float)(r - 1) / sum : 0.0f;
    }
}

// size estimate for the numeric pass: ceil(est * safety) clamped to [1, min(flops, span)]
__global__ void k_cohen_to_est(int32_t n, const float* e, float safety, const int64_t* flops,
                               const int32_t* rlo, const int32_t* rhi, int64_t* est) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int64_t hi = flops[j];
    const int64_t span = (int64_t)rhi[j] - rlo[j] + 1;
    if (span < hi) hi = span;
    if (hi < 1) hi = 1;
    const double v = ceil((double)e[j] * (double)safety);
    est[j] = v < 1.0 ? 1 : (v > (double)hi ? hi : (int64_t)v);
}

int cohen_max_r() { return COHEN_MAX_R; }

void launch_cohen(const CscView& A, int r, uint64_t seed, float* m, float* est, cudaStream_t s) {
    if (A.n == 0) return;
    int64_t blocks = ((int64_t)A.n * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_cohen_layer2<<<(unsigned)blocks, 256, 0, s>>>(A, r, seed, m);
    count_launches(1);
    k_cohen_layer3<<<(unsigned)blocks, 256, 0, s>>>(A, r, m, est);
    count_launches(1);
}

void launch_cohen_to_est(int32_t n, const float* e, float safety, const ExpandBuffers& b,
                         cudaStream_t s) {
    if (n == 0) return;
    k_cohen_to_est<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, e, safety, b.flops, b.rlo,
                                                                b.rhi, b.est);
    count_launches(1);
}

}  // namespace mcl
