// Connected components of the final matrix's undirected pattern
// (Algorithm 1, "return the connected components of A").
//
// Lock-free union-find: every stored entry (i, j) hooks the larger of the
// two roots under the smaller with atomicCAS, so every root is the
// smallest vertex of its set and the final label of a vertex is the
// smallest vertex id of its component.  Retry loops make global progress
// (a failed CAS means another thread linked a root), and every loop is
// bounded; exhausting a bound raises ERR_TIMEOUT instead of spinning.
#include <cstdint>

#include "mcl_device.cuh"
#include "mcl_internal.h"

namespace mcl {

constexpr int CC_FIND_LIMIT = 1 << 22;
constexpr int CC_LINK_LIMIT = 1 << 20;

__device__ __forceinline__ int cc_find(int* parent, int x, DevCounters* ctr) {
    for (int it = 0; it < CC_FIND_LIMIT; ++it) {
        const int p = *reinterpret_cast<volatile int*>(parent + x);
        if (p == x) return x;
        const int gp = *reinterpret_cast<volatile int*>(parent + p);
        if (gp != p) atomicCAS(parent + x, p, gp);  // path halving, benign if it loses
        x = gp;
    }
    atomicOr(&ctr->err, ERR_TIMEOUT);
    return x;
}

__global__ void k_cc_init(int32_t n, int* parent) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) parent[v] = (int)v;
}

// warp per column: link every stored (row, column) pair
__global__ void k_cc_hook(CscView A, int* parent, DevCounters* ctr) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < A.n; j += nw) {
        const int64_t cb = A.colptr[j], ce = A.colptr[j + 1];
        for (int64_t p = cb + lane; p < ce; p += 32) {
            int a = (int)j, b = A.rowidx[p];
            if (a == b) continue;
            int it = 0;
            for (; it < CC_LINK_LIMIT; ++it) {
                a = cc_find(parent, a, ctr);
                b = cc_find(parent, b, ctr);
                if (a == b) break;
                if (a < b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                // a > b: hang root a under root b
                if (atomicCAS(parent + a, a, b) == a) break;
            }
            if (it == CC_LINK_LIMIT) atomicOr(&ctr->err, ERR_TIMEOUT);
        }
    }
}

__global__ void k_cc_label(int32_t n, int* parent, int32_t* labels, DevCounters* ctr) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) labels[v] = cc_find(parent, (int)v, ctr);
}

void launch_components(const CscView& A, int32_t* labels, DevCounters* ctr, cudaStream_t s) {
    if (A.n == 0) return;
    // labels doubles as the parent array (int32, same length)
    int* parent = reinterpret_cast<int*>(labels);
    const unsigned nb = (unsigned)((A.n + 255) / 256);
    k_cc_init<<<nb, 256, 0, s>>>(A.n, parent);
    count_launches(1);
    int64_t blocks = ((int64_t)A.n * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_cc_hook<<<(unsigned)blocks, 256, 0, s>>>(A, parent, ctr);
    count_launches(1);
    k_cc_label<<<nb, 256, 0, s>>>(A.n, parent, labels, ctr);
    count_launches(1);
}

}  // namespace mcl
