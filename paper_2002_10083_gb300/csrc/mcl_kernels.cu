// Kernels of one MCL iteration on sm_103a.
//
//   k_colstats      validation + per column flops_j (Section II notation),
//                   product row span and output capacity
//   k_scan_*        exclusive prefix sums (int64)
//   k_symbolic      exact nnz((AA)_*j): shared-memory bitmap over the row
//                   span, in windows (the symbolic SpGEMM of Sections II, V)
//   k_bin_*         columns -> accumulator configuration and size class
//   k_numeric       the fused hot op: c_ij = sum_k a_ik a_kj (Alg. 1,
//                   expansion) into a shared-memory hash or dense row-range
//                   accumulator, prune/select/recover (Alg. 1, Prune) by
//                   radix select, inflation + FP64 renormalisation and chaos
//   k_prune         the prune rule alone on a materialised matrix
//   k_inflate_normalize, k_chaos, k_compact, k_finalize
//
// Irregular, HBM/L2-bound work: no tensor cores, no TMA.  Reads of the
// gathered columns are coalesced 32-entry runs of (row, value).
#include <atomic>
#include <cfloat>
#include <climits>
#include <cstdint>
#include <mutex>

#include "mcl_device.cuh"
#include "mcl_internal.h"

namespace mcl {

static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// validation + column statistics
// ---------------------------------------------------------------------------

__device__ __forceinline__ void set_err(DevCounters* c, unsigned bit) { atomicOr(&c->err, bit); }

// Warp per column.  Checks colptr bounds, row range and strict order,
// values finite and >= 0; every read is guarded so malformed input only
// raises flags.  Then flops_j = sum_{k in col j} nnz(col k), the span
// [rlo_j, rhi_j] of product rows and cap_j = min(Krec, flops_j, span_j).
__global__ void k_colstats(CscView A, int32_t Krec, ExpandBuffers b) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    DevCounters* C = b.ctr;
    unsigned long long fl_acc = 0, fl_max = 0;
    int deg_max = 0, span_max = 0;
    if (gw == 0 && lane == 0) {
        if (A.colptr[0] != 0 || (b.nnz_is_bound ? A.colptr[A.n] > A.nnz : A.colptr[A.n] != A.nnz))
            set_err(C, ERR_COLPTR);
    }
    for (int64_t j = gw; j < A.n; j += nw) {
        const int64_t cb = A.colptr[j], ce = A.colptr[j + 1];
        const bool okc = cb >= 0 && ce >= cb && ce <= A.nnz;
        if (!okc) {
            if (lane == 0) {
                set_err(C, ERR_COLPTR);
                b.flops[j] = 0;
                b.rlo[j] = 0;
                b.rhi[j] = -1;
                b.cap[j] = 0;
            }
            continue;
        }
        long long f = 0;
        int mn = INT_MAX, mx = -1;
        unsigned bad = 0;
        double csum = 0.0;
        for (int64_t p = cb + lane; p < ce; p += 32) {
            const int k = A.rowidx[p];
            const float v = A.val[p];
            csum += (double)v;
            if (!(v >= 0.0f) || !(v <= FLT_MAX)) bad |= ERR_VALUE;
            if (p > cb && A.rowidx[p - 1] >= k) bad |= ERR_ROW_ORDER;
            if ((unsigned)k >= (unsigned)A.n) {
                bad |= ERR_ROW_RANGE;
                continue;
            }
            const int64_t ks = A.colptr[k], ke = A.colptr[k + 1];
            if (ks < 0 || ke < ks || ke > A.nnz) {
                bad |= ERR_COLPTR;
                continue;
            }
            if (ke > ks) {
                f += ke - ks;
                const int r0 = A.rowidx[ks], r1 = A.rowidx[ke - 1];
                mn = min(mn, r0);
                mx = max(mx, r1);
            }
        }
        bad = __reduce_or_sync(FULL, bad);
        f = warp_sum(f);
        csum = warp_sum(csum);
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) {
            if (bad) set_err(C, bad);
            const bool any = f > 0 && mx >= mn && mn >= 0;
            const int span = any ? (mx - mn + 1) : 0;
            b.flops[j] = f;
            if (b.colsum) b.colsum[j] = csum;
            b.rlo[j] = any ? mn : 0;
            b.rhi[j] = any ? mx : -1;
            long long cap = f < (long long)span ? f : (long long)span;
            if (cap > Krec) cap = Krec;
            const bool carried = b.active && !b.active[j];
            if (carried) cap = ce - cb;  // carried column: copied as is
            b.cap[j] = cap;
            if (!carried) fl_acc += (unsigned long long)f;  // multiply-adds of this iteration
            fl_max = fl_max > (unsigned long long)f ? fl_max : (unsigned long long)f;
            deg_max = max(deg_max, (int)(ce - cb));
            span_max = max(span_max, span);
        }
    }
    if (lane == 0) {
        if (fl_acc) atomicAdd(&C->flops, fl_acc);
        if (fl_max) atomicMax(&C->max_flops, fl_max);
        atomicMax(&C->max_deg, deg_max);
        atomicMax(&C->max_span, span_max);
    }
}

void launch_colstats(const CscView& A, const PruneParams& pp, const ExpandBuffers& b, int num_sms,
                     cudaStream_t s) {
    if (A.n == 0) return;
    int64_t warps = A.n;
    int64_t blocks = (warps * 32 + 255) / 256;
    int64_t maxb = (int64_t)num_sms * 8;
    if (blocks > maxb) blocks = maxb;
    k_colstats<<<(unsigned)blocks, 256, 0, s>>>(A, pp.Krec, b);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// exclusive scan (int64 output), three phases over 4096-element tiles
// ---------------------------------------------------------------------------

constexpr int SCAN_T = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_T * SCAN_ITEMS;

int64_t scan_tmp_len_for(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

template <typename TIn>
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const TIn* in, int64_t n, int64_t* tile) {
    __shared__ long long ws[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long sum = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int64_t i = base + (int64_t)q * SCAN_T + threadIdx.x;
        if (i < n) sum += (long long)in[i];
    }
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long x = ws[threadIdx.x];
        x = warp_sum(x);
        if (threadIdx.x == 0) tile[blockIdx.x] = x;
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_tilesums(int64_t* tile, int64_t ntiles,
                                                           unsigned long long* total) {
    __shared__ long long ws[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += SCAN_T) {
        int64_t i = base + threadIdx.x;
        long long x = i < ntiles ? tile[i] : 0;
        // inclusive warp scan
        long long v = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(FULL, v, o);
            if ((threadIdx.x & 31) >= o) v += y;
        }
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            long long w = ws[threadIdx.x];
            long long iw = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(FULL, iw, o);
                if (threadIdx.x >= (unsigned)o) iw += y;
            }
            ws[threadIdx.x] = iw - w;  // exclusive over warps
        }
        __syncthreads();
        long long excl = carry + ws[threadIdx.x >> 5] + v - x;
        if (i < ntiles) tile[i] = excl;
        __syncthreads();
        if (threadIdx.x == SCAN_T - 1) carry = excl + x;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = (unsigned long long)carry;
}

template <typename TIn>
__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const TIn* in, int64_t n,
                                                       const int64_t* tile, int64_t* out) {
    __shared__ long long ws[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    // each thread owns SCAN_ITEMS consecutive elements
    const int64_t my = base + (int64_t)threadIdx.x * SCAN_ITEMS;
    long long x[SCAN_ITEMS];
    long long local = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        x[q] = (my + q < n) ? (long long)in[my + q] : 0;
        local += x[q];
    }
    long long v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL, v, o);
        if ((threadIdx.x & 31) >= o) v += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long w = ws[threadIdx.x];
        long long iw = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(FULL, iw, o);
            if (threadIdx.x >= (unsigned)o) iw += y;
        }
        ws[threadIdx.x] = iw - w;
    }
    __syncthreads();
    long long run = tile[blockIdx.x] + ws[threadIdx.x >> 5] + v - local;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (my + q < n) out[my + q] = run;
        run += x[q];
    }
    if (my + SCAN_ITEMS - 1 >= n - 1 && my <= n - 1) {
        // the thread holding element n-1 writes out[n] = total
        out[n] = run;
    }
}

template <typename TIn>
void launch_exclusive_scan(const TIn* in, int64_t n, int64_t* out, int64_t* tmp,
                           unsigned long long* total, cudaStream_t s) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), s);
        if (total) cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
        return;
    }
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tiles<TIn><<<(unsigned)tiles, SCAN_T, 0, s>>>(in, n, tmp);
    count_launches(1);
    k_scan_tilesums<<<1, SCAN_T, 0, s>>>(tmp, tiles, total);
    count_launches(1);
    k_scan_apply<TIn><<<(unsigned)tiles, SCAN_T, 0, s>>>(in, n, tmp, out);
    count_launches(1);
}

template void launch_exclusive_scan<int64_t>(const int64_t*, int64_t, int64_t*, int64_t*,
                                             unsigned long long*, cudaStream_t);
template void launch_exclusive_scan<int32_t>(const int32_t*, int64_t, int64_t*, int64_t*,
                                             unsigned long long*, cudaStream_t);

// ---------------------------------------------------------------------------
// exact symbolic pass: nnz((AA)_*j) with a shared-memory bitmap
// ---------------------------------------------------------------------------

constexpr int SYM_T = 512;
constexpr int SYM_WORDS = 16384;  // 64 KB bitmap -> 524,288 rows per window

struct SymShared {
    BlockScratch bs;
    int item;
    int next;
};

__global__ void __launch_bounds__(SYM_T) k_symbolic(CscView A, ExpandBuffers b, int64_t* nnz_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem);
    SymShared* sh = reinterpret_cast<SymShared*>(bm + SYM_WORDS);
    const int tid = threadIdx.x, lane = tid & 31;
    constexpr int WB = SYM_WORDS * 32;
    int32_t* cur = b.cursors + (int64_t)blockIdx.x * 2 * b.cur_stride;
    for (;;) {
        if (tid == 0) sh->item = atomicAdd(&b.ctr->work_ctr, 1);
        __syncthreads();
        const int64_t j = sh->item;
        __syncthreads();
        if (j >= A.n) break;
        const int64_t cb = A.colptr[j], ce = A.colptr[j + 1];
        const int d = (int)(ce - cb);
        const int lo = b.rlo[j], hiE = b.rhi[j] + 1;
        if (d == 0 || hiE <= lo) {
            if (tid == 0) nnz_out[j] = 0;
            continue;
        }
        const int span = hiE - lo;
        const bool windows = span > WB;
        if (windows) {
            if (d > b.cur_stride) {  // cannot happen: cur_stride >= max degree
                if (tid == 0) set_err(b.ctr, ERR_CURSOR);
                continue;
            }
            for (int i = tid; i < d; i += SYM_T) cur[i] = 0;
        }
        long long cnt = 0;
        for (int r0 = lo; r0 < hiE;) {
            const int r1 = (int)min((int64_t)r0 + WB, (int64_t)hiE);
            const int nwords = (r1 - r0 + 31) >> 5;
            for (int i = tid; i < nwords; i += SYM_T) bm[i] = 0u;
            if (tid == 0) sh->next = 0;
            __syncthreads();
            for (;;) {
                int kidx = 0;
                if (lane == 0) kidx = atomicAdd(&sh->next, 1);
                kidx = __shfl_sync(FULL, kidx, 0);
                if (kidx >= d) break;
                const int k = __ldg(A.rowidx + cb + kidx);
                const int64_t ks = __ldg(A.colptr + k), ke = __ldg(A.colptr + k + 1);
                int64_t pos = ks + (windows ? cur[kidx] : 0);
                while (pos < ke) {
                    const int64_t q = pos + lane;
                    const bool valid = q < ke;
                    const int rr = valid ? __ldg(A.rowidx + q) : INT_MAX;
                    const bool in = valid && rr < r1;
                    const unsigned bal = __ballot_sync(FULL, in);
                    if (in) {
                        const int off = rr - r0;
                        const uint32_t bit = 1u << (off & 31);
                        uint32_t* w = bm + (off >> 5);
                        if (!(*reinterpret_cast<volatile uint32_t*>(w) & bit)) atomicOr(w, bit);
                    }
                    const int nin = __popc(bal);
                    pos += nin;
                    if (nin < 32) break;
                }
                if (windows && lane == 0) cur[kidx] = (int)(pos - ks);
            }
            __syncthreads();
            for (int i = tid; i < nwords; i += SYM_T) cnt += __popc(bm[i]);
            __syncthreads();
            r0 = r1;
        }
        double dd[1] = {0.0};
        long long qq[1] = {cnt};
        block_sum<SYM_T>(dd, 0, qq, 1, &sh->bs);
        if (tid == 0) nnz_out[j] = qq[0];
    }
}

// The dynamic shared-memory limit is a per-device attribute of the kernel:
// it is set on the current device before every launch, and the occupancy it
// gives is cached per device (first use under a lock).
static void symbolic_set_smem() {
    cudaFuncSetAttribute(k_symbolic, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(SYM_WORDS * 4 + sizeof(SymShared)));
}

int symbolic_grid(int num_sms) {
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static int occ_dev[kMaxDev] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    int occ = (dev >= 0 && dev < kMaxDev) ? occ_dev[dev] : 0;
    if (occ < 1) {
        symbolic_set_smem();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_symbolic, SYM_T,
                                                      SYM_WORDS * 4 + sizeof(SymShared));
        if (occ < 1) occ = 1;
        if (dev >= 0 && dev < kMaxDev) occ_dev[dev] = occ;
    }
    return occ * num_sms;
}

void launch_symbolic(const CscView& A, const ExpandBuffers& b, int64_t* nnz_out, int num_sms,
                     int grid_cap, cudaStream_t s) {
    if (A.n == 0) return;
    size_t smem = SYM_WORDS * 4 + sizeof(SymShared);
    symbolic_set_smem();
    int grid = symbolic_grid(num_sms);
    if (grid > grid_cap) grid = grid_cap;
    if ((int64_t)grid > A.n) grid = (int)A.n;
    cudaMemsetAsync(&b.ctr->work_ctr, 0, sizeof(int), s);
    k_symbolic<<<grid, SYM_T, smem, s>>>(A, b, nnz_out);
    count_launches(1);
}

// est_j = min(flops_j, span_j): an exact upper bound on nnz((AA)_*j)
__global__ void k_est_from_flops(int32_t n, ExpandBuffers b) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int64_t f = b.flops[j];
    int64_t span = (int64_t)b.rhi[j] - b.rlo[j] + 1;
    if (span < 0) span = 0;
    b.est[j] = f < span ? f : span;
}

// est_j <- max(1, est_j * milli / 1000): deliberate mis-estimation, used by
// tests to drive the overflow (range split) path.
__global__ void k_scale_est(int32_t n, int64_t* est, int milli) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int64_t e = (est[j] * milli) / 1000;
    est[j] = e < 1 ? 1 : e;
}

void launch_scale_est(int32_t n, int64_t* est, int milli, cudaStream_t s) {
    if (n == 0) return;
    k_scale_est<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, est, milli);
    count_launches(1);
}

// cap_j = min(cap_j, nnz_j) for active columns when nnz_j is exact
__global__ void k_cap_tighten(int32_t n, const int64_t* est, int64_t* cap, const uint8_t* active) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || (active && !active[j])) return;
    if (est[j] < cap[j]) cap[j] = est[j];
}

void launch_cap_tighten(int32_t n, const int64_t* est, int64_t* cap, const uint8_t* active,
                        cudaStream_t s) {
    if (n == 0) return;
    k_cap_tighten<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, est, cap, active);
    count_launches(1);
}

void launch_est_from_flops(const CscView& A, const ExpandBuffers& b, cudaStream_t s) {
    if (A.n == 0) return;
    k_est_from_flops<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(A.n, b);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// binning: configuration by estimated size, size classes for LPT order
// ---------------------------------------------------------------------------

// Configuration 0 (small CTA) takes columns whose estimate fits one small
// window's value capacity and whose span needs few windows; configuration 1
// takes the rest.  The size class orders work longest-first by flops_j.
__device__ __forceinline__ int bucket_of(int64_t est, int64_t flops, int span, int mask,
                                         int small_max) {
    int c = 1;
    if ((mask & 1) && est <= small_max && span <= 8 * 16384) c = 0;
    if (!(mask & 2)) c = 0;
    int64_t f = flops >> 12;
    const int lg = f > 0 ? 63 - __clzll((long long)f) : 0;
    const int z = NZ - 1 - (lg < NZ - 1 ? lg : NZ - 1);
    return c * NZ + z;
}

__global__ void k_bin_count(int32_t n, int mask, int small_max, ExpandBuffers b) {
    __shared__ int hist[NBUCKET];
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (b.active && !b.active[j]) {
            b.bucket[j] = -1;
            continue;
        }
        int bk = bucket_of(b.est[j], b.flops[j], b.rhi[j] - b.rlo[j] + 1, mask, small_max);
        b.bucket[j] = bk;
        atomicAdd(&hist[bk], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x)
        if (hist[i]) atomicAdd(&b.ctr->bin_cnt[i], hist[i]);
}

__global__ void k_bin_offsets(DevCounters* c) {
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < NBUCKET; ++i) {
            c->bin_off[i] = run;
            run += c->bin_cnt[i];
            c->bin_fill[i] = 0;
        }
        c->bin_off[NBUCKET] = run;
        for (int q = 0; q < NCONF; ++q) c->conf_ctr[q] = 0;
    }
}

__global__ void k_bin_scatter(int32_t n, ExpandBuffers b) {
    __shared__ int hist[NBUCKET];
    __shared__ int base[NBUCKET];
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bk = -1, rank = 0;
    if (j < n) {
        bk = b.bucket[j];
        if (bk >= 0) rank = atomicAdd(&hist[bk], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x)
        base[i] = hist[i] ? atomicAdd(&b.ctr->bin_fill[i], hist[i]) : 0;
    __syncthreads();
    if (bk >= 0) b.work[b.ctr->bin_off[bk] + base[bk] + rank] = (int32_t)j;
}

void launch_binning(const CscView& A, const PruneParams& pp, const ExpandBuffers& b, int mask,
                    cudaStream_t s) {
    cudaMemsetAsync(b.ctr->bin_cnt, 0, sizeof(int) * NBUCKET, s);
    if (A.n > 0) {
        int64_t blocks = (A.n + 255) / 256;
        k_bin_count<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(A.n, mask, pp.small_max,
                                                                               b);
        count_launches(1);
    }
    k_bin_offsets<<<1, 32, 0, s>>>(b.ctr);
    count_launches(1);
    if (A.n > 0) {
        k_bin_scatter<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(A.n, b);
        count_launches(1);
    }
}

// cap_j for the standalone prune: min(Krec, nnz(B_*j))
__global__ void k_prune_cap(CscView B, int32_t Krec, ExpandBuffers b) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B.n) return;
    int64_t m = B.colptr[j + 1] - B.colptr[j];
    b.cap[j] = m < Krec ? m : Krec;
}

void launch_prune_cap(const CscView& B, int32_t Krec, const ExpandBuffers& b, cudaStream_t s) {
    if (B.n == 0) return;
    k_prune_cap<<<(unsigned)((B.n + 255) / 256), 256, 0, s>>>(B, Krec, b);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// compaction, statistics, standalone inflation and chaos
// ---------------------------------------------------------------------------

// Warp per column: copy the kept entries from the capacity layout to the
// final CSC (or, for a carried inactive column, the input column).
__global__ void k_compact(CscView A, ExpandBuffers b, const int64_t* colptr_out, int32_t* row_out,
                          float* val_out) {
    if (b.ctr->err & ERR_STAGING) return;  // the iteration is redone without the graph
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < A.n; j += nw) {
        const int64_t dst = colptr_out[j];
        const int64_t len = colptr_out[j + 1] - dst;
        if (b.active && !b.active[j]) {
            const int64_t src = A.colptr[j];
            for (int64_t i = lane; i < len; i += 32) {
                row_out[dst + i] = A.rowidx[src + i];
                val_out[dst + i] = A.val[src + i];
            }
        } else {
            const int64_t src = b.off[j] - b.tmp_off0;
            for (int64_t i = lane; i < len; i += 32) {
                row_out[dst + i] = b.tmp_row[src + i];
                val_out[dst + i] = b.tmp_val[src + i];
            }
        }
    }
}

// Compaction of one column batch [c0, c1): colptr_local[j - c0] indexes
// the batch's own output segment.
__global__ void k_compact_range(ExpandBuffers b, int32_t c0, int32_t c1,
                                const int64_t* colptr_local, int32_t* row_out, float* val_out) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = c0 + gw; j < c1; j += nw) {
        const int64_t dst = colptr_local[j - c0];
        const int64_t len = colptr_local[j - c0 + 1] - dst;
        const int64_t src = b.off[j] - b.tmp_off0;
        for (int64_t i = lane; i < len; i += 32) {
            row_out[dst + i] = b.tmp_row[src + i];
            val_out[dst + i] = b.tmp_val[src + i];
        }
    }
}

void launch_compact_range(const CscView& A, const ExpandBuffers& b, int32_t c0, int32_t c1,
                          const int64_t* colptr_local, int32_t* row_out, float* val_out,
                          cudaStream_t s) {
    (void)A;
    if (c1 <= c0) return;
    int64_t blocks = ((int64_t)(c1 - c0) * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_compact_range<<<(unsigned)blocks, 256, 0, s>>>(b, c0, c1, colptr_local, row_out, val_out);
    count_launches(1);
}

__global__ void k_range_mask(int32_t n, int32_t c0, int32_t c1, uint8_t* mask) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) mask[j] = (j >= c0 && j < c1) ? 1 : 0;
}

void launch_range_mask(int32_t n, int32_t c0, int32_t c1, uint8_t* mask, cudaStream_t s) {
    if (n == 0) return;
    k_range_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c0, c1, mask);
    count_launches(1);
}

void launch_compact(const CscView& A, const ExpandBuffers& b, const int64_t* colptr_out,
                    int32_t* row_out, float* val_out, cudaStream_t s) {
    if (A.n == 0) return;
    int64_t blocks = (A.n * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_compact<<<(unsigned)blocks, 256, 0, s>>>(A, b, colptr_out, row_out, val_out);
    count_launches(1);
}

// Reduce chaos_j (max, as ordered bits) and nnz(B_*j) (sum) over active columns.
__global__ void k_finalize_stats(int32_t n, ExpandBuffers b) {
    __shared__ double smax[32];
    __shared__ long long ssum[32];
    double mx = 0.0;
    long long sb = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (b.active && !b.active[j]) continue;
        mx = fmax(mx, b.chaos[j]);
        sb += b.bnnz[j];
    }
    mx = warp_max(mx);
    sb = warp_sum(sb);
    if ((threadIdx.x & 31) == 0) {
        smax[threadIdx.x >> 5] = mx;
        ssum[threadIdx.x >> 5] = sb;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        double m2 = threadIdx.x < (unsigned)nw ? smax[threadIdx.x] : 0.0;
        long long s2 = threadIdx.x < (unsigned)nw ? ssum[threadIdx.x] : 0;
        m2 = warp_max(m2);
        s2 = warp_sum(s2);
        if (threadIdx.x == 0) {
            atomicMax(&b.ctr->chaos_bits, (unsigned long long)__double_as_longlong(m2));
            atomicAdd(&b.ctr->nnz_b, (unsigned long long)s2);
        }
    }
}

void launch_finalize_stats(int32_t n, const ExpandBuffers& b, cudaStream_t s) {
    if (n == 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    k_finalize_stats<<<(unsigned)blocks, 256, 0, s>>>(n, b);
    count_launches(1);
}

// Warp per column: v <- v^r / sum v^r (FP32 power, FP64 sum).
__global__ void k_inflate_normalize(int32_t n, const int64_t* colptr, float* val, float r) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw) {
        const int64_t cb = colptr[j], ce = colptr[j + 1];
        double s = 0.0;
        for (int64_t p = cb + lane; p < ce; p += 32) s += (double)inflate_value(val[p], r);
        s = warp_sum(s);
        for (int64_t p = cb + lane; p < ce; p += 32) {
            const float u = inflate_value(val[p], r);
            val[p] = s > 0.0 ? (float)((double)u / s) : 0.0f;
        }
    }
}

void launch_inflate_normalize(int32_t n, const int64_t* colptr, float* val, float r,
                              cudaStream_t s) {
    if (n == 0) return;
    int64_t blocks = ((int64_t)n * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_inflate_normalize<<<(unsigned)blocks, 256, 0, s>>>(n, colptr, val, r);
    count_launches(1);
}

// Warp per column: chaos_j = max(0, max a - sum a^2) in FP64; max over j.
__global__ void k_chaos(int32_t n, const int64_t* colptr, const float* val, double* chaos_cols,
                        DevCounters* ctr) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double best = 0.0;
    for (int64_t j = gw; j < n; j += nw) {
        const int64_t cb = colptr[j], ce = colptr[j + 1];
        double mx = 0.0, sq = 0.0;
        for (int64_t p = cb + lane; p < ce; p += 32) {
            const double a = (double)val[p];
            mx = a > mx ? a : mx;
            sq += a * a;
        }
        mx = warp_max(mx);
        sq = warp_sum(sq);
        double c = mx - sq;
        if (c < 0.0) c = 0.0;
        if (lane == 0 && chaos_cols) chaos_cols[j] = c;
        best = c > best ? c : best;
    }
    if (lane == 0)
        atomicMax(&ctr->chaos_bits, (unsigned long long)__double_as_longlong(best));
}

void launch_chaos(int32_t n, const int64_t* colptr, const float* val, double* chaos_cols,
                  DevCounters* ctr, cudaStream_t s) {
    if (n == 0) return;
    int64_t blocks = ((int64_t)n * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_chaos<<<(unsigned)blocks, 256, 0, s>>>(n, colptr, val, chaos_cols, ctr);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// batched components: per-column component, active mask, per-component chaos
// ---------------------------------------------------------------------------

// comp_of_col[j] = c with off[c] <= j < off[c+1] (binary search); flags a
// column whose rows leave its component (the batch must be block diagonal).
__global__ void k_comp_assign(CscView A, const int32_t* off, int32_t ncomp, int32_t* comp_of_col,
                              DevCounters* ctr) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.n) return;
    int lo = 0, hi = ncomp;  // invariant: off[lo] <= j < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid;
    }
    comp_of_col[j] = lo;
    const int64_t cb = A.colptr[j], ce = A.colptr[j + 1];
    if (ce > cb) {
        const int r0 = A.rowidx[cb], r1 = A.rowidx[ce - 1];
        if (r0 < off[lo] || r1 >= off[lo + 1]) atomicOr(&ctr->err, ERR_ROW_RANGE);
    }
}

__global__ void k_active_from_comp(int32_t n, const int32_t* comp_of_col, const uint8_t* comp_active,
                                   uint8_t* active) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) active[j] = comp_active[comp_of_col[j]];
}

// kept count of a carried (inactive) column = its input length
__global__ void k_fill_inactive(CscView A, const uint8_t* active, int32_t* kept) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < A.n && !active[j]) kept[j] = (int32_t)(A.colptr[j + 1] - A.colptr[j]);
}

// max chaos_j per component over its active columns (ordered bits, >= 0);
// the lanes of a warp are grouped by component, one atomic per group
__global__ void k_comp_chaos(int32_t n, const int32_t* comp_of_col, const uint8_t* active,
                             const double* chaos, unsigned long long* comp_bits) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = j < n && active[j];
    const int c = valid ? comp_of_col[j] : -1;
    const unsigned long long bits = valid ? (unsigned long long)__double_as_longlong(chaos[j]) : 0ull;
    unsigned rem = __ballot_sync(FULL, valid);
    while (rem) {
        const int leader = __ffs(rem) - 1;
        const int cl = __shfl_sync(FULL, c, leader);
        const bool mine = valid && c == cl;
        unsigned long long v = mine ? bits : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(FULL, v, o);
            v = y > v ? y : v;
        }
        if (lane == leader) atomicMax(comp_bits + cl, v);
        rem &= ~__ballot_sync(FULL, mine);
    }
}

void launch_comp_assign(const CscView& A, const int32_t* off, int32_t ncomp, int32_t* comp_of_col,
                        DevCounters* ctr, cudaStream_t s) {
    if (A.n == 0) return;
    k_comp_assign<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(A, off, ncomp, comp_of_col, ctr);
    count_launches(1);
}

void launch_active_from_comp(int32_t n, const int32_t* comp_of_col, const uint8_t* comp_active,
                             uint8_t* active, cudaStream_t s) {
    if (n == 0) return;
    k_active_from_comp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, comp_of_col, comp_active,
                                                                    active);
    count_launches(1);
}

void launch_fill_inactive(const CscView& A, const uint8_t* active, int32_t* kept, cudaStream_t s) {
    if (A.n == 0) return;
    k_fill_inactive<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(A, active, kept);
    count_launches(1);
}

void launch_comp_chaos(int32_t n, const int32_t* comp_of_col, const uint8_t* active,
                       const double* chaos, unsigned long long* comp_bits, cudaStream_t s) {
    if (n == 0) return;
    k_comp_chaos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, comp_of_col, active, chaos,
                                                              comp_bits);
    count_launches(1);
}

// Components whose chaos dropped below eps stop; the rest are counted.
__global__ void k_comp_retire(int32_t ncomp, const unsigned long long* comp_bits, double eps,
                              uint8_t* comp_active, DevCounters* ctr) {
    if (ctr->err & ERR_STAGING) return;  // the iteration did not run; it is redone
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    int live = 0;
    if (q < ncomp && comp_active[q]) {
        if (__longlong_as_double((long long)comp_bits[q]) < eps)
            comp_active[q] = 0;
        else
            live = 1;
    }
    live = __reduce_add_sync(FULL, live);
    if ((threadIdx.x & 31) == 0 && live) atomicAdd(&ctr->n_active, live);
}

void launch_comp_retire(int32_t ncomp, const unsigned long long* comp_bits, double eps,
                        uint8_t* comp_active, DevCounters* ctr, cudaStream_t s) {
    if (ncomp <= 0) return;
    k_comp_retire<<<(unsigned)((ncomp + 255) / 256), 256, 0, s>>>(ncomp, comp_bits, eps,
                                                                   comp_active, ctr);
    count_launches(1);
}

// Flags an output staging that cannot hold the capacities of this iteration
// (the numeric pass and the compaction then write nothing).
__global__ void k_staging_guard(DevCounters* ctr, int64_t capacity) {
    if (threadIdx.x == 0 && (int64_t)ctr->cap_total > capacity) atomicOr(&ctr->err, ERR_STAGING);
}

void launch_staging_guard(DevCounters* ctr, int64_t capacity, cudaStream_t s) {
    k_staging_guard<<<1, 32, 0, s>>>(ctr, capacity);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// groups of components: the diagonal block [lo, hi) of a block-diagonal CSC
// as a matrix of its own (rows re-based), and the way back
// ---------------------------------------------------------------------------

// colptr_g[i] = colptr[lo + i] - colptr[lo] for i in [0, ng] (grid-stride:
// the grid is capped)
__global__ void k_block_colptr(const int64_t* colptr, int32_t lo, int32_t ng, int64_t* colptr_g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= ng;
         i += (int64_t)gridDim.x * blockDim.x)
        colptr_g[i] = colptr[lo + i] - colptr[lo];
}

// dst[p] = src[p] + delta for p in [0, m)
__global__ void k_add_i32(const int32_t* src, int64_t m, int32_t delta, int32_t* dst) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = src[p] + delta;
}

// colptr[lo + i] = colptr_g[i] + base for i in [0, ng) (and colptr[lo + ng]
// when last)
__global__ void k_place_colptr(const int64_t* colptr_g, int32_t lo, int32_t ng, int64_t base,
                               int last, int64_t* colptr) {
    const int64_t end = last ? (int64_t)ng + 1 : (int64_t)ng;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x)
        colptr[lo + i] = colptr_g[i] + base;
}

static unsigned grid_for(int64_t m) {
    int64_t b = (m + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

void launch_block_colptr(const int64_t* colptr, int32_t lo, int32_t ng, int64_t* colptr_g,
                         cudaStream_t s) {
    k_block_colptr<<<grid_for((int64_t)ng + 1), 256, 0, s>>>(colptr, lo, ng, colptr_g);
    count_launches(1);
}

void launch_add_i32(const int32_t* src, int64_t m, int32_t delta, int32_t* dst, cudaStream_t s) {
    if (m <= 0) return;
    k_add_i32<<<grid_for(m), 256, 0, s>>>(src, m, delta, dst);
    count_launches(1);
}

void launch_place_colptr(const int64_t* colptr_g, int32_t lo, int32_t ng, int64_t base, int last,
                         int64_t* colptr, cudaStream_t s) {
    k_place_colptr<<<grid_for((int64_t)ng + 1), 256, 0, s>>>(colptr_g, lo, ng, base, last, colptr);
    count_launches(1);
}

// The device counters into host-mapped memory, one 8-byte word per thread.
__global__ void k_copy_counters(const DevCounters* src, DevCounters* dst) {
    constexpr int W = (int)(sizeof(DevCounters) / 8);
    static_assert(sizeof(DevCounters) % 8 == 0, "counters are whole 8-byte words");
    const int i = threadIdx.x;
    if (i < W) reinterpret_cast<unsigned long long*>(dst)[i] =
        reinterpret_cast<const unsigned long long*>(src)[i];
}

void launch_copy_counters(const DevCounters* src, DevCounters* dst, cudaStream_t s) {
    k_copy_counters<<<1, (int)((sizeof(DevCounters) / 8 + 31) / 32 * 32), 0, s>>>(src, dst);
    count_launches(1);
}

__global__ void k_fill_colptr(int32_t n, int64_t* colptr) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j <= n) colptr[j] = 0;
}

void launch_fill_colptr(int32_t n, int64_t* colptr, cudaStream_t s) {
    k_fill_colptr<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(n, colptr);
    count_launches(1);
}

}  // namespace mcl
