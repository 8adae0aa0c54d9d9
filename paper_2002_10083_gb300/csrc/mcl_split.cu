// The expansion with its inner dimension split into stages, and the binary
// merge of the stages' partial products (Section IV, "Binary merge";
// Algorithm 2).
//
// B = A A = sum_t P_t, where stage t multiplies the columns of A by the rows
// k of A in block t of the inner index: P_t(:, j) = sum over k in block t of
// a_kj A(:, k).  A partial product is unpruned, its columns sorted by row,
// and its entries are the exact 64-bit fixed-point sums the numeric pass
// uses (every column's scale comes from the same column sum s_j =
// sum_k a_kj colsum_k(A), in the same order), so partial products add
// exactly and the merged product, pruned, equals the one-pass iteration bit
// for bit.
//
// One kernel does both jobs on row-sorted inputs: for each output column a
// CTA walks its sources (the columns of A of one stage, scaled by a_kj, or
// the columns of the partial products being merged) in windows of RA_WB
// rows; a shared bitmap marks the rows present (count mode: their number),
// a prefix count of the bitmap gives each row its position in the output
// column, and the values are added there with 64-bit integer atomics (fill
// mode), so the output comes out sorted and its sums do not depend on the
// order of the additions.
#include <climits>
#include <cstdint>

#include "mcl_device.cuh"
#include "mcl_internal.h"

namespace mcl {

// Column sums of B from the identity sum_i (AA)_ij = sum_k a_kj colsum_k(A):
// warp per column, lane l taking the column's entries l, l + 32, ..., then a
// butterfly -- the order of the numeric pass, so the same doubles.
__global__ void k_bsum(CscView A, const double* colsum, double* bsum) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < A.n; j += nw) {
        const int64_t cb = A.colptr[j];
        const int d = (int)(A.colptr[j + 1] - cb);
        double s = 0.0;
        for (int i = lane; i < d; i += 32) s += (double)A.val[cb + i] * colsum[A.rowidx[cb + i]];
        s = warp_sum(s);
        if (lane == 0) bsum[j] = s;
    }
}

void launch_bsum(const CscView& A, const double* colsum, double* bsum, cudaStream_t s) {
    if (A.n == 0) return;
    int64_t blocks = ((int64_t)A.n * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_bsum<<<(unsigned)blocks, 256, 0, s>>>(A, colsum, bsum);
    count_launches(1);
}

constexpr int RA_T = 512;
constexpr int RA_WORDS = 16384;          // 64 KB bitmap
constexpr int RA_WB = RA_WORDS * 32;     // rows per window

struct RankShared {
    BlockScratch bs;
    int wsm[34];
    int item;
    int next;
    int ns;
    int lo, hi;  // row span of the column's sources
    long long base;
};

// Sources of one output column, per CTA in global scratch (stride entries):
// row arrays, value arrays (FP32 of A or uint64 sums), lengths, a_kj and
// the cursors of the window walk.
struct RankScratch {
    const int32_t** rows;
    const void** vals;
    int32_t* len;
    float* akj;
    int32_t* cur;
    int32_t* nxt;
};



template <int T>
__device__ __forceinline__ int block_min_max(int x, bool is_max, BlockScratch* bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = is_max ? warp_max(x) : warp_min(x);
    if (lane == 0) bs->q[2][warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long y = lane < T / 32 ? bs->q[2][lane] : (is_max ? INT_MIN : INT_MAX);
        int yi = (int)y;
        yi = is_max ? warp_max(yi) : warp_min(yi);
        if (lane == 0) bs->q[2][32] = yi;
    }
    __syncthreads();
    const int r = (int)bs->q[2][32];
    __syncthreads();
    return r;
}

// STAGE: sources are the columns k of A in [k0, k1) referenced by column j;
// otherwise the columns j of the partial products.  FILL: write the output
// (else count it).
template <bool STAGE, bool FILL>
__global__ void __launch_bounds__(RA_T) k_rank_acc(RankArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem);
    int32_t* wpre = reinterpret_cast<int32_t*>(bm + RA_WORDS);  // FILL only
    RankShared* sh = reinterpret_cast<RankShared*>(smem + (size_t)RA_WORDS * 4 * (FILL ? 2 : 1));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NWP = RA_T / 32;
    unsigned long long* sb = reinterpret_cast<unsigned long long*>(a.scratch) +
                             (int64_t)blockIdx.x * 6 * a.stride;
    RankScratch rs{reinterpret_cast<const int32_t**>(sb),
                   reinterpret_cast<const void**>(sb + a.stride),
                   reinterpret_cast<int32_t*>(sb + 2 * a.stride),
                   reinterpret_cast<float*>(sb + 3 * a.stride),
                   reinterpret_cast<int32_t*>(sb + 4 * a.stride),
                   reinterpret_cast<int32_t*>(sb + 5 * a.stride)};
    for (;;) {
        if (tid == 0) sh->item = atomicAdd(&a.ctr->work_ctr, 1);
        __syncthreads();
        const int64_t j = sh->item;
        __syncthreads();
        if (j >= a.n) break;
        // ---- the column's sources ----
        int ns = 0;
        int64_t i0 = 0;
        if (STAGE) {
            const int64_t cb = a.A.colptr[j], ce = a.A.colptr[j + 1];
            if (tid == 0) {
                int64_t lo = cb, hi = ce;  // first entry with row >= k0
                while (lo < hi) {
                    const int64_t m = (lo + hi) >> 1;
                    if (a.A.rowidx[m] < a.k0) lo = m + 1; else hi = m;
                }
                int64_t lo2 = lo, hi2 = ce;  // first entry with row >= k1
                while (lo2 < hi2) {
                    const int64_t m = (lo2 + hi2) >> 1;
                    if (a.A.rowidx[m] < a.k1) lo2 = m + 1; else hi2 = m;
                }
                sh->ns = (int)(lo2 - lo);
                sh->base = lo;
            }
            __syncthreads();
            ns = sh->ns;
            i0 = sh->base;
        } else {
            ns = a.nparts;
        }
        if (ns > a.stride) {  // cannot happen: the stride exceeds the longest column
            if (tid == 0) {
                atomicOr(&a.ctr->err, ERR_CURSOR);
                if (!FILL) a.nnz_out[j] = 0;
            }
            __syncthreads();
            continue;
        }
        int mn = INT_MAX, mx = INT_MIN;
        for (int s = tid; s < ns; s += RA_T) {
            const int32_t* rows;
            const void* vals;
            int len;
            float f = 1.0f;
            if (STAGE) {
                const int k = a.A.rowidx[i0 + s];
                const int64_t ks = a.A.colptr[k];
                rows = a.A.rowidx + ks;
                vals = a.A.val + ks;
                len = (int)(a.A.colptr[k + 1] - ks);
                f = a.A.val[i0 + s];
            } else {
                const int64_t ps = a.pcol[s][j];
                rows = a.prow[s] + ps;
                vals = a.pval[s] + ps;
                len = (int)(a.pcol[s][j + 1] - ps);
            }
            rs.rows[s] = rows;
            rs.vals[s] = vals;
            rs.len[s] = len;
            rs.akj[s] = f;
            rs.cur[s] = 0;
            if (len > 0) {
                mn = min(mn, rows[0]);
                mx = max(mx, rows[len - 1]);
            }
        }
        const int lo = block_min_max<RA_T>(mn, false, &sh->bs);
        const int hiE = block_min_max<RA_T>(mx, true, &sh->bs) + 1;
        FixScale fx;
        fx.init(STAGE ? a.bsum[j] : 1.0);
        long long cnt = 0;
        int64_t obase = FILL ? a.colptr_out[j] : 0;
        int32_t* cur = rs.cur;
        int32_t* nxt = rs.nxt;
        for (int r0 = lo; r0 < hiE && hiE > lo;) {
            const int r1 = (int)min((int64_t)r0 + RA_WB, (int64_t)hiE);
            const int nwords = (r1 - r0 + 31) >> 5;
            for (int i = tid; i < nwords; i += RA_T) bm[i] = 0u;
            if (tid == 0) sh->next = 0;
            __syncthreads();
            // ---- mark the rows of the window ----
            for (;;) {
                int s = 0;
                if (lane == 0) s = atomicAdd(&sh->next, 1);
                s = __shfl_sync(FULL, s, 0);
                if (s >= ns) break;
                const int32_t* rows = rs.rows[s];
                const int len = rs.len[s];
                int pos = cur[s];
                while (pos < len) {
                    const int p = pos + lane;
                    const int row = p < len ? __ldg(rows + p) : INT_MAX;
                    const bool in = row < r1;
                    if (in) {
                        const int off = row - r0;
                        atomicOr(bm + (off >> 5), 1u << (off & 31));
                    }
                    const int nin = __popc(__ballot_sync(FULL, in));
                    pos += nin;
                    if (nin < 32) break;
                }
                if (lane == 0) nxt[s] = pos;
            }
            __syncthreads();
            if (!FILL) {
                for (int i = tid; i < nwords; i += RA_T) cnt += __popc(bm[i]);
                __syncthreads();
            } else {
                // ---- positions: exclusive prefix counts of the bitmap words ----
                constexpr int PER = RA_WORDS / RA_T;
                int loc[PER];
                int tsum = 0;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    const int w = tid * PER + q;
                    loc[q] = tsum;
                    tsum += w < nwords ? __popc(bm[w]) : 0;
                }
                // block exclusive scan of tsum
                int incl = tsum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) sh->wsm[warp] = incl;
                __syncthreads();
                if (warp == 0) {
                    const int w0 = lane < NWP ? sh->wsm[lane] : 0;
                    int wi = w0;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(FULL, wi, o);
                        if (lane >= o) wi += y;
                    }
                    if (lane < NWP) sh->wsm[lane] = wi - w0;
                    if (lane == 31) sh->wsm[32] = wi;
                }
                __syncthreads();
                const int tbase = sh->wsm[warp] + incl - tsum;
#pragma unroll
                for (int q = 0; q < PER; ++q) wpre[tid * PER + q] = tbase + loc[q];
                const int wtot = sh->wsm[32];
                if (tid == 0) sh->next = 0;
                __syncthreads();
                // ---- add every product at its row's position ----
                for (;;) {
                    int s = 0;
                    if (lane == 0) s = atomicAdd(&sh->next, 1);
                    s = __shfl_sync(FULL, s, 0);
                    if (s >= ns) break;
                    const int32_t* rows = rs.rows[s];
                    const int len = rs.len[s];
                    const float f = rs.akj[s];
                    for (int pos = cur[s]; pos < nxt[s]; pos += 32) {
                        const int p = pos + lane;
                        if (p < nxt[s]) {
                            const int row = __ldg(rows + p);
                            const int off = row - r0;
                            const uint32_t word = bm[off >> 5];
                            const int rank =
                                wpre[off >> 5] + __popc(word & ((1u << (off & 31)) - 1u));
                            unsigned long long q;
                            if (STAGE)
                                q = fx.q(__ldg(reinterpret_cast<const float*>(rs.vals[s]) + p), f);
                            else
                                q = reinterpret_cast<const unsigned long long*>(rs.vals[s])[p];
                            const int64_t at = obase + rank;
                            a.row_out[at] = row;
                            atomicAdd(a.val_out + at, q);
                        }
                    }
                }
                obase += wtot;
                __syncthreads();
            }
            int32_t* t = cur;
            cur = nxt;
            nxt = t;
            r0 = r1;
        }
        if (!FILL) {
            double dd[1] = {0.0};
            long long qq[1] = {cnt};
            block_sum<RA_T>(dd, 0, qq, 1, &sh->bs);
            if (tid == 0) a.nnz_out[j] = qq[0];
        }
    }
}

template <bool STAGE, bool FILL>
static void rank_launch(const RankArgs& a, int num_sms, cudaStream_t s) {
    const size_t smem = (size_t)RA_WORDS * 4 * (FILL ? 2 : 1) + sizeof(RankShared);
    auto kern = k_rank_acc<STAGE, FILL>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, RA_T, smem);
    if (occ < 1) occ = 1;
    int grid = occ * num_sms;
    if (grid > a.grid_cap) grid = a.grid_cap;
    if ((int64_t)grid > a.n) grid = a.n > 0 ? (int)a.n : 1;
    cudaMemsetAsync(&a.ctr->work_ctr, 0, sizeof(int), s);
    kern<<<grid, RA_T, smem, s>>>(a);
    count_launches(1);
}

void launch_split_count(const RankArgs& a, bool stage, int num_sms, cudaStream_t s) {
    if (a.n == 0) return;
    if (stage)
        rank_launch<true, false>(a, num_sms, s);
    else
        rank_launch<false, false>(a, num_sms, s);
}

void launch_split_fill(const RankArgs& a, bool stage, int num_sms, cudaStream_t s) {
    if (a.n == 0) return;
    if (stage)
        rank_launch<true, true>(a, num_sms, s);
    else
        rank_launch<false, true>(a, num_sms, s);
}

}  // namespace mcl
