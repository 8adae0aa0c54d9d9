// Internal interface between the C ABI (mcl_api.cu) and the kernels
// (mcl_kernels.cu, mcl_cc.cu).  Not installed; not part of the ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcl {

// Configurations of the fused numeric pass (mcl_numeric.cu): 0 = small CTA
// and window for small columns, 1 = large CTA and window for the rest.
constexpr int NCONF = 2;
constexpr int NZ = 8;                    // size classes per configuration
constexpr int NBUCKET = NCONF * NZ;
// device-side counters (one small block of memory per context)
struct DevCounters {
    unsigned long long misses;       // columns whose nnz exceeded the estimate
    unsigned long long splits;       // range overflows resolved by halving
    unsigned long long flops;        // sum of flops_j
    unsigned long long nnz_b;        // sum of nnz(B_*j)
    unsigned long long chaos_bits;   // max chaos_j as ordered bits (>= 0)
    unsigned long long cap_total;    // sum of output capacities
    unsigned long long nnz_out;      // sum of kept counts
    unsigned long long max_flops;    // max_j flops_j
    int max_deg;
    int max_span;
    unsigned err;                    // bit flags (ERR_*)
    int pad;
    int bin_cnt[NBUCKET];
    int bin_off[NBUCKET + 1];
    int bin_fill[NBUCKET];
    int conf_ctr[NCONF];
    int work_ctr;
    int n_active;                    // components still iterating (graph replay)
    int pad2;
};

enum : unsigned {
    ERR_COLPTR = 1u,      // colptr not monotone / out of [0, nnz]
    ERR_ROW_RANGE = 2u,   // row index outside [0, n)
    ERR_ROW_ORDER = 4u,   // rows not strictly increasing in a column
    ERR_VALUE = 8u,       // value negative, NaN or infinite
    ERR_INTERNAL = 16u,   // device consistency check failed
    ERR_TIMEOUT = 32u,    // bounded loop gave up
    ERR_CURSOR = 64u,     // cursor scratch too small
    ERR_STAGING = 128u,   // output staging of a graph replay too small (nothing written)
};

struct CscView {
    int32_t n;
    int64_t nnz;
    const int64_t* colptr;
    const int32_t* rowidx;
    const float* val;
};

struct PruneParams {
    float theta;
    int32_t K;
    float p;
    int32_t Krec;
    int32_t ksel;   // max(K, Krec)
    float r;
    int32_t inflate;
    // tuning (autotuner): columns estimated at <= small_max entries use the
    // small configuration; shape of the large one; entries planned per
    // hashed window
    int32_t small_max;
    int32_t table;
    int32_t plan;
};

struct ExpandBuffers {
    int64_t* flops;     // [n]
    double* colsum;     // [n]   column sums of A (FP64)
    int32_t* rlo;       // [n]
    int32_t* rhi;       // [n]
    int64_t* cap;       // [n]   output capacity min(Krec, flops, span)
    int64_t* off;       // [n+1] exclusive scan of cap
    int64_t* est;       // [n]   size estimate used for binning
    int32_t* bucket;    // [n]
    int32_t* work;      // [n]
    int32_t* kept;      // [n]
    double* chaos;      // [n]
    int64_t* bnnz;      // [n]
    int32_t* tmp_row;   // [cap_total] (or one column batch's share)
    float* tmp_val;     // [cap_total]
    int64_t tmp_off0;   // staging index of column j is off[j] - tmp_off0
    int32_t* cursors;   // per CTA: source metadata, 6 * cur_stride int32
    int64_t cur_stride;
    int32_t* bucket_row;   // per CTA: bucket_cap (row, bits(a_ik * a_kj)) pairs (int2)
    int32_t* woff;         // per CTA: window offsets into the bucket (WINDOW_MAX + 1)
    int64_t bucket_cap;
    int64_t* scan_tmp;  // tile sums
    int64_t scan_tmp_len;
    DevCounters* ctr;
    const uint8_t* active;  // optional per-column mask (NULL: all active)
    int32_t nnz_is_bound;   // A.nnz is the capacity of A's arrays, not colptr[n]
};

// --- launch accounting (every launcher adds the kernels it starts) ---
void count_launches(int k);
long long launches_total();

// --- launchers (mcl_kernels.cu) ---
void launch_colstats(const CscView& A, const PruneParams& pp, const ExpandBuffers& b,
                     int num_sms, cudaStream_t s);
int64_t scan_tmp_len_for(int64_t n);
template <typename TIn>
void launch_exclusive_scan(const TIn* in, int64_t n, int64_t* out, int64_t* tmp,
                           unsigned long long* total, cudaStream_t s);
void launch_symbolic(const CscView& A, const ExpandBuffers& b, int64_t* nnz_out, int num_sms,
                     int grid_cap, cudaStream_t s);
int symbolic_grid(int num_sms);
void launch_scale_est(int32_t n, int64_t* est, int milli, cudaStream_t s);
void launch_cap_tighten(int32_t n, const int64_t* est, int64_t* cap, const uint8_t* active,
                        cudaStream_t s);
void launch_est_from_flops(const CscView& A, const ExpandBuffers& b, cudaStream_t s);
void launch_binning(const CscView& A, const PruneParams& pp, const ExpandBuffers& b, int mask,
                    cudaStream_t s);
int numeric_grid(int conf, const PruneParams& pp, int num_sms);
size_t numeric_smem(int conf, const PruneParams& pp);
constexpr int WINDOW_MAX = 4096;  // windows per column in bucket mode
void launch_numeric(int conf, const CscView& A, const PruneParams& pp, const ExpandBuffers& b,
                    int grid, cudaStream_t s);
void launch_compact(const CscView& A, const ExpandBuffers& b, const int64_t* colptr_out,
                    int32_t* row_out, float* val_out, cudaStream_t s);
void launch_finalize_stats(int32_t n, const ExpandBuffers& b, cudaStream_t s);
void launch_range_mask(int32_t n, int32_t c0, int32_t c1, uint8_t* mask, cudaStream_t s);
void launch_compact_range(const CscView& A, const ExpandBuffers& b, int32_t c0, int32_t c1,
                          const int64_t* colptr_local, int32_t* row_out, float* val_out,
                          cudaStream_t s);
void launch_prune_cap(const CscView& B, int32_t Krec, const ExpandBuffers& b, cudaStream_t s);
void launch_prune(const CscView& B, const PruneParams& pp, const ExpandBuffers& b, int num_sms,
                  cudaStream_t s);
void launch_inflate_normalize(int32_t n, const int64_t* colptr, float* val, float r,
                              cudaStream_t s);
void launch_chaos(int32_t n, const int64_t* colptr, const float* val, double* chaos_cols,
                  DevCounters* ctr, cudaStream_t s);
void launch_fill_colptr(int32_t n, int64_t* colptr, cudaStream_t s);
void launch_comp_assign(const CscView& A, const int32_t* off, int32_t ncomp, int32_t* comp_of_col,
                        DevCounters* ctr, cudaStream_t s);
void launch_active_from_comp(int32_t n, const int32_t* comp_of_col, const uint8_t* comp_active,
                             uint8_t* active, cudaStream_t s);
void launch_fill_inactive(const CscView& A, const uint8_t* active, int32_t* kept, cudaStream_t s);
void launch_comp_chaos(int32_t n, const int32_t* comp_of_col, const uint8_t* active,
                       const double* chaos, unsigned long long* comp_bits, cudaStream_t s);
void launch_comp_retire(int32_t ncomp, const unsigned long long* comp_bits, double eps,
                        uint8_t* comp_active, DevCounters* ctr, cudaStream_t s);
void launch_staging_guard(DevCounters* ctr, int64_t capacity, cudaStream_t s);
void launch_copy_counters(const DevCounters* src, DevCounters* dst, cudaStream_t s);
void launch_block_colptr(const int64_t* colptr, int32_t lo, int32_t ng, int64_t* colptr_g,
                         cudaStream_t s);
void launch_add_i32(const int32_t* src, int64_t m, int32_t delta, int32_t* dst, cudaStream_t s);
void launch_place_colptr(const int64_t* colptr_g, int32_t lo, int32_t ng, int64_t base, int last,
                         int64_t* colptr, cudaStream_t s);

// --- inner-dimension split and binary merge (mcl_split.cu) ---
constexpr int MCL_SPLIT_MAX_PARTS = 32;  // partial products merged at once
struct RankArgs {
    CscView A;              // stage mode: the matrix
    int32_t k0, k1;         // stage mode: the block [k0, k1) of the inner index
    int nparts;             // merge mode: the partial products
    const int64_t* pcol[MCL_SPLIT_MAX_PARTS];
    const int32_t* prow[MCL_SPLIT_MAX_PARTS];
    const unsigned long long* pval[MCL_SPLIT_MAX_PARTS];
    int32_t n;
    const double* bsum;     // stage mode: column sums of B (fixed-point scales)
    void* scratch;          // per CTA: 6 * stride 8-byte slots
    int64_t stride;         // >= the longest column of A and >= nparts
    int grid_cap;           // CTAs the scratch holds
    int64_t* nnz_out;       // count mode: entries per output column
    const int64_t* colptr_out;  // fill mode
    int32_t* row_out;
    unsigned long long* val_out;  // fill mode: zeroed before the launch
    DevCounters* ctr;
};
void launch_bsum(const CscView& A, const double* colsum, double* bsum, cudaStream_t s);
void launch_split_count(const RankArgs& a, bool stage, int num_sms, cudaStream_t s);
void launch_split_fill(const RankArgs& a, bool stage, int num_sms, cudaStream_t s);
void launch_prune_fixed(int32_t n, const int64_t* colptr, const int32_t* rowidx,
                        const unsigned long long* q, const double* bsum, const PruneParams& pp,
                        const ExpandBuffers& b, int num_sms, cudaStream_t s);

// --- estimator (mcl_estimator.cu) ---
void launch_colmax_features(const CscView& A, int32_t iteration, const float* prev_logcf,
                            float* colmax, float* feats, cudaStream_t s,
                            const int32_t* iter_dev = nullptr);
void launch_iter_bump(int32_t* it, cudaStream_t s);
void launch_mlp_forward(const float* feats, int64_t n, const uint16_t* wbits, const float* norm,
                        float* out, int64_t* est, float safety, const int64_t* flops,
                        const int32_t* rlo, const int32_t* rhi, cudaStream_t s);
void launch_mlp_backward(const float* feats, const float* targets, int64_t n,
                         const uint16_t* wbits, const float* norm, float scale, float* grad,
                         double* loss, cudaStream_t s);
void launch_adam(float* master, float* m, float* v, const float* grad, int64_t step, float lr,
                 float b1, float b2, float eps, uint16_t* wbits, cudaStream_t s);
void launch_logcf(int32_t n, const int64_t* flops, const int64_t* bnnz, float* logcf,
                  cudaStream_t s);

// --- Cohen's estimator (mcl_cohen.cu) ---
int cohen_max_r();
void launch_cohen(const CscView& A, int r, uint64_t seed, float* m, float* est, cudaStream_t s);
void launch_cohen_to_est(int32_t n, const float* e, float safety, const ExpandBuffers& b,
                         cudaStream_t s);

// --- components (mcl_cc.cu) ---
void launch_components(const CscView& A, int32_t* labels, DevCounters* ctr, cudaStream_t s);

}  // namespace mcl
