// Device building blocks shared by the MCL kernels (sm_103a).
//
// Ranking keys: an entry (row i, value v >= 0) of a column is packed as
//     key = (bits(v) << 32) | (0x7FFFFFFF - i)
// so that key order (descending) is value descending, then row ascending --
// the order in which the prune rule ranks a column (Alg. 1, Prune; equal
// values keep the smaller row).  For v >= 0 the IEEE bit pattern is
// monotone in v.  Keys of distinct rows are distinct, and every key is >= 1.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcl {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t EMPTY_SLOT = 0x00000000FFFFFFFFull;  // key -1, value +0.0f

__device__ __forceinline__ uint64_t make_key(float v, int row) {
    return ((uint64_t)__float_as_uint(v) << 32) | (uint32_t)(0x7FFFFFFF - row);
}
__device__ __forceinline__ int key_row(uint64_t k) { return 0x7FFFFFFF - (int)(uint32_t)k; }
__device__ __forceinline__ float key_val(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}
template <typename V>
__device__ __forceinline__ V warp_max(V x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V y = __shfl_xor_sync(FULL, x, o);
        x = y > x ? y : x;
    }
    return x;
}
template <typename V>
__device__ __forceinline__ V warp_min(V x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V y = __shfl_xor_sync(FULL, x, o);
        x = y < x ? y : x;
    }
    return x;
}

// Scratch the block-level helpers use (lives in shared memory).
struct BlockScratch {
    double d[4][33];
    long long q[4][33];
    uint64_t sel_prefix;
    int sel_need;
    int sel_done;
    double sel_target;
    int sel_found;
    int sel_above;
    int cnt;
    int pad;
};

// Sums of up to four doubles and four integers over the block (two barriers).
template <int T>
__device__ __forceinline__ void block_sum(double* dv, int nd, long long* qv, int nq,
                                          BlockScratch* bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = T / 32;
    for (int a = 0; a < nd; ++a) {
        double x = warp_sum(dv[a]);
        if (lane == 0) bs->d[a][warp] = x;
    }
    for (int a = 0; a < nq; ++a) {
        long long x = warp_sum(qv[a]);
        if (lane == 0) bs->q[a][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        for (int a = 0; a < nd; ++a) {
            double x = lane < NW ? bs->d[a][lane] : 0.0;
            x = warp_sum(x);
            if (lane == 0) bs->d[a][32] = x;
        }
        for (int a = 0; a < nq; ++a) {
            long long x = lane < NW ? bs->q[a][lane] : 0ll;
            x = warp_sum(x);
            if (lane == 0) bs->q[a][32] = x;
        }
    }
    __syncthreads();
    for (int a = 0; a < nd; ++a) dv[a] = bs->d[a][32];
    for (int a = 0; a < nq; ++a) qv[a] = bs->q[a][32];
}

template <int T>
__device__ __forceinline__ double block_max_d(double x, BlockScratch* bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = T / 32;
    x = warp_max(x);
    if (lane == 0) bs->d[3][warp] = x;
    __syncthreads();
    if (warp == 0) {
        double y = lane < NW ? bs->d[3][lane] : -1.0e300;
        y = warp_max(y);
        if (lane == 0) bs->d[3][32] = y;
    }
    __syncthreads();
    return bs->d[3][32];
}

// Element i of the concatenation A[0..na) ++ B[0..nb).
__device__ __forceinline__ uint64_t cat_at(const uint64_t* A, int na, const uint64_t* B, int i) {
    return i < na ? A[i] : B[i - na];
}

// Radix select by count over the distinct keys of A ++ B: returns kappa with
// #{x : x >= kappa} == M exactly (1 <= M <= na + nb).  Most-significant
// byte first; stops as soon as the chosen bucket holds exactly the keys
// still needed, returning its prefix with zero low bits.  Histogram updates
// are aggregated per warp over lanes with the same digit.  With SKIP0, zero
// elements are not keys (empty slots of a table; every key is >= 1) and M
// counts nonzero keys only.
template <int T, bool SKIP0 = false>
__device__ uint64_t block_select_count(const uint64_t* A, int na, const uint64_t* B, int nb, int M,
                                       unsigned* hist, BlockScratch* bs) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tot = na + nb;
    uint64_t prefix = 0;
    int need = M;
    for (int shift = 56; shift >= 0; shift -= 8) {
        const uint64_t hmask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
        for (int i = tid; i < 256; i += T) hist[i] = 0u;
        __syncthreads();
        for (int base = 0; base < tot; base += T) {
            const int i = base + tid;
            const bool valid = i < tot;
            const uint64_t x = valid ? cat_at(A, na, B, i) : 0ull;
            const bool in = valid && (!SKIP0 || x != 0ull) && (x & hmask) == prefix;
            const unsigned act = __ballot_sync(FULL, in);
            if (in) {
                const unsigned dg = (unsigned)((x >> shift) & 255u);
                const unsigned grp = __match_any_sync(act, dg);
                if (__ffs(grp) - 1 == lane) atomicAdd(&hist[dg], (unsigned)__popc(grp));
            }
        }
        __syncthreads();
        if (warp == 0) {
            // lane l owns buckets 255-8l ... 248-8l, scanned from the top
            int c[8];
            int lsum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = (int)hist[255 - 8 * lane - q];
                lsum += c[q];
            }
            int incl = lsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            int before = incl - lsum;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (before < need && before + c[q] >= need) {
                    int d = 255 - 8 * lane - q;
                    bs->sel_prefix = prefix | ((uint64_t)d << shift);
                    bs->sel_need = need - before;
                    bs->sel_done = (c[q] == need - before);
                }
                before += c[q];
            }
        }
        __syncthreads();
        prefix = bs->sel_prefix;
        need = bs->sel_need;
        if (bs->sel_done) break;
    }
    __syncthreads();
    return prefix;
}

// Radix select by mass over the distinct keys of A[0..na): the smallest m
// such that the m largest keys carry value mass >= target (target > 0).
// Returns 1 and sets *kappa (a lower bound whose >= set is exactly those m
// keys) and *m; returns 0 if the total mass is below target.  Masses are
// summed in 64-bit fixed point scaled by a power of two that keeps every
// value below 2^50 (exact integer sums, no floating-point atomics); the
// truncation error of a cumulative mass is below na * 2^-50 * max value.
template <int T>
__device__ int block_select_mass(const uint64_t* A, int na, double target, uint64_t* kappa,
                                 int* m, unsigned* hist, unsigned long long* mhist,
                                 BlockScratch* bs) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // largest key = largest value
    uint64_t kmax = 0;
    for (int i = tid; i < na; i += T) kmax = A[i] > kmax ? A[i] : kmax;
    kmax = warp_max(kmax);
    if (lane == 0) bs->q[3][warp] = (long long)kmax;
    __syncthreads();
    if (warp == 0) {
        uint64_t y = lane < T / 32 ? (uint64_t)bs->q[3][lane] : 0ull;
        y = warp_max(y);
        if (lane == 0) bs->q[3][32] = (long long)y;
    }
    __syncthreads();
    const float maxv = key_val((uint64_t)bs->q[3][32]);
    int e = 0;
    frexpf(maxv > 0.0f ? maxv : 1.0f, &e);  // maxv < 2^e
    const int sh50 = 50 - e;                // v * 2^sh50 < 2^50 is exact in FP32
    const double tf = ceil(ldexp(target, sh50));
    if (!(tf < 9.0e18)) {  // beyond any reachable sum
        __syncthreads();
        return 0;
    }
    unsigned long long need = (unsigned long long)tf;
    uint64_t prefix = 0;
    int above = 0;
    int found = 1;
    for (int shift = 56; shift >= 0; shift -= 8) {
        const uint64_t hmask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
        for (int i = tid; i < 256; i += T) {
            hist[i] = 0u;
            mhist[i] = 0ull;
        }
        __syncthreads();
        for (int base = 0; base < na; base += T) {
            const int i = base + tid;
            const bool valid = i < na;
            const uint64_t x = valid ? A[i] : 0ull;
            const bool in = valid && (x & hmask) == prefix;
            const unsigned act = __ballot_sync(FULL, in);
            if (in) {
                const unsigned dg = (unsigned)((x >> shift) & 255u);
                const unsigned grp = __match_any_sync(act, dg);
                // group sum of the fixed-point masses (< 2^50 each) as two
                // 25-bit halves, each summed exactly in 32 bits
                const unsigned long long fx = __float2ull_rz(ldexpf(key_val(x), sh50));
                const unsigned lo25 = __reduce_add_sync(grp, (unsigned)(fx & 0x1FFFFFFull));
                const unsigned hi25 = __reduce_add_sync(grp, (unsigned)(fx >> 25));
                if (__ffs(grp) - 1 == lane) {
                    atomicAdd(&hist[dg], (unsigned)__popc(grp));
                    atomicAdd(&mhist[dg], ((unsigned long long)hi25 << 25) + lo25);
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            int c[8];
            unsigned long long mm[8];
            unsigned long long lsum = 0;
            int lcnt = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = (int)hist[255 - 8 * lane - q];
                mm[q] = mhist[255 - 8 * lane - q];
                lsum += mm[q];
                lcnt += c[q];
            }
            unsigned long long incl = lsum;
            int inclc = lcnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(FULL, incl, o);
                int yc = __shfl_up_sync(FULL, inclc, o);
                if (lane >= o) {
                    incl += y;
                    inclc += yc;
                }
            }
            unsigned long long before = incl - lsum;
            int beforec = inclc - lcnt;
            int hitq = -1;
            unsigned long long hb = 0;
            int hbc = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (hitq < 0) {
                    if (c[q] > 0 && before + mm[q] >= need) {
                        hitq = q;
                        hb = before;
                        hbc = beforec;
                    } else {
                        before += mm[q];
                        beforec += c[q];
                    }
                }
            }
            unsigned hm = __ballot_sync(FULL, hitq >= 0);
            if (hm == 0u) {
                if (lane == 0) bs->sel_found = 0;
            } else if (lane == __ffs(hm) - 1) {
                int d = 255 - 8 * lane - hitq;
                bs->sel_prefix = prefix | ((uint64_t)d << shift);
                bs->sel_target = (double)(need - hb);
                bs->sel_above = above + hbc;
                bs->sel_need = c[hitq];
                bs->sel_found = 1;
                bs->q[2][32] = (long long)(need - hb);
            }
        }
        __syncthreads();
        if (!bs->sel_found) {
            found = 0;
            break;
        }
        prefix = bs->sel_prefix;
        need = (unsigned long long)bs->q[2][32];
        above = bs->sel_above;
        if (bs->sel_need == 1) break;  // one key left in the bucket: the crossing key
    }
    __syncthreads();
    if (found) {
        *kappa = prefix;
        *m = above + 1;
    }
    return found;
}

// Ascending sort of s[0..n) by the block (any n >= 0): the bitonic network
// in its all-ascending form (each merge of two sorted runs starts with a
// reversed compare, i <-> i ^ (k - 1), followed by half-cleaners).  Every
// comparator puts the smaller key at the lower index, so positions >= n act
// as +infinity and are simply skipped.  Ends with a barrier.
template <int T>
__device__ void block_sort_asc(uint64_t* s, int n) {
    int P = 1, lg = 0;
    while (P < n) {
        P <<= 1;
        ++lg;
    }
    for (int lk = 1; lk <= lg; ++lk) {
        const int k = 1 << lk, hk = k >> 1;
        for (int t = threadIdx.x; t < (P >> 1); t += T) {
            const int blk = t >> (lk - 1), off = t & (hk - 1);
            const int i = blk * k + off, j = blk * k + (k - 1 - off);
            if (j < n) {
                const uint64_t x = s[i], y = s[j];
                if (x > y) {
                    s[i] = y;
                    s[j] = x;
                }
            }
        }
        __syncthreads();
        for (int lj = lk - 2; lj >= 0; --lj) {
            const int jj = 1 << lj;
            for (int t = threadIdx.x; t < (P >> 1); t += T) {
                const int i = ((t >> lj) << (lj + 1)) + (t & (jj - 1)), j = i + jj;
                if (j < n) {
                    const uint64_t x = s[i], y = s[j];
                    if (x > y) {
                        s[i] = y;
                        s[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Fixed-point scale of a column: q = trunc(v * 2^f) with 2^f = sc1 * sc2
// (two exact power-of-two factors, each representable in FP32).
struct FixScale {
    float sc1, sc2, is1, is2;
    int f;
    __device__ static float pow2(int e) { return __int_as_float((e + 127) << 23); }
    __device__ void init(double s) {
        int e = 0;
        frexp(s > 0.0 ? s * (1.0 + 1.0 / 1048576.0) : 1.0, &e);  // s (with margin) < 2^e
        f = 62 - e;
        const int f1 = max(-126, min(127, f)), f2 = max(-126, min(127, f - f1));
        sc1 = pow2(f1);
        sc2 = pow2(f2);
        is1 = pow2(-f1);
        is2 = pow2(-f2);
    }
    __device__ __forceinline__ unsigned long long q(float aik, float akj) const {
        const float v = __fmul_rn(aik, akj);  // the FP32 product
        return __float2ull_rz(__fmul_rn(__fmul_rn(v, sc1), sc2));
    }
    __device__ __forceinline__ unsigned long long qv(float v) const {  // v: an FP32 product
        return __float2ull_rz(__fmul_rn(__fmul_rn(v, sc1), sc2));
    }
    __device__ __forceinline__ float value(unsigned long long x) const {
        return __fmul_rn(__fmul_rn(__ull2float_rn(x), is1), is2);
    }
};

// Inflation (Alg. 1, Hadamard power r) of one FP32 value.
__device__ __forceinline__ float inflate_value(float v, float r) {
    if (r == 2.0f) return v * v;
    if (r == 1.0f) return v;
    return powf(v, r);
}

__host__ __device__ __forceinline__ int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace mcl
