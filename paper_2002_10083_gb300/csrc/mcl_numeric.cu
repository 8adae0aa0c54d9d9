// The fused numeric pass of one MCL iteration (Algorithm 1: expansion,
// Prune, inflation) with a shared-memory accumulator of exact fixed-point
// sums.
//
// One CTA owns one output column j at a time (persistent grid, work list in
// longest-first order).  Products a_ik * a_kj are formed in FP32 and added
// as 64-bit integers: each product is scaled by 2^f_j, where 2^(62 - f_j)
// bounds the column sum s_j = sum_k a_kj colsum_k(A) (known before any
// product and bounding every product and every entry, all values being
// >= 0), and truncated.  Integer addition is associative, so an entry of
// B_*j does not depend on the order of its additions, on the window plan or
// on the CTA shape: runs are bit-identical.  The sum is exact up to the
// truncation of each product (below 2^-62 s_j), far below FP32 resolution
// for any entry that can survive the prune.
//
// The column's row span is cut into row windows sized from the output-size
// estimate (about PLAN entries each; windows of at most HS rows give every
// row its own slot, no hashing):
//
//   1. insert:  every product of the window is added into its slot: row - r0
//               in a window of at most HS rows, else linear probing from a
//               multiplicative hash (int32 row keys claimed by
//               compare-and-swap, uint64 sums added with integer atomics);
//   2. extract: over the table, the ranking key (FP32 value bits, row) of
//               every entry replaces its sum in place, with the exact column
//               statistics (count, count and mass at or above the
//               threshold); the keys above the running top-k bound tau go to
//               a candidate buffer that is cut back to the top ksel keys
//               (radix select) when full;
//   3. clear:   the table.
//
// Windows come from per-window product buckets (a counting pass and a
// scatter of (row, FP32 product) into window order) or, without bucket
// space, from per-source cursors over the sorted rows.  A hashed window whose
// probe runs exceed PMAX slots is split by rows and redone (counted as a
// split), and the rest of the column starts at the width that fitted;
// results never depend on the size estimate.  Finally the prune rule picks
// m* (threshold / top-k / recovery), the kept keys are sorted by row,
// inflated, renormalised with an FP64 sum and written with chaos_j.
#include <cfloat>
#include <climits>
#include <cstdint>

#include "mcl_device.cuh"
#include "mcl_internal.h"

namespace mcl {

__device__ __forceinline__ void set_err2(DevCounters* c, unsigned bit) { atomicOr(&c->err, bit); }

struct WinShared {
    BlockScratch bs;
    int wsm[34];
    int item;
    int next;
    // window plan published by thread 0 (rows [pr0, pr1) when prs)
    int pf0, pf1, pr0, pr1, prs, pdone;
    // per-window flags, double-buffered by window parity
    int ovf2[2];   // the window exceeded its table
    int went2[2];  // entries of the window's table
    int next2[2];  // source counter of the warp-per-source insert
    double red;    // result of an ordered sum
};

// Sum of f(s[i]) over i < m in an order that does not depend on the block
// size: warp 0 alone, lane l taking i = l, l + 32, ..., then a fixed
// butterfly; the result is broadcast to the block.  Two barriers.
template <class F>
__device__ __forceinline__ double ordered_sum(const uint64_t* s, int m, F f, double* slot) {
    if (threadIdx.x < 32) {
        double x = 0.0;
        for (int i = threadIdx.x; i < m; i += 32) x += f(s[i]);
        x = warp_sum(x);
        if (threadIdx.x == 0) *slot = x;
    }
    __syncthreads();
    const double r = *slot;
    __syncthreads();
    return r;
}

// Exclusive block scan of one int per thread; *total gets the sum.  Three
// barriers (the last protects the scratch for the next call).
template <int T>
__device__ __forceinline__ int block_scan_excl(int x, int* total, int* wsm) {
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsm[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < NW ? wsm[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) wsm[lane] = wi - w;
        if (lane == 31) wsm[32] = wi;
    }
    __syncthreads();
    const int res = wsm[warp] + incl - x;
    *total = wsm[32];
    __syncthreads();
    return res;
}

// Stable in-place compaction of a[0..n) keeping keys >= cut; returns the
// new length.  Each thread owns IPT consecutive elements per round; all
// reads of a round precede its writes (the scan's barriers), and outputs
// never land past the round's inputs.
template <int T, int IPT>
__device__ int compact_stable(uint64_t* a, int n, uint64_t cut, int* wsm) {
    int outpos = 0;
    for (int base = 0; base < n; base += T * IPT) {
        uint64_t x[IPT];
        int c = 0;
        const int i0 = base + threadIdx.x * IPT;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int i = i0 + q;
            x[q] = i < n ? a[i] : 0ull;
            if (i < n && x[q] >= cut) ++c;
        }
        int tot;
        int o = outpos + block_scan_excl<T>(c, &tot, wsm);
#pragma unroll
        for (int q = 0; q < IPT; ++q)
            if (i0 + q < n && x[q] >= cut) a[o++] = x[q];
        outpos += tot;
        __syncthreads();
    }
    return outpos;
}

// Scratch per CTA in global memory (stride = cur_stride sources): source
// column start (int64), length, two cursor arrays (read / write; swapped
// after a window succeeds) and a_kj.
struct SrcMeta {
    int64_t* ks;
    int32_t* len;
    int32_t* cur;
    int32_t* nxt;
    float* akj;
    __device__ SrcMeta(int32_t* base, int64_t stride) {
        ks = reinterpret_cast<int64_t*>(base);
        len = base + 2 * stride;
        cur = len + stride;
        nxt = cur + stride;
        akj = reinterpret_cast<float*>(nxt + stride);
    }
};

// Stable LSD radix sort of s[0..n) ascending by the field s[i] >> 32, whose
// values are below 2^bits, eight bits per pass.  Warp w owns a contiguous
// segment; per pass each warp counts its digits (whist[w][digit]), one block
// scan over (digit, warp) turns the counts into start offsets, and each warp
// scatters its segment in order (equal digits of a 32-element chunk are
// ranked by lane), so the sort is stable.  tmp holds n elements; whist holds
// (T / 32) * 256 counters.  Ends with a barrier.
template <int T>
__device__ void block_radix_sort_hi(uint64_t* s, uint64_t* tmp, int n, int bits, unsigned* whist,
                                    int* wsm) {
    constexpr int NW = T / 32;
    constexpr int DPT = T >= 256 ? 1 : 256 / T;  // digits per thread in the offset scan
    static_assert(T >= 256 ? T % 256 == 0 : 256 % T == 0, "digits per thread");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int seg = ((n + NW - 1) / NW + 31) & ~31;
    const int w0 = min(n, warp * seg), w1 = min(n, w0 + seg);
    uint64_t* src = s;
    uint64_t* dst = tmp;
    for (int sh = 0; sh < bits; sh += 8) {
        for (int i = tid; i < NW * 256; i += T) whist[i] = 0u;
        __syncthreads();
        for (int base = w0; base < w1; base += 32) {
            const int i = base + lane;
            const bool v = i < w1;
            const unsigned dg = v ? (unsigned)(src[i] >> (32 + sh)) & 255u : 0u;
            const unsigned act = __ballot_sync(FULL, v);
            if (v) {
                const unsigned grp = __match_any_sync(act, dg);
                if (__ffs(grp) - 1 == lane) whist[warp * 256 + dg] += (unsigned)__popc(grp);
            }
            __syncwarp();
        }
        __syncthreads();
        {
            const bool own = tid * DPT < 256;  // threads beyond the 256 digits scan zeros
            unsigned c[DPT][NW];
            int tot = 0;
#pragma unroll
            for (int q = 0; q < DPT; ++q)
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    c[q][w] = own ? whist[w * 256 + tid * DPT + q] : 0u;
                    tot += (int)c[q][w];
                }
            int total;
            int run = block_scan_excl<T>(tot, &total, wsm);
            if (own) {
#pragma unroll
                for (int q = 0; q < DPT; ++q)
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        whist[w * 256 + tid * DPT + q] = (unsigned)run;
                        run += (int)c[q][w];
                    }
            }
        }
        __syncthreads();
        for (int base = w0; base < w1; base += 32) {
            const int i = base + lane;
            const bool v = i < w1;
            uint64_t x = 0;
            unsigned dg = 0;
            if (v) {
                x = src[i];
                dg = (unsigned)(x >> (32 + sh)) & 255u;
            }
            const unsigned act = __ballot_sync(FULL, v);
            if (v) {
                const unsigned grp = __match_any_sync(act, dg);
                dst[whist[warp * 256 + dg] + __popc(grp & lanemask_lt())] = x;
                __syncwarp(act);
                if (__ffs(grp) - 1 == lane) whist[warp * 256 + dg] += (unsigned)__popc(grp);
            }
            __syncwarp();
        }
        __syncthreads();
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    if (src != s) {
        for (int i = tid; i < n; i += T) s[i] = src[i];
        __syncthreads();
    }
}

// Value mass of the keys >= cut in a[0..n), as an exact integer sum of the
// values in fixed point (each truncated at 2^-50 of the largest value), so
// that it does not depend on the order of a's elements.  Warp 0 sums; the
// result is broadcast to the block.
template <int T>
__device__ double mass_at_or_above(const uint64_t* a, int n, uint64_t cut, WinShared* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t kmax = 0;
    for (int i = threadIdx.x; i < n; i += T) kmax = a[i] > kmax ? a[i] : kmax;
    kmax = warp_max(kmax);
    if (lane == 0) sh->bs.q[3][warp] = (long long)kmax;
    __syncthreads();
    if (warp == 0) {
        uint64_t y = lane < T / 32 ? (uint64_t)sh->bs.q[3][lane] : 0ull;
        y = warp_max(y);
        const float maxv = key_val(y);
        int e = 0;
        frexpf(maxv > 0.0f ? maxv : 1.0f, &e);  // every value < 2^e
        const int s50 = 50 - e;
        unsigned long long acc = 0;
        for (int i = lane; i < n; i += 32)
            if (a[i] >= cut) acc += __float2ull_rz(ldexpf(key_val(a[i]), s50));
        acc = warp_sum(acc);
        if (lane == 0) sh->red = ldexp((double)acc, -s50);
    }
    __syncthreads();
    const double r = sh->red;
    __syncthreads();
    return r;
}

// Finish a column: prune rule on the candidate keys top[0..ntop) plus exact
// statistics, then the kept keys in row order (sorted here unless the
// buffer is already row-ordered) written with inflation (pp.inflate) or
// their B values; returns m* and chaos_j via the pointers.
// For an unordered buffer, rows lie in [row_lo, row_lo + row_span); the
// radix sort uses top[m .. topcap) and rscratch ((T / 32) * 256 counters)
// as scratch when they suffice, the bitonic network otherwise.
template <int T, int IPT, bool ROW_ORDERED>
__device__ void finish_column(uint64_t* top, int ntop, int topcap, const PruneParams& pp, double S,
                              double MT, long long Tt, int64_t cap, int32_t* out_row,
                              float* out_val, unsigned* hist, unsigned long long* mhist,
                              WinShared* sh, DevCounters* ctr, int row_lo, int row_span,
                              unsigned* rscratch, int* mstar_out, double* chaos_out) {
    const int tid = threadIdx.x;
    const double target = (double)pp.p * S;
    const int q = (int)(Tt < (long long)pp.K ? Tt : (long long)pp.K);
    double mq = 0.0;
    uint64_t kq = 0;
    // q >= Krec: m* = min(Krec, max(q, m_rec)) = Krec whatever the recovery
    // finds, so neither the top-q mass nor m_rec is needed
    const bool krec_bound = q >= pp.Krec;
    if (krec_bound) {
    } else if (Tt <= pp.K) {
        mq = MT;
    } else {
        kq = block_select_count<T>(top, ntop, top, 0, pp.K, hist, &sh->bs);
        mq = mass_at_or_above<T>(top, ntop, kq, sh);
    }
    int mstar;
    uint64_t cut;
    bool have_cut = false;
    if (krec_bound) {
        mstar = pp.Krec;
    } else if (target <= 0.0 || mq >= target) {
        mstar = q;
        if (mstar <= pp.Krec) {
            if (Tt <= pp.K) {
                cut = (uint64_t)__float_as_uint(pp.theta) << 32;  // exactly the entries >= theta
            } else {
                cut = kq;
            }
            have_cut = true;
        }
    } else {
        uint64_t kr = 0;
        int mr = 0;
        const int f = block_select_mass<T>(top, ntop, target, &kr, &mr, hist, mhist, &sh->bs);
        mstar = f ? mr : ntop;
        if (f && mstar <= pp.Krec) {
            cut = kr;
            have_cut = true;
        }
    }
    if (mstar > pp.Krec) mstar = pp.Krec;
    if (mstar > ntop) mstar = ntop;
    if ((int64_t)mstar > cap) {  // cannot happen for validated input; never write past cap
        if (tid == 0) set_err2(ctr, ERR_INTERNAL);
        mstar = (int)cap;
        have_cut = false;
    }
    if (!have_cut || mstar == 0) {
        if (mstar == 0)
            cut = ~0ull;
        else if (mstar >= ntop)
            cut = 0ull;
        else
            cut = block_select_count<T>(top, ntop, top, 0, mstar, hist, &sh->bs);
    }
    // the kept keys (exactly m* of them: keys are distinct) to the front
    int m = mstar > 0 ? compact_stable<T, IPT>(top, ntop, cut, sh->wsm) : 0;
    if (m != mstar) {
        if (tid == 0) set_err2(ctr, ERR_INTERNAL);
        m = m < mstar ? m : mstar;
    }
    if (!ROW_ORDERED && m > 1) {
        // re-key as (row - row_lo, value bits) and sort ascending: rows are distinct
        for (int i = tid; i < m; i += T) {
            const uint64_t x = top[i];
            top[i] = ((uint64_t)(uint32_t)(key_row(x) - row_lo) << 32) | (x >> 32);
        }
        __syncthreads();
        if (rscratch != nullptr && topcap - m >= m) {
            const int bits = 32 - __clz(row_span - 1);
            block_radix_sort_hi<T>(top, top + m, m, bits, rscratch, sh->wsm);
        } else {
            block_sort_asc<T>(top, m);
        }
        for (int i = tid; i < m; i += T) {
            const uint64_t x = top[i];
            top[i] = make_key(__uint_as_float((uint32_t)x), (int)(x >> 32) + row_lo);
        }
        __syncthreads();
    }
    const float rr = pp.r;
    const double U = pp.inflate ? ordered_sum(top, m, [rr](uint64_t x) {
        return (double)inflate_value(key_val(x), rr); }, &sh->red) : 0.0;
    const double invU = U > 0.0 ? 1.0 / U : 0.0;
    double amax = 0.0;
    for (int i = tid; i < m; i += T) {
        const uint64_t x = top[i];
        const float v = key_val(x);
        float outv = v;
        if (pp.inflate) {
            const double a = (double)inflate_value(v, pp.r) * invU;
            outv = (float)a;
            amax = a > amax ? a : amax;
        }
        out_row[i] = key_row(x);
        out_val[i] = outv;
    }
    double ch = 0.0;
    if (pp.inflate) {
        const double mx = block_max_d<T>(amax, &sh->bs);
        const double sq = ordered_sum(top, m, [rr, invU](uint64_t x) {
            const double a = (double)inflate_value(key_val(x), rr) * invU;
            return a * a; }, &sh->red);
        ch = mx - sq;
        if (ch < 0.0) ch = 0.0;
    }
    if (tid == 0) {
        *mstar_out = m;
        *chaos_out = ch;
    }
    __syncthreads();
}

// Append the candidates an enumerator yields to top[0..ntop); first cuts
// the buffer back to ksel entries if they would not fit.  `count(tau)`
// returns this thread's number of keys > tau; `emit(tau, dst, base)` writes
// this thread's keys at dst[base ...] (base: its exclusive scan offset).
template <int T, int IPT, class Enum>
__device__ __forceinline__ void append_candidates(Enum& en, uint64_t* top, int topcap, int ksel,
                                                  int& ntop, uint64_t& tau, int c, unsigned* hist,
                                                  WinShared* sh) {
    int C;
    int base = block_scan_excl<T>(c, &C, sh->wsm);
    if (ntop + C > topcap) {
        // invariant: C <= window capacity = topcap - ksel, so ntop > ksel here
        const uint64_t kap = block_select_count<T>(top, ntop, top, 0, ksel, hist, &sh->bs);
        ntop = compact_stable<T, IPT>(top, ntop, kap, sh->wsm);
        tau = kap;
        c = en.count(tau);
        base = block_scan_excl<T>(c, &C, sh->wsm);
    }
    en.emit(tau, top + ntop, base);
    ntop += C;
    __syncthreads();
}


// ---------------------------------------------------------------------------
// the accumulator: int32 row keys and uint64 fixed-point sums per slot
// ---------------------------------------------------------------------------

constexpr int KEY_EMPTY = -1;
constexpr int PMAX = 64;  // probe run that marks a hashed window as overflowed

__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.shared.add.u64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "l"(v)
                 : "memory");
}

__device__ __forceinline__ int cas_shared(int* p, int cmp, int val) {
    int old;
    asm volatile("atom.shared.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old)
                 : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(cmp), "r"(val)
                 : "memory");
    return old;
}

// Exact unsigned 32-bit division by a run-time constant d >= 1 with one
// multiply-high (the round-up method of Granlund and Montgomery, 1994):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((x - t) >> 1)) >> (l - 1) with t = mulhi(m, x); d = 1 is x.
struct FastDiv {
    uint32_t m;
    int l;
    __device__ void init(uint32_t d) {
        l = 0;
        while ((1ull << l) < d) ++l;
        m = l == 0 ? 0u : (uint32_t)((((1ull << l) - d) << 32) / d + 1ull);
    }
    __device__ __forceinline__ uint32_t div(uint32_t x) const {
        if (l == 0) return x;
        const uint32_t t = __umulhi(m, x);
        return (t + ((x - t) >> 1)) >> (l - 1);
    }
};

// Home slot of a row in a hashed window: multiplicative hash scaled to HS
// slots (any HS).
template <int HS>
__device__ __forceinline__ int table_home(int row) {
    return (int)(((uint64_t)((uint32_t)row * 0x9E3779B1u) * (uint64_t)HS) >> 32);
}

// Add q at `row`: slot row - r0 in an identity window (rows of the window
// span at most HS slots; every writer of a slot stores the same row), else
// linear probing from the row's hash, an empty slot claimed by
// compare-and-swap.  A probe run of PMAX slots sets *ovf and adds nothing.
template <int HS, bool IDENT>
__device__ __forceinline__ void acc_add(int row, unsigned long long q, int r0, int* keys,
                                        unsigned long long* vals, int* ovf) {
    if (IDENT) {
        const unsigned h = (unsigned)(row - r0);
        if (h >= (unsigned)HS) {  // cannot happen: a window's segments hold rows in [r0, r1)
            *ovf = 2;
            return;
        }
        keys[h] = row;
        red_add_u64(vals + h, q);
        return;
    }
    int h = table_home<HS>(row);
    for (int p = 0; p < PMAX; ++p) {
        int k = *reinterpret_cast<volatile int*>(keys + h);
        if (k == KEY_EMPTY) {
            k = cas_shared(keys + h, KEY_EMPTY, row);
            if (k == KEY_EMPTY) k = row;
        }
        if (k == row) {
            red_add_u64(vals + h, q);
            return;
        }
        if (++h == HS) h = 0;
    }
    *ovf = 1;
}

// Expected entries per source and window below which a window walks its
// sources one per lane instead of one per warp.
constexpr int LANE_MODE_MAX = 12;

// The ranking keys of a window's table after extraction (0: empty slot;
// thread t takes slots t, t + T, ...).
template <int T, int HS>
struct KeyEnum {
    const uint64_t* vk;
    __device__ int count(uint64_t tau) const {
        int c = 0;
        for (int h = threadIdx.x; h < HS; h += T) c += vk[h] > tau;
        return c;
    }
    __device__ void emit(uint64_t tau, uint64_t* dst, int base) const {
        for (int h = threadIdx.x; h < HS; h += T) {
            const uint64_t k = vk[h];
            if (k > tau) dst[base++] = k;
        }
    }
};

struct ExpandArgs {
    CscView A;
    PruneParams pp;
    ExpandBuffers b;
    int conf;
    int plan;
};

template <int T, int HS>
struct ExpandLayout {
    static constexpr size_t bytes(int ksel) {
        return (size_t)HS * 12 + (size_t)(ksel + HS) * 8 + 256 * 4 + 256 * 8 + sizeof(WinShared);
    }
};

template <int T, int HS, int MINB>
__global__ void __launch_bounds__(T, MINB) k_expand(ExpandArgs a) {
    const int PLAN = a.plan;  // distinct rows a window is planned for
    constexpr int IPT = 8;
    static_assert(HS >= (T / 32) * 256, "the row sort's counters fit in the key array");
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* vals = reinterpret_cast<unsigned long long*>(smem);
    int* keys = reinterpret_cast<int*>(vals + HS);
    uint64_t* vkeys = reinterpret_cast<uint64_t*>(vals);  // ranking keys after extraction
    uint64_t* top = reinterpret_cast<uint64_t*>(keys + HS);
    const int ksel = a.pp.ksel;
    const int topcap = ksel + HS;  // a window adds at most HS candidates
    unsigned* hist = reinterpret_cast<unsigned*>(top + topcap);
    unsigned long long* mhist = reinterpret_cast<unsigned long long*>(hist + 256);
    WinShared* sh = reinterpret_cast<WinShared*>(mhist + 256);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const CscView& A = a.A;
    const ExpandBuffers& b = a.b;
    DevCounters* ctr = b.ctr;
    SrcMeta meta(b.cursors + (int64_t)blockIdx.x * 6 * b.cur_stride, b.cur_stride);
    // per-CTA bucket of (row, bits(product)) pairs
    int2* bkt = b.bucket_row ? reinterpret_cast<int2*>(b.bucket_row) + (int64_t)blockIdx.x * b.bucket_cap
                             : nullptr;
    // window starts and ends in the bucket (per CTA: WINDOW_MAX + 1 of each)
    int32_t* woff = b.woff ? b.woff + (int64_t)blockIdx.x * 2 * (WINDOW_MAX + 1) : nullptr;
    int32_t* wlim = woff ? woff + (WINDOW_MAX + 1) : nullptr;
    const int wbeg = ctr->bin_off[a.conf * NZ], wend = ctr->bin_off[a.conf * NZ + NZ];
    if (ctr->err & ERR_STAGING) return;  // the iteration is redone without the graph

    for (int i = tid; i < HS; i += T) {
        keys[i] = KEY_EMPTY;
        vals[i] = 0ull;
    }
    const float theta = a.pp.theta;
    for (;;) {
        if (tid == 0) sh->item = atomicAdd(&ctr->conf_ctr[a.conf], 1);
        __syncthreads();
        const int item = sh->item;
        __syncthreads();
        if (wbeg + item >= wend) break;
        const int j = b.work[wbeg + item];
        const int64_t cb = A.colptr[j], ce = A.colptr[j + 1];
        const int d = (int)(ce - cb);
        const int lo = b.rlo[j], hiE = b.rhi[j] + 1;
        if (d == 0 || hiE <= lo) {
            if (tid == 0) {
                b.kept[j] = 0;
                b.chaos[j] = 0.0;
                b.bnnz[j] = 0;
            }
            continue;
        }
        if (d > b.cur_stride) {
            if (tid == 0) {
                set_err2(ctr, ERR_CURSOR);
                b.kept[j] = 0;
                b.chaos[j] = 0.0;
                b.bnnz[j] = 0;
            }
            continue;
        }
        const int span = hiE - lo;
        const int64_t flops_j = b.flops[j];
        int64_t est = b.est[j];
        if (est < 1) est = 1;
        for (int i = tid; i < d; i += T) {
            const int k = A.rowidx[cb + i];
            const int64_t ks = A.colptr[k];
            const float akj = A.val[cb + i];
            meta.ks[i] = ks;
            meta.len[i] = (int)(A.colptr[k + 1] - ks);
            meta.cur[i] = 0;
            meta.akj[i] = akj;
        }
        // column sum of B_*j from the identity sum_i (AA)_ij = sum_k a_kj sum_i a_ik,
        // FP64 in a fixed order (warp 0, lane-strided, butterfly), independent of T
        if (warp == 0) {
            double s = 0.0;
            for (int i = lane; i < d; i += 32) s += (double)A.val[cb + i] * b.colsum[A.rowidx[cb + i]];
            s = warp_sum(s);
            if (lane == 0) sh->red = s;
        }
        // ---- plan: about est / PLAN windows of equal row width.  With bucket
        // space the products go to per-window buckets, and a window that
        // overflows the table is split by rows (later windows of the column
        // then start at the split width).  Otherwise the window width adapts
        // to the entries seen. ----
        int64_t nw64 = (est + PLAN - 1) / PLAN;
        if (nw64 < 1) nw64 = 1;
        if (nw64 > span) nw64 = span;
        bool bucket = false;
        if (nw64 > 1 && bkt != nullptr && flops_j <= b.bucket_cap) {
            const int64_t wmax = WINDOW_MAX < HS ? WINDOW_MAX : HS;
            if (nw64 > wmax) nw64 = wmax;
            bucket = true;
        }
        int width = (int)(((int64_t)span + nw64 - 1) / nw64);
        if (width < HS && span > width) {
            // a window of at most HS rows has a slot per row (no hashing): use the
            // widest such windows
            const int64_t nid = ((int64_t)span + HS - 1) / HS;
            if (nid < nw64) {
                nw64 = nid;
                width = (int)(((int64_t)span + nw64 - 1) / nw64);
            }
        }
        const int nwin = (int)(((int64_t)span + width - 1) / width);
        int ntop = 0;
        uint64_t tau = 0;
        unsigned long long s_mt = 0;
        long long s_t = 0, s_n = 0;
        FastDiv fdiv;
        fdiv.init((uint32_t)width);
        __syncthreads();
        const double S = sh->red;
        FixScale fx;
        fx.init(S);

        if (bucket) {
            int* wcnt = reinterpret_cast<int*>(vals);  // nwin <= HS counters each
            int* wcur = wcnt + HS;
            // Scatter (row, a_ik * a_kj) into the window buckets from the cursors wcur;
            // with a capacity capw per window (window w owns [w capw, (w + 1) capw))
            // a run that would pass its window's end sets sh->next2[1] and writes
            // nothing past it.
            auto scatter = [&](int capw) {
                if (tid == 0) sh->next = 0;
                __syncthreads();
                for (;;) {
                    int kidx = 0;
                    if (lane == 0) kidx = atomicAdd(&sh->next, 1);
                    kidx = __shfl_sync(FULL, kidx, 0);
                    if (kidx >= d) break;
                    const int len = meta.len[kidx];
                    const int64_t ks = meta.ks[kidx];
                    const int32_t* rows = A.rowidx + ks;
                    const float* vv = A.val + ks;
                    const float akj = meta.akj[kidx];
                    // the next 128 products are loaded while this chunk is routed
                    int rr[4];
                    float pv[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int p = 32 * c + lane;
                        rr[c] = p < len ? __ldg(rows + p) : 0;
                        pv[c] = p < len ? __ldg(vv + p) : 0.0f;
                    }
                    for (int pb = 0; pb < len; pb += 128) {
                        int nr[4];
                        float nv[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int p = pb + 128 + 32 * c + lane;
                            nr[c] = p < len ? __ldg(rows + p) : 0;
                            nv[c] = p < len ? __ldg(vv + p) : 0.0f;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const bool v = pb + 32 * c + lane < len;
                            const unsigned act = __ballot_sync(FULL, v);  // a prefix of the lanes
                            if (act == 0u) break;
                            const int row = rr[c];
                            const uint32_t w = v ? fdiv.div((uint32_t)(row - lo)) : 0xFFFFFFFFu;
                            const uint32_t wp = __shfl_up_sync(FULL, w, 1);
                            const bool head = v && (lane == 0 || wp != w);
                            const unsigned heads = __ballot_sync(FULL, head);
                            int base = 0;
                            if (head) {
                                const unsigned after = heads & ~((2u << lane) - 1u);
                                const int end = after ? __ffs(after) - 1 : __popc(act);
                                base = atomicAdd(wcur + w, end - lane);
                                if (capw > 0 && base + (end - lane) > ((int)w + 1) * capw)
                                    sh->next2[1] = 1;
                            }
                            // the head of this lane's run: the highest head at or below it
                            const int hl = 31 - __clz(heads & ((2u << lane) - 1u));
                            base = __shfl_sync(FULL, base, hl);
                            if (v) {
                                const int pos = base + lane - hl;
                                if (capw == 0 || pos < ((int)w + 1) * capw)
                                    bkt[pos] = make_int2(row, __float_as_int(pv[c] * akj));
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            rr[c] = nr[c];
                            pv[c] = nv[c];
                        }
                    }
                }
                __syncthreads();
            };
            // products per window of equal row width are near their mean for
            // rows spread over the span: try fixed capacities of twice the mean
            // share first (1.25x left 13.5k of the 1M-vertex graph's columns to
            // the counting pass, 2x 1.6k)
            const int64_t capw64 = ((flops_j + nwin - 1) / nwin) * 2 + 64;
            bool counted = true;
            if (capw64 * nwin <= b.bucket_cap) {
                const int capw = (int)capw64;
                for (int i = tid; i < nwin; i += T) wcur[i] = i * capw;
                if (tid == 0) sh->next2[1] = 0;
                __syncthreads();
                scatter(capw);
                counted = sh->next2[1] != 0;  // a window was fuller than its capacity
                if (!counted)
                    for (int i = tid; i < nwin; i += T) {
                        woff[i] = i * capw;
                        wlim[i] = wcur[i];
                    }
                __syncthreads();
            }
            if (counted) {
                // ---- count the products of every window ----
                for (int i = tid; i < nwin; i += T) wcnt[i] = 0;
                if (tid == 0) sh->next = 0;
                __syncthreads();
                for (;;) {
                    int kidx = 0;
                    if (lane == 0) kidx = atomicAdd(&sh->next, 1);
                    kidx = __shfl_sync(FULL, kidx, 0);
                    if (kidx >= d) break;
                    const int len = meta.len[kidx];
                    const int32_t* rows = A.rowidx + meta.ks[kidx];
                    for (int pb = 0; pb < len; pb += 128) {
                        int rr[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int p = pb + 32 * c + lane;
                            rr[c] = p < len ? __ldg(rows + p) : 0;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            // rows are sorted, so equal windows form runs of lanes
                            const bool v = pb + 32 * c + lane < len;
                            const unsigned act = __ballot_sync(FULL, v);  // a prefix of the lanes
                            if (act == 0u) break;
                            const uint32_t w = v ? fdiv.div((uint32_t)(rr[c] - lo)) : 0xFFFFFFFFu;
                            const uint32_t wp = __shfl_up_sync(FULL, w, 1);
                            const bool head = v && (lane == 0 || wp != w);
                            const unsigned heads = __ballot_sync(FULL, head);
                            if (head) {
                                const unsigned after = heads & ~((2u << lane) - 1u);
                                const int end = after ? __ffs(after) - 1 : __popc(act);
                                atomicAdd(wcnt + w, end - lane);
                            }
                        }
                    }
                }
                __syncthreads();
                // ---- window offsets (exclusive scan), scatter cursors ----
                {
                    const int per = (nwin + T - 1) / T;
                    const int i0 = min(nwin, tid * per), i1 = min(nwin, i0 + per);
                    int c = 0;
                    for (int i = i0; i < i1; ++i) c += wcnt[i];
                    int tot;
                    int run = block_scan_excl<T>(c, &tot, sh->wsm);
                    for (int i = i0; i < i1; ++i) {
                        woff[i] = run;
                        wcur[i] = run;
                        run += wcnt[i];
                        wlim[i] = run;
                    }
                    if (tid == 0 && (int64_t)tot != flops_j) set_err2(ctr, ERR_INTERNAL);
                }
                __syncthreads();
                scatter(0);
            }
            for (int i = tid; i < HS; i += T) vals[i] = 0ull;
        }

        // ---- windows ----
        // Thread 0 plans every window and publishes it; bucket mode: bucket
        // window f0 = [f0, f1) (rows [r0, r1) of it while it is split);
        // cursor mode: rows [r0, r1).
        int f0 = 0, f1 = 0;
        bool rowsplit = false;
        int split_w = 0;  // > 0: rows per piece when windows are being split
        int r0 = lo, r1 = lo;
        int cwidth = width;  // cursor mode: current window width
        int32_t* cur = meta.cur;
        int32_t* nxt = meta.nxt;
        const bool lane_mode =
            !bucket && (double)flops_j * (double)width < (double)LANE_MODE_MAX * (double)d * (double)span;
        auto plan = [&](int f) {  // thread 0 only
            while (f < nwin && wlim[f] == woff[f]) ++f;  // empty windows
            f0 = f;
            f1 = f;
            rowsplit = false;
            if (f >= nwin) return;
            if (split_w > 0) {
                const int ws = lo + f * width;
                const int we = (int)min((int64_t)ws + width, (int64_t)hiE);
                if (split_w < we - ws) {
                    rowsplit = true;
                    f1 = f + 1;
                    r0 = ws;
                    r1 = ws + split_w;
                    return;
                }
                split_w = 0;
            }
            f1 = f + 1;
        };
        auto publish = [&](int nextpar) {  // thread 0 only
            sh->pf0 = f0;
            sh->pf1 = f1;
            sh->pr0 = r0;
            sh->pr1 = r1;
            sh->prs = rowsplit ? 1 : 0;
            sh->pdone = bucket ? f0 >= nwin : r0 >= hiE;
            sh->ovf2[nextpar] = 0;
            sh->went2[nextpar] = 0;
            sh->next2[nextpar] = 0;
        };
        if (tid == 0) {
            if (bucket)
                plan(0);
            else
                r1 = (int)min((int64_t)lo + cwidth, (int64_t)hiE);
            publish(0);
        }
        for (int it = 0;; ++it) {
            const int par = it & 1;
            __syncthreads();  // this window's plan and flags are published
            if (sh->pdone) break;
            const int F0 = sh->pf0, F1 = sh->pf1, R0 = sh->pr0, R1 = sh->pr1;
            const bool RS = sh->prs != 0;
            int* ovfp = &sh->ovf2[par];
            // rows of this window: a bucket window (or its split piece) or the cursor range;
            // at most HS rows wide, it maps row - wr0 to its slot (no hashing)
            const int wr0 = bucket ? (RS ? R0 : lo + F0 * width) : R0;
            const int wr1 =
                bucket ? (RS ? R1 : (int)min((int64_t)lo + (int64_t)(F0 + 1) * width, (int64_t)hiE))
                       : R1;
            const bool ident = wr1 - wr0 <= HS;
            auto add = [&](int row, unsigned long long q) {
                if (ident)
                    acc_add<HS, true>(row, q, wr0, keys, vals, ovfp);
                else
                    acc_add<HS, false>(row, q, wr0, keys, vals, ovfp);
            };
            // ---- 1. insert the products of the window ----
            if (bucket) {
                const int bs = woff[F0], be = wlim[F0];
                // four products per lane in flight while the previous four update
                // the table (the loads are issued before the shared atomics)
                int2 cx[4];
                int pb = bs + warp * 128;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = pb + 32 * u + lane;
                    cx[u] = p < be ? bkt[p] : make_int2(-1, 0);
                }
                for (; pb < be; pb += T * 4) {
                    int2 nx[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int p = pb + T * 4 + 32 * u + lane;
                        nx[u] = p < be ? bkt[p] : make_int2(-1, 0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int row = cx[u].x;
                        bool valid = row >= 0;
                        if (RS) valid = valid && row >= R0 && row < R1;
                        if (valid) add(row, fx.qv(__int_as_float(cx[u].y)));
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) cx[u] = nx[u];
                }
            } else if (lane_mode) {
                for (int kidx = tid; kidx < d; kidx += T) {
                    const int64_t ks = meta.ks[kidx];
                    const int32_t* rows = A.rowidx + ks;
                    const float* vv = A.val + ks;
                    const float akj = meta.akj[kidx];
                    const int len = meta.len[kidx];
                    int pos = cur[kidx];
                    for (; pos < len; ++pos) {
                        const int row = __ldg(rows + pos);
                        if (row >= R1) break;
                        add(row, fx.q(__ldg(vv + pos), akj));
                    }
                    nxt[kidx] = pos;
                }
            } else {
                for (;;) {
                    int kidx = 0;
                    if (lane == 0) kidx = atomicAdd(&sh->next2[par], 1);
                    kidx = __shfl_sync(FULL, kidx, 0);
                    if (kidx >= d) break;
                    const int64_t ks = meta.ks[kidx];
                    const int32_t* rows = A.rowidx + ks;
                    const float* vv = A.val + ks;
                    const float akj = meta.akj[kidx];
                    const int len = meta.len[kidx];
                    int pos = cur[kidx];
                    while (pos < len) {
                        const int p = pos + lane;
                        const int row = p < len ? __ldg(rows + p) : INT_MAX;
                        const bool valid = row < R1;
                        if (valid) add(row, fx.q(__ldg(vv + p), akj));
                        const int nin = __popc(__ballot_sync(FULL, valid));
                        pos += nin;
                        if (nin < 32) break;
                    }
                    if (lane == 0) nxt[kidx] = pos;
                }
            }
            __syncthreads();
            if (*ovfp) {
                for (int i = tid; i < HS; i += T) {
                    keys[i] = KEY_EMPTY;
                    vals[i] = 0ull;
                }
                if (*ovfp == 2 && tid == 0) set_err2(ctr, ERR_INTERNAL);  // cannot happen
                if (tid == 0) {
                    atomicAdd(&ctr->splits, 1ull);
                    if (bucket && !rowsplit) {
                        // split the window's rows (a single row never overflows)
                        rowsplit = true;
                        r0 = lo + f0 * width;
                        const int we = (int)min((int64_t)r0 + width, (int64_t)hiE);
                        r1 = r0 + (we - r0) / 2;
                    } else {
                        r1 = r0 + (r1 - r0) / 2;
                        cwidth = r1 - r0;
                    }
                    publish(par ^ 1);
                }
                continue;
            }
            // ---- 2. statistics and candidates: every entry becomes its ranking key
            // in place (exact statistics from the fixed-point sums), row keys cleared ----
            KeyEnum<T, HS> en{vkeys};
            int c = 0, cnt = 0;
            for (int h = tid; h < HS; h += T) {
                const int row = keys[h];
                if (row != KEY_EMPTY) {
                    const unsigned long long q = vals[h];
                    const float v = fx.value(q);
                    const uint64_t key = make_key(v, row);
                    ++cnt;
                    if (v >= theta) {
                        ++s_t;
                        s_mt += q;
                    }
                    c += key > tau;
                    vkeys[h] = key;
                    keys[h] = KEY_EMPTY;
                }
            }
            s_n += cnt;
            {
                const int wc = warp_sum(cnt);
                if (lane == 0 && wc) atomicAdd(&sh->went2[par], wc);
            }
            append_candidates<T, IPT>(en, top, topcap, ksel, ntop, tau, c, hist, sh);
            // ---- 3. clear the table ----
            for (int i = tid; i < HS; i += T) vkeys[i] = 0ull;
            if (!bucket) {  // cursors advance past the window
                int32_t* t = cur;
                cur = nxt;
                nxt = t;
            }
            // ---- 4. next window ----
            if (tid == 0) {
                const int went = sh->went2[par];  // complete: append_candidates ends with a barrier
                if (bucket) {
                    if (rowsplit) {
                        const int we =
                            (int)min((int64_t)lo + (int64_t)(f0 + 1) * width, (int64_t)hiE);
                        int wd = r1 - r0;
                        if (went < PLAN / 2 && wd < width) wd *= 2;
                        r0 = r1;
                        if (r0 >= we) {
                            split_w = wd;
                            plan(f0 + 1);
                        } else {
                            r1 = min(we, r0 + wd);
                        }
                    } else {
                        plan(f1);
                    }
                } else {
                    r0 = r1;
                    if (went < PLAN / 2 && cwidth < (1 << 29))
                        cwidth *= 2;
                    else if (went > PLAN + PLAN / 2 && cwidth > 1)
                        cwidth /= 2;
                    r1 = (int)min((int64_t)r0 + cwidth, (int64_t)hiE);
                }
                publish(par ^ 1);
            }
        }
        double dv[1] = {0.0};
        long long qv[3] = {s_t, s_n, (long long)s_mt};
        block_sum<T>(dv, 0, qv, 3, &sh->bs);
        const double MT = ldexp((double)(unsigned long long)qv[2], -fx.f);
        int mstar = 0;
        double ch = 0.0;
        const int64_t obase = b.off[j];
        // the table's key array is free here: radix counters of the row sort
        finish_column<T, IPT, false>(top, ntop, topcap, a.pp, S, MT, qv[0], b.cap[j],
                                     b.tmp_row + (obase - b.tmp_off0),
                                     b.tmp_val + (obase - b.tmp_off0), hist, mhist, sh, ctr, lo,
                                     span, reinterpret_cast<unsigned*>(keys), &mstar, &ch);
        for (int i = tid; i < (T / 32) * 256; i += T) keys[i] = KEY_EMPTY;
        if (tid == 0) {
            b.kept[j] = mstar;
            b.chaos[j] = ch;
            b.bnnz[j] = qv[1];
            if (qv[1] > est) atomicAdd(&ctr->misses, 1ull);
        }
    }
}

// Configurations: 0 = small columns (128 threads, 1024 slots, windows of
// 512 rows, 8 CTAs per SM); 1 = everything else, in one of three shapes
// that the autotuner picks from (threads, table slots, CTAs per SM):
//   table 0: 256 x 2048 x 4,  table 1: 512 x 4096 x 2,  table 2: 256 x 4096 x 2.
// The candidate buffer holds ksel + HS keys (a window adds at most HS).
template <int T_, int HS_, int MINB_>
struct Conf {
    static constexpr int T = T_, HS = HS_, MINB = MINB_;
};
using Conf0 = Conf<128, 1024, 8>;
using Conf1a = Conf<256, 2048, 4>;
using Conf1b = Conf<512, 4096, 2>;
using Conf1c = Conf<256, 4096, 2>;

template <class C>
static size_t conf_smem(int ksel) { return ExpandLayout<C::T, C::HS>::bytes(ksel); }

template <class C>
static int conf_grid(int ksel, int num_sms) {
    const size_t smem = conf_smem<C>(ksel);
    auto kern = k_expand<C::T, C::HS, C::MINB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::T, smem);
    if (occ < 1) occ = 1;
    return occ * num_sms;
}

template <class C>
static void conf_launch(int conf, const CscView& A, const PruneParams& pp, const ExpandBuffers& b,
                        int grid, cudaStream_t s) {
    int plan = conf == 0 ? C::HS / 2 : (pp.plan > 0 ? pp.plan : C::HS / 2);
    if (plan > (3 * C::HS) / 4) plan = (3 * C::HS) / 4;
    if (plan < 64) plan = 64;
    ExpandArgs a{A, pp, b, conf, plan};
    k_expand<C::T, C::HS, C::MINB><<<grid, C::T, conf_smem<C>(pp.ksel), s>>>(a);
}

size_t numeric_smem(int conf, const PruneParams& pp) {
    if (conf == 0) return conf_smem<Conf0>(pp.ksel);
    return pp.table == 1 ? conf_smem<Conf1b>(pp.ksel)
                         : pp.table == 2 ? conf_smem<Conf1c>(pp.ksel) : conf_smem<Conf1a>(pp.ksel);
}

int numeric_grid(int conf, const PruneParams& pp, int num_sms) {
    if (conf == 0) return conf_grid<Conf0>(pp.ksel, num_sms);
    return pp.table == 1 ? conf_grid<Conf1b>(pp.ksel, num_sms)
                         : pp.table == 2 ? conf_grid<Conf1c>(pp.ksel, num_sms)
                                         : conf_grid<Conf1a>(pp.ksel, num_sms);
}

void launch_numeric(int conf, const CscView& A, const PruneParams& pp, const ExpandBuffers& b,
                    int grid, cudaStream_t s) {
    if (conf == 0)
        conf_launch<Conf0>(conf, A, pp, b, grid, s);
    else if (pp.table == 1)
        conf_launch<Conf1b>(conf, A, pp, b, grid, s);
    else if (pp.table == 2)
        conf_launch<Conf1c>(conf, A, pp, b, grid, s);
    else
        conf_launch<Conf1a>(conf, A, pp, b, grid, s);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// the prune rule alone on a materialised matrix (same candidate machinery;
// a column's entries are already row-ordered)
// ---------------------------------------------------------------------------

constexpr int PR_T = 256, PR_VC = 2048;

struct ColumnChunkEnum {
    const int32_t* rows;
    const float* vals;
    int i0, i1;
    __device__ int count(uint64_t tau) const {
        int c = 0;
        for (int i = i0; i < i1; ++i) c += make_key(vals[i], rows[i]) > tau;
        return c;
    }
    __device__ void emit(uint64_t tau, uint64_t* dst, int base) const {
        dst += base;
        for (int i = i0; i < i1; ++i) {
            const uint64_t k = make_key(vals[i], rows[i]);
            if (k > tau) *dst++ = k;
        }
    }
};

struct PruneArgs2 {
    CscView B;
    PruneParams pp;
    ExpandBuffers b;
};

__global__ void __launch_bounds__(PR_T) k_prune(PruneArgs2 a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ksel = a.pp.ksel;
    const int topcap = ksel + PR_VC;
    uint64_t* top = reinterpret_cast<uint64_t*>(smem);
    unsigned* hist = reinterpret_cast<unsigned*>(top + topcap);
    unsigned long long* mhist = reinterpret_cast<unsigned long long*>(hist + 256);
    WinShared* sh = reinterpret_cast<WinShared*>(mhist + 256);
    const int tid = threadIdx.x;
    const CscView& B = a.B;
    const ExpandBuffers& b = a.b;
    for (;;) {
        if (tid == 0) sh->item = atomicAdd(&b.ctr->work_ctr, 1);
        __syncthreads();
        const int64_t j = sh->item;
        __syncthreads();
        if (j >= B.n) break;
        const int64_t cb = B.colptr[j], ce = B.colptr[j + 1];
        int ntop = 0;
        uint64_t tau = 0;
        double s_sum = 0.0, s_mt = 0.0;
        long long s_t = 0;
        for (int64_t base = cb; base < ce; base += PR_VC) {
            const int cnt = (int)min((int64_t)PR_VC, ce - base);
            const int per = (cnt + PR_T - 1) / PR_T;
            ColumnChunkEnum en{B.rowidx + base, B.val + base, min(cnt, tid * per),
                               min(cnt, tid * per + per)};
            int c = 0;
            for (int i = en.i0; i < en.i1; ++i) {
                const float v = en.vals[i];
                s_sum += (double)v;
                if (v >= a.pp.theta) {
                    ++s_t;
                    s_mt += (double)v;
                }
                c += make_key(v, en.rows[i]) > tau;
            }
            append_candidates<PR_T, 8>(en, top, topcap, ksel, ntop, tau, c, hist, sh);
        }
        double dv[2] = {s_sum, s_mt};
        long long qv[1] = {s_t};
        block_sum<PR_T>(dv, 2, qv, 1, &sh->bs);
        int mstar = 0;
        double ch = 0.0;
        const int64_t obase = b.off[j];
        finish_column<PR_T, 8, true>(top, ntop, topcap, a.pp, dv[0], dv[1], qv[0], b.cap[j],
                                     b.tmp_row + (obase - b.tmp_off0),
                                     b.tmp_val + (obase - b.tmp_off0), hist, mhist, sh, b.ctr, 0,
                                     0, nullptr, &mstar, &ch);
        if (tid == 0) {
            b.kept[j] = mstar;
            b.chaos[j] = ch;
            b.bnnz[j] = ce - cb;
        }
    }
}

// The prune rule, inflation and renormalisation of a merged product whose
// entries are the exact 64-bit fixed-point sums of the numeric pass
// (rows sorted per column; column j's scale from the column sum bsum[j]):
// the statistics and keys of the numeric pass, so the same iteration.
struct FixedChunkEnum {
    const int32_t* rows;
    const unsigned long long* q;
    FixScale fx;
    int i0, i1;
    __device__ int count(uint64_t tau) const {
        int c = 0;
        for (int i = i0; i < i1; ++i) c += make_key(fx.value(q[i]), rows[i]) > tau;
        return c;
    }
    __device__ void emit(uint64_t tau, uint64_t* dst, int base) const {
        dst += base;
        for (int i = i0; i < i1; ++i) {
            const uint64_t k = make_key(fx.value(q[i]), rows[i]);
            if (k > tau) *dst++ = k;
        }
    }
};

struct PruneFixedArgs {
    int32_t n;
    const int64_t* colptr;
    const int32_t* rowidx;
    const unsigned long long* q;
    const double* bsum;
    PruneParams pp;
    ExpandBuffers b;
};

__global__ void __launch_bounds__(PR_T) k_prune_fixed(PruneFixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ksel = a.pp.ksel;
    const int topcap = ksel + PR_VC;
    uint64_t* top = reinterpret_cast<uint64_t*>(smem);
    unsigned* hist = reinterpret_cast<unsigned*>(top + topcap);
    unsigned long long* mhist = reinterpret_cast<unsigned long long*>(hist + 256);
    WinShared* sh = reinterpret_cast<WinShared*>(mhist + 256);
    const int tid = threadIdx.x;
    const ExpandBuffers& b = a.b;
    for (;;) {
        if (tid == 0) sh->item = atomicAdd(&b.ctr->work_ctr, 1);
        __syncthreads();
        const int64_t j = sh->item;
        __syncthreads();
        if (j >= a.n) break;
        const int64_t cb = a.colptr[j], ce = a.colptr[j + 1];
        const double S = a.bsum[j];
        FixScale fx;
        fx.init(S);
        int ntop = 0;
        uint64_t tau = 0;
        unsigned long long s_mt = 0;
        long long s_t = 0;
        for (int64_t base = cb; base < ce; base += PR_VC) {
            const int cnt = (int)min((int64_t)PR_VC, ce - base);
            const int per = (cnt + PR_T - 1) / PR_T;
            FixedChunkEnum en{a.rowidx + base, a.q + base, fx, min(cnt, tid * per),
                              min(cnt, tid * per + per)};
            int c = 0;
            for (int i = en.i0; i < en.i1; ++i) {
                const unsigned long long qi = en.q[i];
                const float v = fx.value(qi);
                if (v >= a.pp.theta) {
                    ++s_t;
                    s_mt += qi;
                }
                c += make_key(v, en.rows[i]) > tau;
            }
            append_candidates<PR_T, 8>(en, top, topcap, ksel, ntop, tau, c, hist, sh);
        }
        double dv[1] = {0.0};
        long long qv[2] = {s_t, (long long)s_mt};
        block_sum<PR_T>(dv, 0, qv, 2, &sh->bs);
        const double MT = ldexp((double)(unsigned long long)qv[1], -fx.f);
        int mstar = 0;
        double ch = 0.0;
        const int64_t obase = b.off[j];
        finish_column<PR_T, 8, true>(top, ntop, topcap, a.pp, S, MT, qv[0], b.cap[j],
                                     b.tmp_row + (obase - b.tmp_off0),
                                     b.tmp_val + (obase - b.tmp_off0), hist, mhist, sh, b.ctr, 0,
                                     0, nullptr, &mstar, &ch);
        if (tid == 0) {
            b.kept[j] = mstar;
            b.chaos[j] = ch;
            b.bnnz[j] = ce - cb;
        }
    }
}

void launch_prune_fixed(int32_t n, const int64_t* colptr, const int32_t* rowidx,
                        const unsigned long long* q, const double* bsum, const PruneParams& pp,
                        const ExpandBuffers& b, int num_sms, cudaStream_t s) {
    if (n == 0) return;
    const size_t smem = (size_t)(pp.ksel + PR_VC) * 8 + 256 * 4 + 256 * 8 + sizeof(WinShared);
    cudaFuncSetAttribute(k_prune_fixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_prune_fixed, PR_T, smem);
    if (occ < 1) occ = 1;
    int grid = occ * num_sms;
    if ((int64_t)grid > n) grid = (int)n;
    cudaMemsetAsync(&b.ctr->work_ctr, 0, sizeof(int), s);
    k_prune_fixed<<<grid, PR_T, smem, s>>>(PruneFixedArgs{n, colptr, rowidx, q, bsum, pp, b});
    count_launches(1);
}

void launch_prune(const CscView& B, const PruneParams& pp, const ExpandBuffers& b, int num_sms,
                  cudaStream_t s) {
    if (B.n == 0) return;
    const size_t smem = (size_t)(pp.ksel + PR_VC) * 8 + 256 * 4 + 256 * 8 + sizeof(WinShared);
    cudaFuncSetAttribute(k_prune, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_prune, PR_T, smem);
    if (occ < 1) occ = 1;
    int grid = occ * num_sms;
    if ((int64_t)grid > B.n) grid = (int)B.n;
    cudaMemsetAsync(&b.ctr->work_ctr, 0, sizeof(int), s);
    k_prune<<<grid, PR_T, smem, s>>>(PruneArgs2{B, pp, b});
    count_launches(1);
}

}  // namespace mcl

