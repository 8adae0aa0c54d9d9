// The fused numeric pass of one MCL iteration (Algorithm 1: expansion,
// Prune, inflation) with an order-preserving shared-memory accumulator.
//
// One CTA owns one output column j at a time (persistent grid, LPT order).
// The column's row span is processed in windows of at most WW*32 rows:
//
//   1. bitmap:     every product row of the window sets a bit (the exact
//                  symbolic pass of Sections II and V, restricted to the
//                  window);
//   2. prefix:     block scan of the words' popcounts, so that
//                  rank(row) = prefix[word] + popc(word & lower bits) is a
//                  collision-free, row-order-preserving index;
//   3. accumulate: c_ij += a_ik * a_kj (FP32) at vals[rank(i)] -- a dense
//                  array without keys, probes or compare-and-swap;
//   4. extract:    in row order: exact column statistics (sum, count and
//                  mass above the threshold) and ranking keys above the
//                  running top-k bound tau, appended stably to a row-ordered
//                  candidate buffer, which is cut back to the top ksel
//                  entries (radix select + stable compaction) only when full.
//
// A window whose entries exceed the value capacity is cut at the last
// bitmap word that fits (counted as a split) and the next window narrows
// to the observed density; results never depend on the size estimate.
// Finally the prune rule picks m* (threshold / top-k / recovery), the kept
// keys are compacted stably (so rows come out sorted without a sort),
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
    int cutw;
    int pad;
};

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

// Scratch per CTA in global memory (stride = cur_stride sources):
//   [0 .. s)      int64 start of the source column
//   [s .. 2s)     (as int32 pairs) length, cursor
//   ...           see SrcMeta below
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

// Finish a column: prune rule on the row-ordered candidate keys top[0..ntop)
// plus exact statistics; stable output of the kept entries with inflation
// (inflate != 0) or their B values; returns m* and chaos_j via the pointers.
template <int T, int IPT>
__device__ void finish_column(uint64_t* top, int ntop, const PruneParams& pp, double S, double MT,
                              long long Tt, int64_t cap, int32_t* out_row, float* out_val,
                              unsigned* hist, unsigned long long* mhist, WinShared* sh, DevCounters* ctr,
                              int* mstar_out, double* chaos_out) {
    const int tid = threadIdx.x;
    const double target = (double)pp.p * S;
    const int q = (int)(Tt < (long long)pp.K ? Tt : (long long)pp.K);
    double mq;
    uint64_t kq = 0;
    if (Tt <= pp.K) {
        mq = MT;
    } else {
        kq = block_select_count<T>(top, ntop, top, 0, pp.K, hist, &sh->bs);
        double part = 0.0;
        for (int i = tid; i < ntop; i += T) {
            const uint64_t x = top[i];
            if (x >= kq) part += (double)key_val(x);
        }
        double dv[1] = {part};
        long long qv[1] = {0};
        block_sum<T>(dv, 1, qv, 0, &sh->bs);
        mq = dv[0];
    }
    int mstar;
    uint64_t cut;
    bool have_cut = false;
    if (target <= 0.0 || mq >= target) {
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
    // pass 1: per-thread kept counts and inflated sum over contiguous chunks
    const int per = (ntop + T - 1) / T;
    const int i0 = tid * per, i1 = min(ntop, i0 + per);
    int c = 0;
    double usum = 0.0;
    if (mstar > 0) {
        for (int i = i0; i < i1; ++i) {
            const uint64_t x = top[i];
            if (x >= cut) {
                ++c;
                if (pp.inflate) usum += (double)inflate_value(key_val(x), pp.r);
            }
        }
    }
    double dv[1] = {usum};
    long long qv[1] = {0};
    block_sum<T>(dv, 1, qv, 0, &sh->bs);
    const double U = dv[0];
    const double invU = U > 0.0 ? 1.0 / U : 0.0;
    int tot;
    int o = block_scan_excl<T>(c, &tot, sh->wsm);
    if (tid == 0 && tot != mstar) set_err2(ctr, ERR_INTERNAL);
    double amax = 0.0, asq = 0.0;
    if (mstar > 0) {
        for (int i = i0; i < i1; ++i) {
            const uint64_t x = top[i];
            if (x >= cut) {
                if (o >= mstar) break;
                const float v = key_val(x);
                float outv = v;
                if (pp.inflate) {
                    const double a = (double)inflate_value(v, pp.r) * invU;
                    outv = (float)a;
                    amax = a > amax ? a : amax;
                    asq += a * a;
                }
                out_row[o] = key_row(x);
                out_val[o] = outv;
                ++o;
            }
        }
    }
    double ch = 0.0;
    if (pp.inflate) {
        const double mx = block_max_d<T>(amax, &sh->bs);
        double dv2[1] = {asq};
        block_sum<T>(dv2, 1, qv, 0, &sh->bs);
        ch = mx - dv2[0];
        if (ch < 0.0) ch = 0.0;
    }
    if (tid == 0) {
        *mstar_out = mstar;
        *chaos_out = ch;
    }
    __syncthreads();
}

// Append the candidates an enumerator yields (stably, in its order) to the
// row-ordered buffer top[0..ntop); first cuts the buffer back to ksel
// entries if they would not fit.  `count(tau)` returns this thread's number
// of keys > tau; `emit(tau, dst, base)` writes every thread's keys in the
// enumerator's stable order, given each thread's exclusive scan offset.
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

// Enumerates a window's entries (bitmap + prefix + dense values).  Warp w
// owns words [w*wpw, (w+1)*wpw); lane l takes words w*wpw + 32q + l, so
// shared-memory accesses are conflict-free and the stable (row) order is
// round q, then lane.
struct WindowEnum {
    const uint32_t* bm;
    const int32_t* pre;
    const float* vals;
    int nw, wpw, r0;
    __device__ int word(int q) const { return (threadIdx.x >> 5) * wpw + 32 * q + (threadIdx.x & 31); }
    __device__ int count(uint64_t tau) const {
        int c = 0;
        for (int q = 0; q < wpw / 32; ++q) {
            const int w = word(q);
            if (w >= nw) break;
            uint32_t m = bm[w];
            int r = pre[w];
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                if (make_key(vals[r], r0 + 32 * w + b) > tau) ++c;
                ++r;
            }
        }
        return c;
    }
    // base: this thread's exclusive block-scan offset of count()
    __device__ void emit(uint64_t tau, uint64_t* dst, int base) const {
        const int lane = threadIdx.x & 31;
        int run = __shfl_sync(FULL, base, 0);  // the warp's first output slot
        for (int q = 0; q < wpw / 32; ++q) {
            const int w = word(q);
            int c = 0;
            uint32_t m0 = 0;
            int r0w = 0;
            if (w < nw) {
                m0 = bm[w];
                r0w = pre[w];
                uint32_t m = m0;
                int r = r0w;
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    if (make_key(vals[r], r0 + 32 * w + b) > tau) ++c;
                    ++r;
                }
            }
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            int pos = run + incl - c;
            uint32_t m = m0;
            int r = r0w;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const uint64_t key = make_key(vals[r], r0 + 32 * w + b);
                if (key > tau) dst[pos++] = key;
                ++r;
            }
            run += __shfl_sync(FULL, incl, 31);
        }
    }
};

// Expected entries per source and window below which a window walks its
// sources one per lane instead of one per warp.
constexpr int LANE_MODE_MAX = 12;

struct ExpandArgs {
    CscView A;
    PruneParams pp;
    ExpandBuffers b;
    int conf;
};

template <int T, int WW, int VC>
struct ExpandLayout {
    static constexpr size_t bytes(int ksel) {
        return (size_t)WW * 4 + (size_t)WW * 4 + (size_t)VC * 4 + (size_t)(ksel + VC) * 8 +
               256 * 4 + 256 * 8 + sizeof(WinShared);
    }
};

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

template <int T, int WW, int VC, int MINB>
__global__ void __launch_bounds__(T, MINB) k_expand(ExpandArgs a) {
    constexpr int WROWS = WW * 32;
    constexpr int IPT = 8;
    constexpr int NWARP = T / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem);
    int32_t* pre = reinterpret_cast<int32_t*>(bm + WW);
    float* vals = reinterpret_cast<float*>(pre + WW);
    uint64_t* top = reinterpret_cast<uint64_t*>(vals + VC);
    const int ksel = a.pp.ksel;
    const int topcap = ksel + VC;
    unsigned* hist = reinterpret_cast<unsigned*>(top + topcap);
    unsigned long long* mhist = reinterpret_cast<unsigned long long*>(hist + 256);
    WinShared* sh = reinterpret_cast<WinShared*>(mhist + 256);

    const int tid = threadIdx.x, lane = tid & 31;
    const CscView& A = a.A;
    const ExpandBuffers& b = a.b;
    DevCounters* ctr = b.ctr;
    SrcMeta meta(b.cursors + (int64_t)blockIdx.x * 6 * b.cur_stride, b.cur_stride);
    int32_t* brow = b.bucket_row ? b.bucket_row + (int64_t)blockIdx.x * b.bucket_cap : nullptr;
    float* bval = b.bucket_val ? b.bucket_val + (int64_t)blockIdx.x * b.bucket_cap : nullptr;
    int32_t* woff = b.woff ? b.woff + (int64_t)blockIdx.x * (WINDOW_MAX + 1) : nullptr;
    const int wbeg = ctr->bin_off[a.conf * NZ], wend = ctr->bin_off[a.conf * NZ + NZ];

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
        // column sum of B_*j from the identity sum_i (AA)_ij = sum_k a_kj sum_i a_ik
        // (FP64; exact up to FP64 rounding, independent of the FP32 accumulation)
        double s_sum = 0.0;
        for (int i = tid; i < d; i += T) {
            const int k = A.rowidx[cb + i];
            const int64_t ks = A.colptr[k];
            const float akj = A.val[cb + i];
            meta.ks[i] = ks;
            meta.len[i] = (int)(A.colptr[k + 1] - ks);
            meta.cur[i] = 0;
            meta.akj[i] = akj;
            s_sum += (double)akj * b.colsum[k];
        }
        // ---- plan: one window, bucketed windows, or source-cursor windows ----
        int nwin = 1, width = span;
        bool bucket = false;
        const bool single = span <= WROWS && est * 4 <= (int64_t)VC * 3;
        if (!single && brow != nullptr && flops_j <= b.bucket_cap) {
            const int64_t nw1 = ((int64_t)span + WROWS - 1) / WROWS;
            const int64_t nw2 = (est * 4 + (int64_t)VC * 3 - 1) / ((int64_t)VC * 3);
            const int64_t nwr = nw1 > nw2 ? nw1 : nw2;
            if (nwr <= (WINDOW_MAX < WW ? WINDOW_MAX : WW)) {
                width = (int)((((int64_t)span + nwr - 1) / nwr + 31) & ~31ll);
                nwin = (int)(((int64_t)span + width - 1) / width);
                bucket = true;
            }
        }
        int ntop = 0;
        uint64_t tau = 0;
        double s_mt = 0.0;
        long long s_t = 0, s_n = 0;
        FastDiv fdiv;
        fdiv.init((uint32_t)width);
        __syncthreads();

        if (bucket) {
            // ---- count the products of every window ----
            int* wcnt = reinterpret_cast<int*>(bm);
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
                        const bool v = pb + 32 * c + lane < len;
                        const unsigned act = __ballot_sync(FULL, v);
                        if (v) {
                            const uint32_t w = fdiv.div((uint32_t)(rr[c] - lo));
                            const unsigned grp = __match_any_sync(act, w);
                            if (__ffs(grp) - 1 == lane) atomicAdd(wcnt + w, __popc(grp));
                        }
                    }
                }
            }
            __syncthreads();
            // ---- window offsets (exclusive scan), scatter cursors in pre ----
            {
                const int per = (nwin + T - 1) / T;
                const int i0 = min(nwin, tid * per), i1 = min(nwin, i0 + per);
                int c = 0;
                for (int i = i0; i < i1; ++i) c += wcnt[i];
                int tot;
                int run = block_scan_excl<T>(c, &tot, sh->wsm);
                for (int i = i0; i < i1; ++i) {
                    woff[i] = run;
                    pre[i] = run;
                    run += wcnt[i];
                }
                if (tid == 0) woff[nwin] = tot;
                if (tid == 0 && (int64_t)tot != flops_j) set_err2(ctr, ERR_INTERNAL);
            }
            if (tid == 0) sh->next = 0;
            __syncthreads();
            // ---- scatter (row, a_ik * a_kj) into the window buckets ----
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
                for (int pb = 0; pb < len; pb += 128) {
                    int rr[4];
                    float pv[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int p = pb + 32 * c + lane;
                        rr[c] = p < len ? __ldg(rows + p) : 0;
                        pv[c] = p < len ? __ldg(vv + p) : 0.0f;
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                    const bool v = pb + 32 * c + lane < len;
                    const unsigned act = __ballot_sync(FULL, v);
                    if (v) {
                        const int row = rr[c];
                        const float prod = pv[c] * akj;
                        const uint32_t w = fdiv.div((uint32_t)(row - lo));
                        const unsigned grp = __match_any_sync(act, w);
                        const int leader = __ffs(grp) - 1;
                        int base = 0;
                        if (lane == leader) base = atomicAdd(pre + w, __popc(grp));
                        base = __shfl_sync(grp, base, leader);
                        const int pos = base + __popc(grp & lanemask_lt());
                        brow[pos] = row;
                        bval[pos] = prod;
                    }
                    }
                }
            }
            __syncthreads();
        }

        int wrows;
        {
            const double rows = 0.8 * (double)VC * (double)span / (double)est;
            wrows = rows >= (double)WROWS ? WROWS : (int)rows;
            wrows &= ~31;
            if (wrows < 32) wrows = 32;
            if (single) wrows = ((span + 31) & ~31) < WROWS ? ((span + 31) & ~31) : WROWS;
        }
        int r0 = lo;
        int win = 0;
        int bs0 = 0, be0 = 0, wend_row = hiE;
        if (bucket) {
            bs0 = woff[0];
            be0 = woff[1];
            wend_row = min(hiE, lo + width);
        }
        while (r0 < hiE) {
            int r1;
            if (bucket) {
                if (r0 >= wend_row) {  // next bucket window
                    ++win;
                    bs0 = woff[win];
                    be0 = woff[win + 1];
                    wend_row = (int)min((int64_t)lo + (int64_t)(win + 1) * width, (int64_t)hiE);
                    r0 = (int)((int64_t)lo + (int64_t)win * width);
                    if (be0 == bs0) {  // empty window
                        r0 = wend_row;
                        continue;
                    }
                }
                r1 = wend_row;
                if (r1 - r0 > WROWS) r1 = r0 + WROWS;
            } else {
                r1 = (int)min((int64_t)r0 + wrows, (int64_t)hiE);
            }
            const int nw = (r1 - r0 + 31) >> 5;
            // ---- 1. bitmap of the window's product rows ----
            for (int i = tid; i < nw; i += T) bm[i] = 0u;
            if (tid == 0) sh->next = 0;
            const bool lane_mode = !bucket && (double)flops_j * (double)(r1 - r0) <
                                                  (double)LANE_MODE_MAX * (double)d * (double)span;
            __syncthreads();
            if (bucket) {
#pragma unroll 4
                for (int p = bs0 + tid; p < be0; p += T) {
                    const int r = brow[p];
                    if (r >= r0 && r < r1) {
                        const int off = r - r0;
                        atomicOr(bm + (off >> 5), 1u << (off & 31));
                    }
                }
            } else if (lane_mode) {
                for (int kidx = tid; kidx < d; kidx += T) {
                    const int len = meta.len[kidx];
                    const int32_t* rows = A.rowidx + meta.ks[kidx];
                    int pos = meta.cur[kidx];
                    while (pos < len) {
                        const int r = __ldg(rows + pos);
                        if (r >= r1) break;
                        const int off = r - r0;
                        atomicOr(bm + (off >> 5), 1u << (off & 31));
                        ++pos;
                    }
                    meta.nxt[kidx] = pos;
                }
            } else {
                for (;;) {
                    int kidx = 0;
                    if (lane == 0) kidx = atomicAdd(&sh->next, 1);
                    kidx = __shfl_sync(FULL, kidx, 0);
                    if (kidx >= d) break;
                    const int len = meta.len[kidx];
                    const int32_t* rows = A.rowidx + meta.ks[kidx];
                    int pos = meta.cur[kidx];
                    while (pos < len) {
                        int rr[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int p = pos + 32 * c + lane;
                            rr[c] = p < len ? __ldg(rows + p) : INT_MAX;
                        }
                        int consumed = 0;
                        bool stop = false;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (!stop) {
                                const bool in = rr[c] < r1;
                                const unsigned bal = __ballot_sync(FULL, in);
                                if (in) {
                                    const int off = rr[c] - r0;
                                    atomicOr(bm + (off >> 5), 1u << (off & 31));
                                }
                                const int nin = __popc(bal);
                                consumed += nin;
                                stop = nin < 32;
                            }
                        }
                        pos += consumed;
                        if (stop) break;
                    }
                    if (lane == 0) meta.nxt[kidx] = pos;
                }
            }
            __syncthreads();
            // ---- 2. prefix of popcounts: warp-contiguous, lane-interleaved words ----
            const int wpw = ((nw + NWARP * 32 - 1) / (NWARP * 32)) * 32;
            const int wbase = (tid >> 5) * wpw;
            int cnt = 0;
            for (int q = 0; q < wpw / 32; ++q) {
                const int w = wbase + 32 * q + lane;
                if (w < nw) cnt += __popc(bm[w]);
            }
            int total;
            int run = block_scan_excl<T>(cnt, &total, sh->wsm);
            run = __shfl_sync(FULL, run, 0);
            for (int q = 0; q < wpw / 32; ++q) {
                const int w = wbase + 32 * q + lane;
                const int c1 = w < nw ? __popc(bm[w]) : 0;
                int incl = c1;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                if (w < nw) pre[w] = run + incl - c1;
                run += __shfl_sync(FULL, incl, 31);
            }
            int r1c = r1, nwc = nw, Nw = total;
            const bool ovf = total > VC;
            if (ovf) {
                // cut at the first word whose entries would not fit
                if (tid == 0) sh->cutw = nw;
                __syncthreads();
                for (int q = 0; q < wpw / 32; ++q) {
                    const int w = wbase + 32 * q + lane;
                    if (w < nw) {
                        const int p0 = pre[w];
                        if (p0 <= VC && p0 + __popc(bm[w]) > VC) sh->cutw = w;
                    }
                }
                __syncthreads();
                nwc = sh->cutw;  // >= 1: one word holds at most 32 <= VC entries
                r1c = r0 + 32 * nwc;
                Nw = pre[nwc];
                wrows = max(32, 32 * nwc);
                if (tid == 0) atomicAdd(&ctr->splits, 1ull);
            }
            // ---- 3. accumulate c_ij at vals[rank(i)] ----
            for (int i = tid; i < Nw; i += T) vals[i] = 0.0f;
            if (tid == 0) sh->next = 0;
            __syncthreads();
            if (bucket) {
#pragma unroll 4
                for (int p = bs0 + tid; p < be0; p += T) {
                    const int r = brow[p];
                    if (r >= r0 && r < r1c) {
                        const int off = r - r0;
                        const int w = off >> 5;
                        const int rk = pre[w] + __popc(bm[w] & ((1u << (off & 31)) - 1u));
                        atomicAdd(vals + rk, bval[p]);
                    }
                }
            } else if (lane_mode) {
                for (int kidx = tid; kidx < d; kidx += T) {
                    const int64_t ks = meta.ks[kidx];
                    const int32_t* rows = A.rowidx + ks;
                    const float* vv = A.val + ks;
                    const float akj = meta.akj[kidx];
                    const int end = meta.nxt[kidx];
                    int p = meta.cur[kidx];
                    for (; p < end; ++p) {
                        const int row = __ldg(rows + p);
                        if (row >= r1c) break;
                        const int off = row - r0;
                        const int w = off >> 5;
                        const int rk = pre[w] + __popc(bm[w] & ((1u << (off & 31)) - 1u));
                        atomicAdd(vals + rk, __ldg(vv + p) * akj);
                    }
                    meta.cur[kidx] = p;
                }
            } else {
                for (;;) {
                    int kidx = 0;
                    if (lane == 0) kidx = atomicAdd(&sh->next, 1);
                    kidx = __shfl_sync(FULL, kidx, 0);
                    if (kidx >= d) break;
                    const int64_t ks = meta.ks[kidx];
                    const int32_t* rows = A.rowidx + ks;
                    const float* vv = A.val + ks;
                    const float akj = meta.akj[kidx];
                    const int pos = meta.cur[kidx];
                    const int end = meta.nxt[kidx];
                    if (!ovf) {
#pragma unroll 4
                        for (int p = pos + lane; p < end; p += 32) {
                            const int off = __ldg(rows + p) - r0;
                            const float v = __ldg(vv + p) * akj;
                            const int w = off >> 5;
                            const int rk = pre[w] + __popc(bm[w] & ((1u << (off & 31)) - 1u));
                            atomicAdd(vals + rk, v);
                        }
                        if (lane == 0) meta.cur[kidx] = end;
                    } else {
                        int used = 0;
                        for (int pb = pos; pb < end; pb += 32) {
                            const int p = pb + lane;
                            int row = INT_MAX;
                            if (p < end) row = __ldg(rows + p);
                            const bool in = row < r1c;
                            used += __popc(__ballot_sync(FULL, in));
                            if (in) {
                                const int off = row - r0;
                                const float v = __ldg(vv + p) * akj;
                                const int w = off >> 5;
                                const int rk = pre[w] + __popc(bm[w] & ((1u << (off & 31)) - 1u));
                                atomicAdd(vals + rk, v);
                            }
                        }
                        if (lane == 0) meta.cur[kidx] = pos + used;
                    }
                }
            }
            __syncthreads();
            // ---- 4. statistics and candidates, in row order ----
            const int wpw2 = ((nwc + NWARP * 32 - 1) / (NWARP * 32)) * 32;
            WindowEnum en{bm, pre, vals, nwc, wpw2, r0};
            int c = 0;
            for (int q = 0; q < wpw2 / 32; ++q) {
                const int w = en.word(q);
                if (w >= nwc) break;
                uint32_t m = bm[w];
                int r = pre[w];
                s_n += __popc(m);
                while (m) {
                    const int bb = __ffs(m) - 1;
                    m &= m - 1;
                    const float v = vals[r];
                    ++r;
                    if (v >= a.pp.theta) {
                        ++s_t;
                        s_mt += (double)v;
                    }
                    if (make_key(v, r0 + 32 * w + bb) > tau) ++c;
                }
            }
            append_candidates<T, IPT>(en, top, topcap, ksel, ntop, tau, c, hist, sh);
            const int width_done = r1c - r0;
            r0 = r1c;
            if (!ovf && !bucket) {
                // next window from the observed density
                const double dens = (double)max(Nw, 1) / (double)width_done;
                const double rows = 0.8 * (double)VC / dens;
                int nwr = rows >= (double)WROWS ? WROWS : (int)rows;
                nwr &= ~31;
                if (nwr > 2 * wrows) nwr = 2 * wrows;
                wrows = nwr < 32 ? 32 : nwr;
            }
        }
        double dv[2] = {s_sum, s_mt};
        long long qv[2] = {s_t, s_n};
        block_sum<T>(dv, 2, qv, 2, &sh->bs);
        int mstar = 0;
        double ch = 0.0;
        const int64_t obase = b.off[j];
        finish_column<T, IPT>(top, ntop, a.pp, dv[0], dv[1], qv[0], b.cap[j],
                              b.tmp_row + (obase - b.tmp_off0), b.tmp_val + (obase - b.tmp_off0),
                              hist, mhist, sh, ctr, &mstar, &ch);
        if (tid == 0) {
            b.kept[j] = mstar;
            b.chaos[j] = ch;
            b.bnnz[j] = qv[1];
            if (qv[1] > est) atomicAdd(&ctr->misses, 1ull);
        }
    }
}

// configurations: 0 = small columns, 1 = everything else
#define CONF0 128, 512, 1024, 6
#define CONF1 256, 2048, 2048, 4

size_t numeric_smem(int conf, int ksel) {
    return conf == 0 ? ExpandLayout<128, 512, 1024>::bytes(ksel)
                     : ExpandLayout<256, 2048, 2048>::bytes(ksel);
}

int numeric_threads(int conf) { return conf == 0 ? 128 : 256; }

int numeric_grid(int conf, int ksel, int num_sms) {
    const size_t smem = numeric_smem(conf, ksel);
    int occ = 0;
    if (conf == 0) {
        cudaFuncSetAttribute(k_expand<CONF0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_expand<CONF0>, 128, smem);
    } else {
        cudaFuncSetAttribute(k_expand<CONF1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_expand<CONF1>, 256, smem);
    }
    if (occ < 1) occ = 1;
    return occ * num_sms;
}

// capacity of a window's values per configuration (for binning)
int conf_value_capacity(int conf) { return conf == 0 ? 1024 : 2048; }

void launch_numeric(int conf, const CscView& A, const PruneParams& pp, const ExpandBuffers& b,
                    int grid, cudaStream_t s) {
    ExpandArgs a{A, pp, b, conf};
    const size_t smem = numeric_smem(conf, pp.ksel);
    if (conf == 0)
        k_expand<CONF0><<<grid, 128, smem, s>>>(a);
    else
        k_expand<CONF1><<<grid, 256, smem, s>>>(a);
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
        finish_column<PR_T, 8>(top, ntop, a.pp, dv[0], dv[1], qv[0], b.cap[j],
                               b.tmp_row + (obase - b.tmp_off0), b.tmp_val + (obase - b.tmp_off0),
                               hist, mhist, sh, b.ctr, &mstar, &ch);
        if (tid == 0) {
            b.kept[j] = mstar;
            b.chaos[j] = ch;
            b.bnnz[j] = ce - cb;
        }
    }
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
