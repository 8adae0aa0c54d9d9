// C ABI of the MCL expansion library: context, scratch, argument checks and
// the host-side order of the kernels of one iteration (see mcl.h).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "mcl.h"
#include "mcl_internal.h"

using namespace mcl;

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct mcl_ctx {
    int device = 0;
    int num_sms = 0;
    mcl_alloc_fn alloc = nullptr;
    mcl_free_fn release = nullptr;
    void* user = nullptr;
    char err[512] = {0};
    // scratch
    Buf flops, colsum, rlo, rhi, cap, off, est, bucket, work, kept, chaos, bnnz, tmp_row, tmp_val,
        cursors, scan, ctr, active, bucket_row, woff, comp_off, comp_of_col, comp_bits,
        comp_active;
    size_t bucket_budget = (size_t)32 << 30;  // bytes of product buckets (large config)
    size_t phase_budget = 0;                  // bytes of output staging per column batch (0: one)
    Buf phase_colptr;
    DevCounters* hctr = nullptr;      // mapped pinned host mirror of the device counters
    DevCounters* hctr_dev = nullptr;  // its device address (written by a kernel, no copy engine)
    mcl_stats stats{};
    cudaEvent_t ev[8] = {};
    // options
    int sizing = -1;        // -1: from params (exact or learned); 0 exact; 1 flops bound
    int run_exact = 0;      // mcl_run: learned estimates missed too often, size exactly
    int conf_mask = 0x3;    // numeric configurations allowed
    int validate = 1;
    int est_milli = 1000;   // estimate scale (test knob)
    int graph_mode = 1;     // batched mcl_run replays iterations >= 2 as CUDA graphs
    int small_max = 512;    // autotuned: small-configuration bound on the estimate
    int table = 0;          // autotuned: shape of the large configuration
    int plan = 0;           // autotuned: rows planned per window (0: half the table)
    int64_t graph_cap = 0;  // entries of the replay buffers (0: per-component bound)
    size_t group_budget = 0;  // bytes per group of components in a batched mcl_run (0: one group)
    int in_group = 0;         // mcl_run is running one group
    // learned estimator (weights on device)
    Buf mlp_w, mlp_norm, colmax, feats, prev_logcf, iter_dev;
    int has_estimator = 0;
    float est_safety = 1.25f;
    int iteration = 1;
    int prev_valid = 0;
    // Cohen's estimator
    int cohen_r = 8;
    uint64_t cohen_seed = 2002;
    Buf cohen_m, cohen_e;
    // inner-dimension split
    Buf split_bsum, split_cnt, split_scratch;
};

namespace {

mcl_status fail(mcl_ctx* c, mcl_status st, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

void* dev_alloc(mcl_ctx* c, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->alloc) return c->alloc(bytes, c->user, (void*)s);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(mcl_ctx* c, void* p, cudaStream_t s) {
    if (!p) return;
    if (c->release)
        c->release(p, c->user, (void*)s);
    else
        cudaFreeAsync(p, s);
}

bool ensure(mcl_ctx* c, Buf& b, size_t bytes, cudaStream_t s) {
    if (b.p && b.bytes >= bytes) return true;
    dev_free(c, b.p, s);
    size_t nb = bytes + bytes / 8 + 256;
    b.p = dev_alloc(c, nb, s);
    b.bytes = b.p ? nb : 0;
    return b.p != nullptr;
}

#define CUDA_TRY(ctx, call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, MCL_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

mcl_status check_launch(mcl_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, MCL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return MCL_OK;
}

mcl_status err_flags(mcl_ctx* c, unsigned f) {
    if (!f) return MCL_OK;
    if (f & (ERR_COLPTR | ERR_ROW_RANGE | ERR_ROW_ORDER | ERR_VALUE))
        return fail(c, MCL_ERR_INVALID, "malformed CSC input (flags 0x%x: %s%s%s%s)", f,
                    (f & ERR_COLPTR) ? "colptr " : "", (f & ERR_ROW_RANGE) ? "row-range " : "",
                    (f & ERR_ROW_ORDER) ? "row-order " : "", (f & ERR_VALUE) ? "value " : "");
    if (f & ERR_TIMEOUT) return fail(c, MCL_ERR_TIMEOUT, "a bounded device loop gave up");
    return fail(c, MCL_ERR_INTERNAL, "device consistency check failed (flags 0x%x)", f);
}

mcl_status check_params(mcl_ctx* c, const mcl_params* prm, PruneParams* pp, bool need_inflation) {
    if (!prm) return fail(c, MCL_ERR_INVALID, "params is NULL");
    if (prm->select_k < 1 || prm->select_k > MCL_MAX_SELECT_K)
        return fail(c, MCL_ERR_INVALID, "select_k must be in [1, %d]", MCL_MAX_SELECT_K);
    int krec = prm->recover_k > 0 ? prm->recover_k : prm->select_k;
    if (krec > MCL_MAX_SELECT_K)
        return fail(c, MCL_ERR_INVALID, "recover_k must be <= %d", MCL_MAX_SELECT_K);
    if (!(prm->recover_pct >= 0.0f && prm->recover_pct <= 1.0f))
        return fail(c, MCL_ERR_INVALID, "recover_pct must be in [0, 1]");
    if (!(prm->threshold >= 0.0f) || !(prm->threshold <= 3.0e38f))
        return fail(c, MCL_ERR_INVALID, "threshold must be finite and >= 0");
    if (need_inflation && !(prm->inflation > 0.0f && prm->inflation <= 1.0e6f))
        return fail(c, MCL_ERR_INVALID, "inflation must be > 0");
    pp->small_max = c->small_max;
    pp->table = c->table;
    pp->plan = c->plan;
    pp->theta = prm->threshold;
    pp->K = prm->select_k;
    pp->p = prm->recover_pct;
    pp->Krec = krec;
    pp->ksel = prm->select_k > krec ? prm->select_k : krec;
    pp->r = prm->inflation;
    pp->inflate = 1;
    return MCL_OK;
}

mcl_status check_csc(mcl_ctx* c, const mcl_csc* A, const char* name) {
    if (!A) return fail(c, MCL_ERR_INVALID, "%s is NULL", name);
    if (A->n < 0 || A->n > 0x7FFFFFFE) return fail(c, MCL_ERR_INVALID, "%s: bad n", name);
    if (A->nnz < 0) return fail(c, MCL_ERR_INVALID, "%s: bad nnz", name);
    if (!A->colptr) return fail(c, MCL_ERR_INVALID, "%s: colptr is NULL", name);
    if (A->nnz > 0 && (!A->rowidx || !A->val))
        return fail(c, MCL_ERR_INVALID, "%s: rowidx/val is NULL", name);
    return MCL_OK;
}

CscView view(const mcl_csc* A) {
    return CscView{A->n, A->nnz, A->colptr, A->rowidx, A->val};
}

ExpandBuffers buffers(mcl_ctx* c) {
    ExpandBuffers b{};
    b.flops = (int64_t*)c->flops.p;
    b.colsum = (double*)c->colsum.p;
    b.rlo = (int32_t*)c->rlo.p;
    b.rhi = (int32_t*)c->rhi.p;
    b.cap = (int64_t*)c->cap.p;
    b.off = (int64_t*)c->off.p;
    b.est = (int64_t*)c->est.p;
    b.bucket = (int32_t*)c->bucket.p;
    b.work = (int32_t*)c->work.p;
    b.kept = (int32_t*)c->kept.p;
    b.chaos = (double*)c->chaos.p;
    b.bnnz = (int64_t*)c->bnnz.p;
    b.tmp_row = (int32_t*)c->tmp_row.p;
    b.tmp_val = (float*)c->tmp_val.p;
    b.cursors = (int32_t*)c->cursors.p;
    b.cur_stride = 0;
    b.bucket_row = nullptr;
    b.woff = nullptr;
    b.bucket_cap = 0;
    b.scan_tmp = (int64_t*)c->scan.p;
    b.ctr = (DevCounters*)c->ctr.p;
    b.active = nullptr;
    b.nnz_is_bound = 0;
    return b;
}

mcl_status ensure_columns(mcl_ctx* c, int64_t n, cudaStream_t s) {
    const size_t n1 = (size_t)n + 1;
    bool ok = ensure(c, c->flops, n1 * 8, s) && ensure(c, c->colsum, n1 * 8, s) &&
              ensure(c, c->rlo, n1 * 4, s) &&
              ensure(c, c->rhi, n1 * 4, s) && ensure(c, c->cap, n1 * 8, s) &&
              ensure(c, c->off, n1 * 8, s) && ensure(c, c->est, n1 * 8, s) &&
              ensure(c, c->bucket, n1 * 4, s) && ensure(c, c->work, n1 * 4, s) &&
              ensure(c, c->kept, n1 * 4, s) && ensure(c, c->chaos, n1 * 8, s) &&
              ensure(c, c->bnnz, n1 * 8, s) &&
              ensure(c, c->scan, (size_t)scan_tmp_len_for(n1) * 8, s) &&
              ensure(c, c->ctr, sizeof(DevCounters), s);
    if (!ok) return fail(c, MCL_ERR_OOM, "scratch allocation failed (n=%lld)", (long long)n);
    return MCL_OK;
}

mcl_status read_counters(mcl_ctx* c, cudaStream_t s) {
    // a kernel writes the mirror, so that the read does not queue on a copy
    // engine behind the caller's large transfers on other streams
    launch_copy_counters((const DevCounters*)c->ctr.p, c->hctr_dev, s);
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return MCL_OK;
}

double chaos_from_bits(unsigned long long b) {
    double d;
    memcpy(&d, &b, 8);
    return d;
}

int max_numeric_grid(mcl_ctx* c, const PruneParams& pp) {
    int g = 0;
    for (int q = 0; q < NCONF; ++q) {
        int gq = numeric_grid(q, pp, c->num_sms);
        if (gq > g) g = gq;
    }
    int gs = symbolic_grid(c->num_sms);
    return g > gs ? g : gs;
}

}  // namespace

// Learned estimate: features -> MLP -> b.est (needs colstats done).
static mcl_status internal_estimate(mcl_ctx* c, const mcl_csc* A, const ExpandBuffers& b,
                                    cudaStream_t s) {
    const size_t n1 = (size_t)A->n + 1;
    if (!ensure(c, c->colmax, n1 * 4, s) || !ensure(c, c->feats, n1 * 4 * MCL_NFEATURES, s))
        return fail(c, MCL_ERR_OOM, "estimator scratch allocation failed");
    const float* prev = (c->prev_valid && c->prev_logcf.bytes >= n1 * 4)
                            ? (const float*)c->prev_logcf.p : nullptr;
    launch_colmax_features(view(A), c->iteration, prev, (float*)c->colmax.p, (float*)c->feats.p, s);
    launch_mlp_forward((const float*)c->feats.p, A->n, (const uint16_t*)c->mlp_w.p,
                       (const float*)c->mlp_norm.p, nullptr, b.est, c->est_safety, b.flops, b.rlo,
                       b.rhi, s);
    return check_launch(c, "estimator");
}

extern "C" {

const char* mcl_version(void) { return "mcl-gb300 1.0 (sm_103a)"; }

int64_t mcl_launch_count(void) { return (int64_t)launches_total(); }

mcl_status mcl_create(mcl_ctx** out, int device, mcl_alloc_fn alloc, mcl_free_fn release,
                      void* alloc_user) {
    if (!out) return MCL_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MCL_ERR_INVALID;
    }
    if ((alloc == nullptr) != (release == nullptr)) return MCL_ERR_INVALID;
    mcl_ctx* c = new mcl_ctx();
    c->device = device;
    c->alloc = alloc;
    c->release = release;
    c->user = alloc_user;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaHostAlloc((void**)&c->hctr, sizeof(DevCounters), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&c->hctr_dev, c->hctr, 0) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return MCL_ERR_CUDA;
    }
    for (auto& e : c->ev) cudaEventCreate(&e);
    *out = c;
    return MCL_OK;
}

void mcl_destroy(mcl_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    Buf* all[] = {&c->phase_colptr, &c->bucket_row, &c->woff, &c->comp_off,
                  &c->comp_of_col,
                  &c->comp_bits, &c->comp_active,
                  &c->flops, &c->colsum, &c->rlo, &c->rhi,  &c->cap,     &c->off,  &c->est,
                  &c->bucket, &c->work,   &c->kept,    &c->chaos,   &c->bnnz, &c->tmp_row,
                  &c->tmp_val, &c->cursors, &c->scan,  &c->ctr,     &c->active, &c->mlp_w,
                  &c->mlp_norm, &c->colmax, &c->feats, &c->prev_logcf, &c->cohen_m, &c->cohen_e,
                  &c->split_bsum, &c->split_cnt, &c->split_scratch,
                  &c->iter_dev};
    for (Buf* b : all) dev_free(c, b->p, 0);
    cudaDeviceSynchronize();
    for (auto& e : c->ev) cudaEventDestroy(e);
    if (c->hctr) cudaFreeHost(c->hctr);
    delete c;
}

const char* mcl_last_error(mcl_ctx* c) { return c ? c->err : "null context"; }

mcl_status mcl_get_stats(mcl_ctx* c, mcl_stats* st) {
    if (!c || !st) return MCL_ERR_INVALID;
    *st = c->stats;
    return MCL_OK;
}

mcl_status mcl_set_option(mcl_ctx* c, int option, int64_t value) {
    if (!c) return MCL_ERR_INVALID;
    switch (option) {
        case 1:  // sizing: -1 from params, 0 exact symbolic, 1 flops bound, 3 Cohen
            if (value < -1 || value > 3 || value == 2) return fail(c, MCL_ERR_INVALID, "bad sizing option");
            c->sizing = (int)value;
            return MCL_OK;
        case 2:  // numeric configuration mask
            if ((value & 0x3) == 0) return fail(c, MCL_ERR_INVALID, "conf mask selects nothing");
            c->conf_mask = (int)(value & 0x3);
            return MCL_OK;
        case 3:
            c->validate = value != 0;
            return MCL_OK;
        case 4:  // estimate scale in thousandths (1000 = as estimated)
            if (value < 1 || value > 1000000) return fail(c, MCL_ERR_INVALID, "bad scale");
            c->est_milli = (int)value;
            return MCL_OK;
        case 7:  // keys per vertex of Cohen's estimator
            if (value < 2 || value > cohen_max_r()) return fail(c, MCL_ERR_INVALID, "bad key count");
            c->cohen_r = (int)value;
            return MCL_OK;
        case 9:  // graph replay of batched iterations (0 off, 1 on)
            c->graph_mode = value != 0;
            return MCL_OK;
        case 10:  // entries of the graph replay buffers (0: per-component bound)
            if (value < 0) return fail(c, MCL_ERR_INVALID, "bad capacity");
            c->graph_cap = value;
            return MCL_OK;
        case 11:  // largest estimate of the small configuration
            if (value < 0 || value > 512) return fail(c, MCL_ERR_INVALID, "small bound in [0, 512]");
            c->small_max = (int)value;
            return MCL_OK;
        case 12:  // shape of the large configuration
            if (value < 0 || value > 2) return fail(c, MCL_ERR_INVALID, "table shape in [0, 2]");
            c->table = (int)value;
            return MCL_OK;
        case 13:  // entries planned per hashed window of the large configuration (0: half the table)
            if (value < 0 || value > 3072) return fail(c, MCL_ERR_INVALID, "plan in [0, 3072]");
            c->plan = (int)value;
            return MCL_OK;
        case 15:  // bytes of product buckets of the numeric pass
            if (value < 0) return fail(c, MCL_ERR_INVALID, "bad bucket budget");
            c->bucket_budget = (size_t)value;
            return MCL_OK;
        case 14:  // device bytes one group of components may use in a batched mcl_run
            if (value < 0) return fail(c, MCL_ERR_INVALID, "bad group budget");
            c->group_budget = (size_t)value;
            return MCL_OK;
        case 8:  // seed of Cohen's keys
            c->cohen_seed = (uint64_t)value;
            return MCL_OK;
        case 6:  // column-batch staging budget in bytes (0: one batch)
            if (value < 0) return fail(c, MCL_ERR_INVALID, "bad budget");
            c->phase_budget = (size_t)value;
            return MCL_OK;
        case 5:  // iteration index for the estimator's features
            if (value < 1 || value > 1000000) return fail(c, MCL_ERR_INVALID, "bad iteration");
            c->iteration = (int)value;
            return MCL_OK;
        default:
            return fail(c, MCL_ERR_INVALID, "unknown option %d", option);
    }
}

// One fused iteration on the given stream.  `active` (device uint8[n] or
// NULL) marks the columns to expand; inactive columns are copied through.
static mcl_status expand_impl(mcl_ctx* c, const mcl_csc* A, const mcl_params* prm, mcl_csc* out,
                              double* chaos, cudaStream_t s, const uint8_t* active) {
    PruneParams pp;
    mcl_status st = check_params(c, prm, &pp, true);
    if (st) return st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (!out) return fail(c, MCL_ERR_INVALID, "out is NULL");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int64_t n = A->n;
    if ((st = ensure_columns(c, n, s))) return st;
    ExpandBuffers b = buffers(c);
    b.active = active;
    const CscView Av = view(A);
    cudaEventRecord(c->ev[0], s);
    CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
    launch_colstats(Av, pp, b, c->num_sms, s);
    if ((st = check_launch(c, "colstats"))) return st;
    cudaEventRecord(c->ev[1], s);
    if ((st = read_counters(c, s))) return st;
    if ((st = err_flags(c, c->hctr->err))) return st;
    const int max_deg = c->hctr->max_deg;
    b.cur_stride = (max_deg + 31) & ~31;
    if (b.cur_stride < 32) b.cur_stride = 32;
    const int grid_max = max_numeric_grid(c, pp);
    if (!ensure(c, c->cursors, (size_t)grid_max * 6 * b.cur_stride * 4, s))
        return fail(c, MCL_ERR_OOM, "cursor scratch allocation failed");
    b.cursors = (int32_t*)c->cursors.p;
    // ---- size estimate ----
    const int sizing =
        c->sizing >= 0 ? c->sizing : (prm->use_estimator && !c->run_exact ? 2 : 0);
    if (sizing == 2) {
        if (!c->has_estimator)
            return fail(c, MCL_ERR_INVALID, "use_estimator set but no estimator loaded");
        if ((st = internal_estimate(c, A, b, s))) return st;
    } else if (sizing == 1) {
        launch_est_from_flops(Av, b, s);
    } else if (sizing == 3) {
        const size_t n1 = (size_t)n + 1;
        if (!ensure(c, c->cohen_m, n1 * c->cohen_r * 4, s) || !ensure(c, c->cohen_e, n1 * 4, s))
            return fail(c, MCL_ERR_OOM, "estimator scratch allocation failed");
        launch_cohen(Av, c->cohen_r, c->cohen_seed, (float*)c->cohen_m.p, (float*)c->cohen_e.p, s);
        launch_cohen_to_est((int32_t)n, (const float*)c->cohen_e.p, 1.0f, b, s);
    } else {
        launch_symbolic(Av, b, b.est, c->num_sms, grid_max, s);
        // exact counts bound each column's output: cap_j = min(cap_j, nnz_j)
        launch_cap_tighten((int32_t)n, b.est, b.cap, active, s);
    }
    if (c->est_milli != 1000) launch_scale_est(A->n, b.est, c->est_milli, s);
    if ((st = check_launch(c, "estimate"))) return st;
    launch_exclusive_scan<int64_t>(b.cap, n, b.off, b.scan_tmp, &b.ctr->cap_total, s);
    cudaEventRecord(c->ev[2], s);
    if ((st = read_counters(c, s))) return st;
    const int64_t cap_total = (int64_t)c->hctr->cap_total;
    // column batches (phases): the output staging of a batch fits the budget
    int64_t budget_entries = c->phase_budget > 0 ? (int64_t)(c->phase_budget / 8) : 0;
    if (budget_entries > 0 && budget_entries < pp.Krec) budget_entries = pp.Krec;
    const bool phased = budget_entries > 0 && cap_total > budget_entries && active == nullptr;
    const int64_t stage = phased ? budget_entries : cap_total;
    if (!ensure(c, c->tmp_row, (size_t)stage * 4 + 4, s) ||
        !ensure(c, c->tmp_val, (size_t)stage * 4 + 4, s))
        return fail(c, MCL_ERR_OOM, "scratch allocation failed (capacity %lld)", (long long)stage);
    b.tmp_row = (int32_t*)c->tmp_row.p;
    b.tmp_val = (float*)c->tmp_val.p;
    b.tmp_off0 = 0;
    // ---- binning + numeric over the columns a mask selects ----
    int used = 0;
    auto run_numeric = [&](const ExpandBuffers& bb) -> mcl_status {
        launch_binning(Av, pp, bb, c->conf_mask, s);
        for (int q = NCONF - 1; q >= 0; --q) {
            if (!((c->conf_mask >> q) & 1)) continue;
            const int g = numeric_grid(q, pp, c->num_sms);
            ExpandBuffers bq = bb;
            bq.bucket_row = nullptr;
            bq.woff = nullptr;
            bq.bucket_cap = 0;
            if (q == NCONF - 1) {
                // product buckets for multi-window columns of the large configuration
                // (optional: without them the windows walk per-source cursors)
                const int64_t maxf = (int64_t)c->hctr->max_flops;
                int64_t capb = (int64_t)(c->bucket_budget / ((size_t)g * 8));
                if (capb > maxf) capb = maxf;
                if (capb > (int64_t)1 << 30) capb = (int64_t)1 << 30;  // int32 bucket positions
                if (capb >= 1024 && ensure(c, c->bucket_row, (size_t)g * capb * 8, s) &&
                    ensure(c, c->woff, (size_t)g * 2 * (WINDOW_MAX + 1) * 4, s)) {
                    bq.bucket_row = (int32_t*)c->bucket_row.p;
                    bq.woff = (int32_t*)c->woff.p;
                    bq.bucket_cap = capb;
                }
            }
            launch_numeric(q, Av, pp, bq, g, s);
            ++used;
        }
        return check_launch(c, "numeric");
    };
    int64_t* colptr_out = nullptr;
    int32_t* row_out = nullptr;
    float* val_out = nullptr;
    int64_t nnz_out = 0;
    int phases = 1;
    if (!phased) {
        cudaEventRecord(c->ev[3], s);
        if ((st = run_numeric(b))) return st;
        cudaEventRecord(c->ev[4], s);
        launch_finalize_stats(A->n, b, s);
        // ---- output ----
        colptr_out = (int64_t*)dev_alloc(c, (size_t)(n + 1) * 8, s);
        if (!colptr_out) return fail(c, MCL_ERR_OOM, "output colptr allocation failed");
        if (active) launch_fill_inactive(Av, active, b.kept, s);  // carried columns keep their length
        launch_exclusive_scan<int32_t>(b.kept, n, colptr_out, b.scan_tmp, &b.ctr->nnz_out, s);
        if ((st = check_launch(c, "scan"))) {
            dev_free(c, colptr_out, s);
            return st;
        }
        cudaEventRecord(c->ev[5], s);
        if ((st = read_counters(c, s)) || (st = err_flags(c, c->hctr->err))) {
            dev_free(c, colptr_out, s);
            return st;
        }
        nnz_out = (int64_t)c->hctr->nnz_out;
        row_out = (int32_t*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
        val_out = (float*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
        if (!row_out || !val_out) {
            dev_free(c, colptr_out, s);
            dev_free(c, row_out, s);
            dev_free(c, val_out, s);
            return fail(c, MCL_ERR_OOM, "output allocation failed (nnz %lld)", (long long)nnz_out);
        }
        launch_compact(Av, b, colptr_out, row_out, val_out, s);
        if ((st = check_launch(c, "compact"))) return st;
    } else {
        // plan consecutive column batches whose capacities fit the staging budget
        std::vector<int64_t> hoff((size_t)n + 1);
        CUDA_TRY(c, cudaMemcpyAsync(hoff.data(), b.off, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        std::vector<int32_t> cut;
        cut.push_back(0);
        while (cut.back() < n) {
            const int32_t c0 = cut.back();
            int64_t lo = c0 + 1, hi = n;  // largest c1 with hoff[c1] - hoff[c0] <= budget
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) / 2;
                if (hoff[mid] - hoff[c0] <= budget_entries) lo = mid; else hi = mid - 1;
            }
            cut.push_back((int32_t)lo);
        }
        phases = (int)cut.size() - 1;
        if (!ensure(c, c->active, (size_t)n + 1, s) ||
            !ensure(c, c->phase_colptr, ((size_t)n + 2) * 8, s))
            return fail(c, MCL_ERR_OOM, "batch scratch allocation failed");
        uint8_t* mask = (uint8_t*)c->active.p;
        int64_t* pcol = (int64_t*)c->phase_colptr.p;
        std::vector<int32_t*> seg_row;
        std::vector<float*> seg_val;
        std::vector<int64_t> seg_nnz;
        auto free_segments = [&]() {
            for (size_t q = 0; q < seg_row.size(); ++q) {
                dev_free(c, seg_row[q], s);
                dev_free(c, seg_val[q], s);
            }
        };
        cudaEventRecord(c->ev[3], s);
        for (int ph = 0; ph < phases; ++ph) {
            const int32_t c0 = cut[ph], c1 = cut[ph + 1];
            launch_range_mask((int32_t)n, c0, c1, mask, s);
            ExpandBuffers bb = b;
            bb.active = mask;
            bb.tmp_off0 = hoff[c0];
            if ((st = run_numeric(bb))) {
                free_segments();
                return st;
            }
            launch_exclusive_scan<int32_t>(b.kept + c0, c1 - c0, pcol, b.scan_tmp, &b.ctr->nnz_out, s);
            if ((st = read_counters(c, s)) || (st = err_flags(c, c->hctr->err))) {
                free_segments();
                return st;
            }
            const int64_t nb = (int64_t)c->hctr->nnz_out;
            int32_t* r = (int32_t*)dev_alloc(c, (size_t)nb * 4 + 4, s);
            float* v = (float*)dev_alloc(c, (size_t)nb * 4 + 4, s);
            seg_row.push_back(r);
            seg_val.push_back(v);
            seg_nnz.push_back(nb);
            if (!r || !v) {
                free_segments();
                return fail(c, MCL_ERR_OOM, "batch output allocation failed");
            }
            launch_compact_range(Av, bb, c0, c1, pcol, r, v, s);
            if ((st = check_launch(c, "batch compact"))) {
                free_segments();
                return st;
            }
        }
        cudaEventRecord(c->ev[4], s);
        launch_finalize_stats(A->n, b, s);
        colptr_out = (int64_t*)dev_alloc(c, (size_t)(n + 1) * 8, s);
        if (!colptr_out) {
            free_segments();
            return fail(c, MCL_ERR_OOM, "output colptr allocation failed");
        }
        launch_exclusive_scan<int32_t>(b.kept, n, colptr_out, b.scan_tmp, &b.ctr->nnz_out, s);
        cudaEventRecord(c->ev[5], s);
        if ((st = read_counters(c, s)) || (st = err_flags(c, c->hctr->err))) {
            free_segments();
            dev_free(c, colptr_out, s);
            return st;
        }
        nnz_out = (int64_t)c->hctr->nnz_out;
        row_out = (int32_t*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
        val_out = (float*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
        if (!row_out || !val_out) {
            free_segments();
            dev_free(c, colptr_out, s);
            dev_free(c, row_out, s);
            dev_free(c, val_out, s);
            return fail(c, MCL_ERR_OOM, "output allocation failed (nnz %lld)", (long long)nnz_out);
        }
        // the batches are consecutive column ranges: their segments concatenate
        int64_t at = 0;
        for (size_t q = 0; q < seg_row.size(); ++q) {
            if (seg_nnz[q] > 0) {
                CUDA_TRY(c, cudaMemcpyAsync(row_out + at, seg_row[q], (size_t)seg_nnz[q] * 4,
                                            cudaMemcpyDeviceToDevice, s));
                CUDA_TRY(c, cudaMemcpyAsync(val_out + at, seg_val[q], (size_t)seg_nnz[q] * 4,
                                            cudaMemcpyDeviceToDevice, s));
            }
            at += seg_nnz[q];
        }
        free_segments();
        if (at != nnz_out) return fail(c, MCL_ERR_INTERNAL, "batch outputs do not add up");
    }
    cudaEventRecord(c->ev[6], s);
    out->n = A->n;
    out->nnz = nnz_out;
    out->colptr = colptr_out;
    out->rowidx = row_out;
    out->val = val_out;
    const double ch = chaos_from_bits(c->hctr->chaos_bits);
    if (chaos) *chaos = ch;
    // statistics (elapsed times up to the last synchronisation)
    mcl_stats& S = c->stats;
    S.flops = (int64_t)c->hctr->flops;
    S.nnz_in = A->nnz;
    S.nnz_b = (int64_t)c->hctr->nnz_b;
    S.nnz_out = nnz_out;
    S.estimator_misses = (int64_t)c->hctr->misses;
    S.range_splits = (int64_t)c->hctr->splits;
    S.chaos = ch;
    S.bins_used = used;
    S.phases = phases;
    cudaEventElapsedTime(&S.ms_colstats, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&S.ms_estimate, c->ev[1], c->ev[2]);
    cudaEventElapsedTime(&S.ms_bin, c->ev[2], c->ev[3]);
    cudaEventElapsedTime(&S.ms_numeric, c->ev[3], c->ev[4]);
    cudaEventElapsedTime(&S.ms_chaos, c->ev[4], c->ev[5]);
    cudaEventElapsedTime(&S.ms_total, c->ev[0], c->ev[5]);
    S.ms_compact = 0.0f;
    return MCL_OK;
}

mcl_status mcl_expand(mcl_ctx* c, const mcl_csc* A, const mcl_params* prm, mcl_csc* out,
                      double* chaos, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    return expand_impl(c, A, prm, out, chaos, (cudaStream_t)stream, nullptr);
}

// A partial (or merged) product: row-sorted columns of exact fixed-point sums.
struct Part {
    int64_t* colptr = nullptr;
    int32_t* rowidx = nullptr;
    unsigned long long* val = nullptr;
    int64_t nnz = 0;
};

static void free_part(mcl_ctx* c, Part& p, cudaStream_t s) {
    dev_free(c, p.colptr, s);
    dev_free(c, p.rowidx, s);
    dev_free(c, p.val, s);
    p = Part{};
}

mcl_status mcl_expand_split(mcl_ctx* c, const mcl_csc* A, const mcl_params* prm, int32_t nstages,
                            mcl_csc* out, double* chaos, mcl_merge_stats* stats, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    PruneParams pp;
    mcl_status st = check_params(c, prm, &pp, true);
    if (st) return st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (!out) return fail(c, MCL_ERR_INVALID, "out is NULL");
    if (nstages < 1 || nstages > MCL_SPLIT_MAX_STAGES)
        return fail(c, MCL_ERR_INVALID, "nstages must be in [1, %d]", MCL_SPLIT_MAX_STAGES);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int64_t n = A->n;
    if ((st = ensure_columns(c, n, s))) return st;
    ExpandBuffers b = buffers(c);
    const CscView Av = view(A);
    CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
    launch_colstats(Av, pp, b, c->num_sms, s);  // validation, column sums of A
    if ((st = read_counters(c, s))) return st;
    if ((st = err_flags(c, c->hctr->err))) return st;
    int64_t stride = (int64_t)c->hctr->max_deg;
    if (stride < MCL_SPLIT_MAX_PARTS) stride = MCL_SPLIT_MAX_PARTS;
    stride = (stride + 31) & ~31ll;
    const int grid_cap = 4 * c->num_sms;
    const size_t n1 = (size_t)n + 1;
    if (!ensure(c, c->split_bsum, n1 * 8, s) || !ensure(c, c->split_cnt, n1 * 8, s) ||
        !ensure(c, c->split_scratch, (size_t)grid_cap * 6 * stride * 8, s))
        return fail(c, MCL_ERR_OOM, "split scratch allocation failed");
    double* bsum = (double*)c->split_bsum.p;
    int64_t* cnt = (int64_t*)c->split_cnt.p;
    launch_bsum(Av, b.colsum, bsum, s);
    mcl_merge_stats ms{};
    ms.stages = nstages;
    std::vector<Part> stack;
    int64_t live = 0;
    auto fail_all = [&](mcl_status code, const char* what) {
        for (auto& p : stack) free_part(c, p, s);
        stack.clear();
        return code == MCL_ERR_OOM ? fail(c, code, "%s: out of device memory", what) : code;
    };
    // count, scan, allocate and fill one product (a stage or a merge)
    auto build = [&](RankArgs ra, bool stage, Part& P) -> mcl_status {
        ra.n = (int32_t)n;
        ra.scratch = c->split_scratch.p;
        ra.stride = stride;
        ra.grid_cap = grid_cap;
        ra.ctr = (DevCounters*)c->ctr.p;
        ra.nnz_out = cnt;
        launch_split_count(ra, stage, c->num_sms, s);
        P.colptr = (int64_t*)dev_alloc(c, n1 * 8, s);
        if (!P.colptr) return MCL_ERR_OOM;
        launch_exclusive_scan<int64_t>(cnt, n, P.colptr, b.scan_tmp, &b.ctr->cap_total, s);
        if (n == 0) cudaMemsetAsync(P.colptr, 0, 8, s);
        mcl_status e = read_counters(c, s);
        if (e) return e;
        if (c->hctr->err) return fail(c, MCL_ERR_INTERNAL, "split product raised flags");
        P.nnz = n > 0 ? (int64_t)c->hctr->cap_total : 0;
        P.rowidx = (int32_t*)dev_alloc(c, (size_t)P.nnz * 4 + 4, s);
        P.val = (unsigned long long*)dev_alloc(c, (size_t)P.nnz * 8 + 8, s);
        if (!P.rowidx || !P.val) return MCL_ERR_OOM;
        if (P.nnz > 0) {
            CUDA_TRY(c, cudaMemsetAsync(P.val, 0, (size_t)P.nnz * 8, s));
            ra.colptr_out = P.colptr;
            ra.row_out = P.rowidx;
            ra.val_out = P.val;
            launch_split_fill(ra, stage, c->num_sms, s);
        }
        return check_launch(c, "split product");
    };
    auto merge_top = [&](int count) -> mcl_status {
        RankArgs ra{};
        ra.nparts = count;
        int64_t in = 0;
        for (int q = 0; q < count; ++q) {
            const Part& p = stack[stack.size() - 1 - q];
            ra.pcol[q] = p.colptr;
            ra.prow[q] = p.rowidx;
            ra.pval[q] = p.val;
            in += p.nnz;
        }
        Part M;
        mcl_status e = build(ra, false, M);
        if (e) {
            free_part(c, M, s);
            return e;
        }
        ms.binary_peak_entries = in > ms.binary_peak_entries ? in : ms.binary_peak_entries;
        live += M.nnz;
        ms.live_peak_entries = live > ms.live_peak_entries ? live : ms.live_peak_entries;
        for (int q = 0; q < count; ++q) {
            free_part(c, stack.back(), s);
            stack.pop_back();
        }
        live -= in;
        stack.push_back(M);
        ++ms.merges;
        return MCL_OK;
    };
    for (int t = 1; t <= nstages; ++t) {
        RankArgs ra{};
        ra.A = Av;
        ra.k0 = (int32_t)((int64_t)(t - 1) * n / nstages);
        ra.k1 = (int32_t)((int64_t)t * n / nstages);
        ra.bsum = bsum;
        Part P;
        st = build(ra, true, P);
        if (st) {
            free_part(c, P, s);
            return fail_all(st, "split stage failed");
        }
        ms.partial_entries += P.nnz;
        stack.push_back(P);
        live += P.nnz;
        ms.live_peak_entries = live > ms.live_peak_entries ? live : ms.live_peak_entries;
        // Algorithm 2: merge the top nmerges + 1 lists, nmerges = times t halves evenly
        int nm = 0;
        for (int jj = t; jj != 0 && (jj % 2) == 0; jj /= 2) ++nm;
        if (nm > 0) {
            int count = nm + 1 > (int)stack.size() ? (int)stack.size() : nm + 1;
            while (count > 1) {  // more lists than one merge takes: merge in runs
                const int take = count < MCL_SPLIT_MAX_PARTS ? count : MCL_SPLIT_MAX_PARTS;
                if ((st = merge_top(take))) return fail_all(st, "merge failed");
                count -= take - 1;
            }
        }
    }
    while (stack.size() > 1) {  // lists left when nstages is not a power of two
        const int take = (int)stack.size() < MCL_SPLIT_MAX_PARTS ? (int)stack.size() : MCL_SPLIT_MAX_PARTS;
        if ((st = merge_top(take))) return fail_all(st, "merge failed");
    }
    Part B = stack.back();
    stack.clear();
    ms.merged_entries = B.nnz;
    // ---- the prune rule, inflation and renormalisation of the merged product ----
    const CscView Bv{A->n, B.nnz, B.colptr, B.rowidx, nullptr};
    CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
    launch_prune_cap(Bv, pp.Krec, b, s);
    launch_exclusive_scan<int64_t>(b.cap, n, b.off, b.scan_tmp, &b.ctr->cap_total, s);
    if ((st = read_counters(c, s))) {
        free_part(c, B, s);
        return st;
    }
    const int64_t cap_total = (int64_t)c->hctr->cap_total;
    if (!ensure(c, c->tmp_row, (size_t)cap_total * 4 + 4, s) ||
        !ensure(c, c->tmp_val, (size_t)cap_total * 4 + 4, s)) {
        free_part(c, B, s);
        return fail(c, MCL_ERR_OOM, "scratch allocation failed");
    }
    b.tmp_row = (int32_t*)c->tmp_row.p;
    b.tmp_val = (float*)c->tmp_val.p;
    b.tmp_off0 = 0;
    launch_prune_fixed((int32_t)n, B.colptr, B.rowidx, B.val, bsum, pp, b, c->num_sms, s);
    launch_finalize_stats((int32_t)n, b, s);
    int64_t* colptr_out = (int64_t*)dev_alloc(c, n1 * 8, s);
    if (!colptr_out) {
        free_part(c, B, s);
        return fail(c, MCL_ERR_OOM, "output colptr allocation failed");
    }
    launch_exclusive_scan<int32_t>(b.kept, n, colptr_out, b.scan_tmp, &b.ctr->nnz_out, s);
    if (n == 0) cudaMemsetAsync(colptr_out, 0, 8, s);
    if ((st = read_counters(c, s)) || (st = err_flags(c, c->hctr->err))) {
        free_part(c, B, s);
        dev_free(c, colptr_out, s);
        return st;
    }
    const int64_t nnz_out = n > 0 ? (int64_t)c->hctr->nnz_out : 0;
    int32_t* row_out = (int32_t*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
    float* val_out = (float*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
    if (!row_out || !val_out) {
        free_part(c, B, s);
        dev_free(c, colptr_out, s);
        dev_free(c, row_out, s);
        dev_free(c, val_out, s);
        return fail(c, MCL_ERR_OOM, "output allocation failed");
    }
    launch_compact(CscView{A->n, nnz_out, colptr_out, nullptr, nullptr}, b, colptr_out, row_out,
                   val_out, s);
    if ((st = check_launch(c, "split output"))) {
        free_part(c, B, s);
        return st;
    }
    CUDA_TRY(c, cudaStreamSynchronize(s));
    free_part(c, B, s);
    out->n = A->n;
    out->nnz = nnz_out;
    out->colptr = colptr_out;
    out->rowidx = row_out;
    out->val = val_out;
    if (chaos) *chaos = chaos_from_bits(c->hctr->chaos_bits);
    if (stats) *stats = ms;
    return MCL_OK;
}

mcl_status mcl_symbolic(mcl_ctx* c, const mcl_csc* A, int64_t* flops, int64_t* nnz_out,
                        void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A, "A"))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int64_t n = A->n;
    if ((st = ensure_columns(c, n, s))) return st;
    ExpandBuffers b = buffers(c);
    const CscView Av = view(A);
    PruneParams pp{};
    pp.Krec = 1;
    CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
    launch_colstats(Av, pp, b, c->num_sms, s);
    if ((st = read_counters(c, s))) return st;
    if ((st = err_flags(c, c->hctr->err))) return st;
    b.cur_stride = ((c->hctr->max_deg + 31) & ~31) + 32;
    const int grid = symbolic_grid(c->num_sms);
    if (!ensure(c, c->cursors, (size_t)grid * 6 * b.cur_stride * 4, s))
        return fail(c, MCL_ERR_OOM, "cursor scratch allocation failed");
    b.cursors = (int32_t*)c->cursors.p;
    if (nnz_out) launch_symbolic(Av, b, nnz_out, c->num_sms, grid, s);
    if (flops && n > 0)
        CUDA_TRY(c, cudaMemcpyAsync(flops, b.flops, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    return check_launch(c, "symbolic");
}

mcl_status mcl_prune_select_recover(mcl_ctx* c, const mcl_csc* B, const mcl_params* prm,
                                    mcl_csc* out, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    PruneParams pp;
    mcl_status st = check_params(c, prm, &pp, false);
    if (st) return st;
    pp.inflate = 0;
    if ((st = check_csc(c, B, "B"))) return st;
    if (!out) return fail(c, MCL_ERR_INVALID, "out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int64_t n = B->n;
    if ((st = ensure_columns(c, n, s))) return st;
    ExpandBuffers b = buffers(c);
    const CscView Bv = view(B);
    CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
    launch_colstats(Bv, pp, b, c->num_sms, s);  // validation
    if ((st = read_counters(c, s))) return st;
    if ((st = err_flags(c, c->hctr->err))) return st;
    launch_prune_cap(Bv, pp.Krec, b, s);
    launch_exclusive_scan<int64_t>(b.cap, n, b.off, b.scan_tmp, &b.ctr->cap_total, s);
    if ((st = read_counters(c, s))) return st;
    const int64_t cap_total = (int64_t)c->hctr->cap_total;
    if (!ensure(c, c->tmp_row, (size_t)cap_total * 4 + 4, s) ||
        !ensure(c, c->tmp_val, (size_t)cap_total * 4 + 4, s))
        return fail(c, MCL_ERR_OOM, "scratch allocation failed");
    b.tmp_row = (int32_t*)c->tmp_row.p;
    b.tmp_val = (float*)c->tmp_val.p;
    launch_prune(Bv, pp, b, c->num_sms, s);
    if ((st = check_launch(c, "prune"))) return st;
    int64_t* colptr_out = (int64_t*)dev_alloc(c, (size_t)(n + 1) * 8, s);
    if (!colptr_out) return fail(c, MCL_ERR_OOM, "output colptr allocation failed");
    launch_exclusive_scan<int32_t>(b.kept, n, colptr_out, b.scan_tmp, &b.ctr->nnz_out, s);
    if ((st = read_counters(c, s)) || (st = err_flags(c, c->hctr->err))) {
        dev_free(c, colptr_out, s);
        return st;
    }
    const int64_t nnz_out = (int64_t)c->hctr->nnz_out;
    int32_t* row_out = (int32_t*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
    float* val_out = (float*)dev_alloc(c, (size_t)nnz_out * 4 + 4, s);
    if (!row_out || !val_out) {
        dev_free(c, colptr_out, s);
        dev_free(c, row_out, s);
        dev_free(c, val_out, s);
        return fail(c, MCL_ERR_OOM, "output allocation failed");
    }
    launch_compact(Bv, b, colptr_out, row_out, val_out, s);
    if ((st = check_launch(c, "compact"))) return st;
    out->n = B->n;
    out->nnz = nnz_out;
    out->colptr = colptr_out;
    out->rowidx = row_out;
    out->val = val_out;
    return MCL_OK;
}

mcl_status mcl_inflate_normalize(mcl_ctx* c, mcl_csc* A, float r, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (!(r > 0.0f && r <= 1.0e6f)) return fail(c, MCL_ERR_INVALID, "inflation must be > 0");
    CUDA_TRY(c, cudaSetDevice(c->device));
    launch_inflate_normalize(A->n, A->colptr, A->val, r, (cudaStream_t)stream);
    return check_launch(c, "inflate_normalize");
}

mcl_status mcl_chaos(mcl_ctx* c, const mcl_csc* A, double* chaos, double* chaos_cols,
                     void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (!chaos) return fail(c, MCL_ERR_INVALID, "chaos is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (!ensure(c, c->ctr, sizeof(DevCounters), s)) return fail(c, MCL_ERR_OOM, "scratch");
    DevCounters* ctr = (DevCounters*)c->ctr.p;
    CUDA_TRY(c, cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s));
    launch_chaos(A->n, A->colptr, A->val, chaos_cols, ctr, s);
    if ((st = check_launch(c, "chaos"))) return st;
    if ((st = read_counters(c, s))) return st;
    *chaos = chaos_from_bits(c->hctr->chaos_bits);
    return MCL_OK;
}

mcl_status mcl_components(mcl_ctx* c, const mcl_csc* A, int32_t* labels, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (A->n > 0 && !labels) return fail(c, MCL_ERR_INVALID, "labels is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (!ensure(c, c->ctr, sizeof(DevCounters), s)) return fail(c, MCL_ERR_OOM, "scratch");
    DevCounters* ctr = (DevCounters*)c->ctr.p;
    CUDA_TRY(c, cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s));
    launch_components(view(A), labels, ctr, s);
    if ((st = check_launch(c, "components"))) return st;
    if ((st = read_counters(c, s))) return st;
    return err_flags(c, c->hctr->err);
}

mcl_status mcl_estimator_load(mcl_ctx* c, const uint16_t* w, const float* norm, float safety) {
    if (!c) return MCL_ERR_INVALID;
    if (!w || !norm) return fail(c, MCL_ERR_INVALID, "weights / norm is NULL");
    if (!(safety >= 0.01f && safety <= 1000.0f)) return fail(c, MCL_ERR_INVALID, "bad safety");
    for (int i = 0; i < MCL_NFEATURES; ++i)
        if (!(norm[MCL_NFEATURES + i] > 0.0f)) return fail(c, MCL_ERR_INVALID, "sigma must be > 0");
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (!ensure(c, c->mlp_w, MCL_MLP_NPARAM * 2, 0) ||
        !ensure(c, c->mlp_norm, 2 * MCL_NFEATURES * 4, 0))
        return fail(c, MCL_ERR_OOM, "estimator allocation failed");
    CUDA_TRY(c, cudaMemcpy(c->mlp_w.p, w, MCL_MLP_NPARAM * 2, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->mlp_norm.p, norm, 2 * MCL_NFEATURES * 4, cudaMemcpyHostToDevice));
    c->est_safety = safety;
    c->has_estimator = 1;
    return MCL_OK;
}

mcl_status mcl_features(mcl_ctx* c, const mcl_csc* A, int32_t iteration, const float* prev_logcf,
                        float* feats, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (A->n > 0 && !feats) return fail(c, MCL_ERR_INVALID, "feats is NULL");
    if (iteration < 1) return fail(c, MCL_ERR_INVALID, "iteration must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (!ensure(c, c->colmax, ((size_t)A->n + 1) * 4, s)) return fail(c, MCL_ERR_OOM, "scratch");
    launch_colmax_features(view(A), iteration, prev_logcf, (float*)c->colmax.p, feats, s);
    return check_launch(c, "features");
}

mcl_status mcl_mlp_forward(mcl_ctx* c, const float* feats, int64_t n, const uint16_t* w,
                           const float* norm, float* out, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    if (n < 0 || (n > 0 && (!feats || !w || !norm || !out)))
        return fail(c, MCL_ERR_INVALID, "bad forward arguments");
    CUDA_TRY(c, cudaSetDevice(c->device));
    launch_mlp_forward(feats, n, w, norm, out, nullptr, 1.0f, nullptr, nullptr, nullptr,
                       (cudaStream_t)stream);
    return check_launch(c, "mlp_forward");
}

mcl_status mcl_mlp_backward(mcl_ctx* c, const float* feats, const float* targets, int64_t n,
                            const uint16_t* w, const float* norm, float scale, float* grad,
                            double* loss, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    if (n < 0 || (n > 0 && (!feats || !targets || !w || !norm || !grad || !loss)))
        return fail(c, MCL_ERR_INVALID, "bad backward arguments");
    CUDA_TRY(c, cudaSetDevice(c->device));
    launch_mlp_backward(feats, targets, n, w, norm, scale, grad, loss, (cudaStream_t)stream);
    return check_launch(c, "mlp_backward");
}

mcl_status mcl_adam_step(mcl_ctx* c, float* master, float* m, float* v, const float* grad,
                         int64_t step, float lr, float beta1, float beta2, float eps,
                         uint16_t* w, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    if (!master || !m || !v || !grad || !w || step < 1)
        return fail(c, MCL_ERR_INVALID, "bad adam arguments");
    CUDA_TRY(c, cudaSetDevice(c->device));
    launch_adam(master, m, v, grad, step, lr, beta1, beta2, eps, w, (cudaStream_t)stream);
    return check_launch(c, "adam");
}

mcl_status mcl_estimate(mcl_ctx* c, const mcl_csc* A, int64_t* est, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (!c->has_estimator) return fail(c, MCL_ERR_INVALID, "no estimator loaded");
    if (A->n > 0 && !est) return fail(c, MCL_ERR_INVALID, "est is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    if ((st = ensure_columns(c, A->n, s))) return st;
    ExpandBuffers b = buffers(c);
    PruneParams pp{};
    pp.Krec = 1;
    CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
    launch_colstats(view(A), pp, b, c->num_sms, s);
    if ((st = read_counters(c, s))) return st;
    if ((st = err_flags(c, c->hctr->err))) return st;
    b.est = est;
    return internal_estimate(c, A, b, s);
}

mcl_status mcl_cohen_estimate(mcl_ctx* c, const mcl_csc* A, int32_t keys, uint64_t seed, float* est,
                              void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A, "A"))) return st;
    if (keys < 2 || keys > cohen_max_r())
        return fail(c, MCL_ERR_INVALID, "keys must be in [2, %d]", cohen_max_r());
    if (A->n > 0 && !est) return fail(c, MCL_ERR_INVALID, "est is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaSetDevice(c->device));
    if ((st = ensure_columns(c, A->n, s))) return st;
    // validation pass: the estimate indexes by row, so a malformed A is refused first
    ExpandBuffers b = buffers(c);
    PruneParams pp{};
    pp.Krec = 1;
    CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
    launch_colstats(view(A), pp, b, c->num_sms, s);
    if ((st = read_counters(c, s))) return st;
    if ((st = err_flags(c, c->hctr->err))) return st;
    if (!ensure(c, c->cohen_m, ((size_t)A->n + 1) * keys * 4, s))
        return fail(c, MCL_ERR_OOM, "estimator scratch allocation failed");
    launch_cohen(view(A), keys, seed, (float*)c->cohen_m.p, est, s);
    return check_launch(c, "cohen");
}

static void free_csc(mcl_ctx* c, mcl_csc* M, cudaStream_t s) {
    dev_free(c, M->colptr, s);
    dev_free(c, M->rowidx, s);
    dev_free(c, M->val, s);
    M->colptr = nullptr;
    M->rowidx = nullptr;
    M->val = nullptr;
}

// ---------------------------------------------------------------------------
// Batched iterations replayed as CUDA graphs.  After the first iteration
// every column of an active component holds at most K_rec entries, so one
// iteration needs no host decision: the replay buffers (two CSC matrices
// and the output staging, each of `cap` entries) are allocated once and the
// iteration X -> Y and its mirror Y -> X are captured.  One replay is every
// kernel of an iteration plus a copy of the device counters to the host,
// the only synchronisation.  If an iteration's output capacities exceed the
// buffers, a device guard makes the numeric pass and the compaction write
// nothing (ERR_STAGING) and the host redoes the iteration without graphs.
// ---------------------------------------------------------------------------
struct GraphRun {
    cudaStream_t gs = nullptr;
    cudaGraph_t g[2] = {nullptr, nullptr};
    cudaGraphExec_t x[2] = {nullptr, nullptr};
    mcl_csc buf[2] = {};
    int64_t cap = 0;
    int64_t kernels = 0;  // kernel nodes per replay
};

static void graph_release(mcl_ctx* c, GraphRun& G, cudaStream_t s, int keep) {
    for (int q = 0; q < 2; ++q) {
        if (G.x[q]) cudaGraphExecDestroy(G.x[q]);
        if (G.g[q]) cudaGraphDestroy(G.g[q]);
        G.x[q] = nullptr;
        G.g[q] = nullptr;
        if (q != keep) free_csc(c, &G.buf[q], s);
    }
    if (G.gs) {
        cudaStreamSynchronize(G.gs);
        cudaStreamDestroy(G.gs);
        G.gs = nullptr;
    }
}

// One batched iteration in -> out on stream s: kernel launches and memsets
// only (capturable).  in.nnz is read as a capacity bound.
static void static_iteration(mcl_ctx* c, const mcl_params* prm, const PruneParams& pp, int ncomp,
                             const mcl_csc& in, const mcl_csc& out, int64_t cap, int sizing,
                             int64_t stride, cudaStream_t s) {
    const int32_t n = in.n;
    ExpandBuffers b = buffers(c);
    b.active = (const uint8_t*)c->active.p;
    b.nnz_is_bound = 1;
    b.cur_stride = stride;
    b.tmp_off0 = 0;
    const CscView Av{n, in.nnz, in.colptr, in.rowidx, in.val};
    cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s);
    launch_active_from_comp(n, (const int32_t*)c->comp_of_col.p, (const uint8_t*)c->comp_active.p,
                            (uint8_t*)c->active.p, s);
    launch_colstats(Av, pp, b, c->num_sms, s);
    const int grid_max = max_numeric_grid(c, pp);
    if (sizing == 1) {
        launch_est_from_flops(Av, b, s);
    } else if (sizing == 2) {  // learned: features (iteration index on the device) -> MLP
        launch_colmax_features(Av, 0, (const float*)c->prev_logcf.p, (float*)c->colmax.p,
                               (float*)c->feats.p, s, (const int32_t*)c->iter_dev.p);
        launch_mlp_forward((const float*)c->feats.p, n, (const uint16_t*)c->mlp_w.p,
                           (const float*)c->mlp_norm.p, nullptr, b.est, c->est_safety, b.flops,
                           b.rlo, b.rhi, s);
    } else if (sizing == 3) {
        launch_cohen(Av, c->cohen_r, c->cohen_seed, (float*)c->cohen_m.p, (float*)c->cohen_e.p, s);
        launch_cohen_to_est(n, (const float*)c->cohen_e.p, 1.0f, b, s);
    } else {
        launch_symbolic(Av, b, b.est, c->num_sms, grid_max, s);
        launch_cap_tighten(n, b.est, b.cap, b.active, s);
    }
    if (c->est_milli != 1000) launch_scale_est(n, b.est, c->est_milli, s);
    launch_exclusive_scan<int64_t>(b.cap, n, b.off, b.scan_tmp, &b.ctr->cap_total, s);
    launch_staging_guard(b.ctr, cap, s);
    launch_binning(Av, pp, b, c->conf_mask, s);
    for (int q = NCONF - 1; q >= 0; --q) {
        if (!((c->conf_mask >> q) & 1)) continue;
        const int g = numeric_grid(q, pp, c->num_sms);
        ExpandBuffers bq = b;
        if (q == NCONF - 1 && c->bucket_row.p) {
            bq.bucket_row = (int32_t*)c->bucket_row.p;
            bq.woff = (int32_t*)c->woff.p;
            bq.bucket_cap = (int64_t)(c->bucket_row.bytes / ((size_t)g * 8));
            if (bq.bucket_cap > (int64_t)1 << 30) bq.bucket_cap = (int64_t)1 << 30;
        }
        launch_numeric(q, Av, pp, bq, g, s);
    }
    launch_finalize_stats(n, b, s);
    launch_fill_inactive(Av, b.active, b.kept, s);
    launch_exclusive_scan<int32_t>(b.kept, n, out.colptr, b.scan_tmp, &b.ctr->nnz_out, s);
    launch_compact(Av, b, out.colptr, out.rowidx, out.val, s);
    cudaMemsetAsync(c->comp_bits.p, 0, (size_t)ncomp * 8, s);
    launch_comp_chaos(n, (const int32_t*)c->comp_of_col.p, b.active, b.chaos,
                      (unsigned long long*)c->comp_bits.p, s);
    launch_comp_retire(ncomp, (const unsigned long long*)c->comp_bits.p, prm->chaos_eps,
                       (uint8_t*)c->comp_active.p, b.ctr, s);
    if (sizing == 2) {  // this iteration's compression factors feed the next one's features
        launch_logcf(n, b.flops, b.bnnz, (float*)c->prev_logcf.p, s);
        launch_iter_bump((int32_t*)c->iter_dev.p, s);
    }
    launch_copy_counters((const DevCounters*)c->ctr.p, c->hctr_dev, s);
}

// Allocates the replay buffers, moves `cur` (the output of the first
// iteration, owned) into the first one and captures both graphs.
static mcl_status graph_prepare(mcl_ctx* c, const mcl_params* prm, const PruneParams& pp,
                                const int32_t* comp_offsets, int ncomp, mcl_csc* cur, int sizing,
                                GraphRun& G, cudaStream_t s) {
    const int32_t n = cur->n;
    int64_t cap = 0;  // entries of an iteration's output: column j keeps <= min(K_rec, |comp(j)|)
    for (int q = 0; q < ncomp; ++q) {
        const int64_t sz = comp_offsets[q + 1] - comp_offsets[q];
        cap += sz * (sz < pp.Krec ? sz : pp.Krec);
    }
    if (c->graph_cap > 0 && c->graph_cap < cap) cap = c->graph_cap;
    if (cap < cur->nnz) cap = cur->nnz;
    if (cap < 1) cap = 1;
    int64_t stride = ((int64_t)pp.Krec + 31) & ~31ll;
    if (stride < 32) stride = 32;
    const int grid_max = max_numeric_grid(c, pp);
    const int g1 = numeric_grid(NCONF - 1, pp, c->num_sms);
    int64_t capb = (int64_t)pp.Krec * pp.Krec;
    const int64_t capb_max = (int64_t)(c->bucket_budget / ((size_t)g1 * 8));
    if (capb > capb_max) capb = capb_max;
    const size_t n1 = (size_t)n + 1;
    if (!ensure(c, c->tmp_row, (size_t)cap * 4 + 4, s) || !ensure(c, c->tmp_val, (size_t)cap * 4 + 4, s) ||
        !ensure(c, c->cursors, (size_t)grid_max * 6 * stride * 4, s) ||
        !ensure(c, c->comp_bits, (size_t)ncomp * 8, s))
        return fail(c, MCL_ERR_OOM, "graph replay scratch allocation failed");
    if (sizing == 2) {
        if (!c->has_estimator) return fail(c, MCL_ERR_INVALID, "use_estimator set but no estimator loaded");
        if (!ensure(c, c->colmax, n1 * 4, s) || !ensure(c, c->feats, n1 * 4 * MCL_NFEATURES, s) ||
            !ensure(c, c->prev_logcf, n1 * 4, s) || !ensure(c, c->iter_dev, 4, s))
            return fail(c, MCL_ERR_OOM, "estimator scratch allocation failed");
        // the first replay is iteration 2; the logs of cf of iteration 1 are in prev_logcf
        const int32_t it2 = 2;
        CUDA_TRY(c, cudaMemcpyAsync(c->iter_dev.p, &it2, 4, cudaMemcpyHostToDevice, s));
    } else if (sizing == 3) {
        if (!ensure(c, c->cohen_m, n1 * c->cohen_r * 4, s) || !ensure(c, c->cohen_e, n1 * 4, s))
            return fail(c, MCL_ERR_OOM, "estimator scratch allocation failed");
    }
    if (capb >= 1024 && ensure(c, c->bucket_row, (size_t)g1 * capb * 8, s) &&
        ensure(c, c->woff, (size_t)g1 * 2 * (WINDOW_MAX + 1) * 4, s)) {
        // exact per-CTA capacity recorded in the buffer sizes
        c->bucket_row.bytes = (size_t)g1 * capb * 8;
    } else {
        dev_free(c, c->bucket_row.p, s);
        c->bucket_row = Buf{};
    }
    for (int q = 0; q < 2; ++q) {
        G.buf[q].n = n;
        G.buf[q].nnz = cap;
        G.buf[q].colptr = (int64_t*)dev_alloc(c, ((size_t)n + 1) * 8, s);
        G.buf[q].rowidx = (int32_t*)dev_alloc(c, (size_t)cap * 4 + 4, s);
        G.buf[q].val = (float*)dev_alloc(c, (size_t)cap * 4 + 4, s);
        if (!G.buf[q].colptr || !G.buf[q].rowidx || !G.buf[q].val) {
            for (int r = 0; r <= q; ++r) free_csc(c, &G.buf[r], s);
            return fail(c, MCL_ERR_OOM, "graph replay buffers (%lld entries) do not fit", (long long)cap);
        }
    }
    CUDA_TRY(c, cudaMemcpyAsync(G.buf[0].colptr, cur->colptr, ((size_t)n + 1) * 8,
                                cudaMemcpyDeviceToDevice, s));
    if (cur->nnz > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(G.buf[0].rowidx, cur->rowidx, (size_t)cur->nnz * 4,
                                    cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(c, cudaMemcpyAsync(G.buf[0].val, cur->val, (size_t)cur->nnz * 4,
                                    cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(c, cudaStreamSynchronize(s));
    free_csc(c, cur, s);
    CUDA_TRY(c, cudaStreamCreateWithFlags(&G.gs, cudaStreamNonBlocking));
    G.cap = cap;
    const long long l0 = launches_total();
    for (int q = 0; q < 2; ++q) {
        CUDA_TRY(c, cudaStreamBeginCapture(G.gs, cudaStreamCaptureModeRelaxed));
        static_iteration(c, prm, pp, ncomp, G.buf[q], G.buf[q ^ 1], cap, sizing, stride, G.gs);
        CUDA_TRY(c, cudaStreamEndCapture(G.gs, &G.g[q]));
        CUDA_TRY(c, cudaGraphInstantiate(&G.x[q], G.g[q], 0));
    }
    const long long captured = launches_total() - l0;
    count_launches((int)-captured);  // captured launches run at replay time
    G.kernels = captured / 2;
    return MCL_OK;
}

// Device bytes a batched run of one component of `size` vertices may need:
// the two graph replay buffers and the output staging (8 bytes per entry of
// size * min(size, K_rec) each), the first iteration's output, and the
// per-column scratch.
static int64_t group_cost(int64_t size, int32_t krec) {
    return 32 * size * (size < krec ? size : krec) + 160 * size;
}

// A batched run split into consecutive groups of whole components whose
// costs fit the group budget: each group is copied out as a matrix of its
// own (rows re-based), run to its own convergence by mcl_run, and its labels
// (and final block) are placed back.  The components are independent, so
// the result is the one of a single run.
static mcl_status run_groups(mcl_ctx* c, const mcl_csc* A0, const int32_t* offs,
                             const std::vector<int32_t>& gcut, const mcl_params* prm,
                             int32_t* labels, int32_t* iters, double* chaos_hist,
                             mcl_csc* final_out, cudaStream_t s) {
    const int ngroups = (int)gcut.size() - 1;
    std::vector<double> hist_g((size_t)prm->max_iters, 0.0);
    if (chaos_hist)
        for (int i = 0; i < prm->max_iters; ++i) chaos_hist[i] = 0.0;
    struct Part {
        int32_t lo, ng;
        mcl_csc fin;
    };
    std::vector<Part> parts;
    auto free_parts = [&]() {
        for (auto& p : parts) free_csc(c, &p.fin, s);
        parts.clear();
    };
    int it_max = 0, replays = 0;
    bool converged = true;
    mcl_status st = MCL_OK;
    for (int g = 0; g < ngroups; ++g) {
        const int32_t c0 = gcut[g], c1 = gcut[g + 1];
        const int32_t lo = offs[c0], hi = offs[c1], ng = hi - lo;
        int64_t pp[2] = {0, 0};
        CUDA_TRY(c, cudaMemcpyAsync(&pp[0], A0->colptr + lo, 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaMemcpyAsync(&pp[1], A0->colptr + hi, 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        mcl_csc sub{ng, pp[1] - pp[0], nullptr, nullptr, A0->val ? A0->val + pp[0] : nullptr};
        sub.colptr = (int64_t*)dev_alloc(c, ((size_t)ng + 1) * 8, s);
        sub.rowidx = (int32_t*)dev_alloc(c, (size_t)sub.nnz * 4 + 4, s);
        if (!sub.colptr || !sub.rowidx) {
            dev_free(c, sub.colptr, s);
            dev_free(c, sub.rowidx, s);
            free_parts();
            return fail(c, MCL_ERR_OOM, "group %d of %d: copy allocation failed", g, ngroups);
        }
        launch_block_colptr(A0->colptr, lo, ng, sub.colptr, s);
        launch_add_i32(A0->rowidx + pp[0], sub.nnz, -lo, sub.rowidx, s);
        std::vector<int32_t> offs_g((size_t)(c1 - c0) + 1);
        for (int32_t q = c0; q <= c1; ++q) offs_g[q - c0] = offs[q] - lo;
        int32_t it_g = 0;
        Part part{lo, ng, mcl_csc{}};
        c->in_group = 1;
        st = mcl_run(c, &sub, offs_g.data(), c1 - c0, prm, labels + lo, &it_g, hist_g.data(),
                     final_out ? &part.fin : nullptr, (void*)s);
        c->in_group = 0;
        dev_free(c, sub.colptr, s);
        dev_free(c, sub.rowidx, s);
        if (st != MCL_OK && st != MCL_ERR_NOT_CONVERGED) {
            free_parts();
            return st;
        }
        if (st == MCL_ERR_NOT_CONVERGED) converged = false;
        launch_add_i32(labels + lo, ng, lo, labels + lo, s);  // group-local labels -> global
        it_max = it_g > it_max ? it_g : it_max;
        if (chaos_hist)
            for (int i = 0; i < it_g; ++i) chaos_hist[i] = hist_g[i] > chaos_hist[i] ? hist_g[i] : chaos_hist[i];
        replays += c->stats.graph_replays;
        if (final_out) parts.push_back(part);
    }
    if (final_out) {
        int64_t total = 0;
        for (auto& p : parts) total += p.fin.nnz;
        mcl_csc F{A0->n, total, nullptr, nullptr, nullptr};
        F.colptr = (int64_t*)dev_alloc(c, ((size_t)A0->n + 1) * 8, s);
        F.rowidx = (int32_t*)dev_alloc(c, (size_t)total * 4 + 4, s);
        F.val = (float*)dev_alloc(c, (size_t)total * 4 + 4, s);
        if (!F.colptr || !F.rowidx || !F.val) {
            free_csc(c, &F, s);
            free_parts();
            return fail(c, MCL_ERR_OOM, "final matrix allocation failed");
        }
        int64_t base = 0;
        for (size_t q = 0; q < parts.size(); ++q) {
            const Part& p = parts[q];
            launch_place_colptr(p.fin.colptr, p.lo, p.ng, base, q + 1 == parts.size(), F.colptr, s);
            launch_add_i32(p.fin.rowidx, p.fin.nnz, p.lo, F.rowidx + base, s);
            if (p.fin.nnz > 0)
                CUDA_TRY(c, cudaMemcpyAsync(F.val + base, p.fin.val, (size_t)p.fin.nnz * 4,
                                            cudaMemcpyDeviceToDevice, s));
            base += p.fin.nnz;
        }
        if (parts.empty()) launch_fill_colptr(A0->n, F.colptr, s);
        free_parts();
        *final_out = F;
    }
    if ((st = check_launch(c, "group placement"))) return st;
    c->stats.iterations = it_max;
    c->stats.graph_replays = replays;
    c->stats.groups = ngroups;
    if (iters) *iters = it_max;
    if (!converged) return fail(c, MCL_ERR_NOT_CONVERGED, "max_iters reached in a group");
    return MCL_OK;
}

mcl_status mcl_run(mcl_ctx* c, const mcl_csc* A0, const int32_t* comp_offsets, int32_t ncomp,
                   const mcl_params* prm, int32_t* labels, int32_t* iters, double* chaos_hist,
                   mcl_csc* final_out, void* stream) {
    if (!c) return MCL_ERR_INVALID;
    mcl_status st;
    if ((st = check_csc(c, A0, "A0"))) return st;
    if (!prm || prm->max_iters < 1) return fail(c, MCL_ERR_INVALID, "max_iters must be >= 1");
    if (A0->n > 0 && !labels) return fail(c, MCL_ERR_INVALID, "labels is NULL");
    if (comp_offsets && ncomp < 1) return fail(c, MCL_ERR_INVALID, "ncomp must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const bool batched = comp_offsets && prm->batched;
    if (comp_offsets) {
        if (comp_offsets[0] != 0 || comp_offsets[ncomp] != A0->n)
            return fail(c, MCL_ERR_INVALID, "comp_offsets must run from 0 to n");
        for (int q = 0; q < ncomp; ++q)
            if (comp_offsets[q + 1] < comp_offsets[q])
                return fail(c, MCL_ERR_INVALID, "comp_offsets must be nondecreasing");
    }
    if (!c->in_group) {
        c->stats.groups = 1;
        c->stats.flops_run = 0;
        c->stats.alg_bytes_run = 0;
    }
    if (comp_offsets) {
        CUDA_TRY(c, cudaSetDevice(c->device));
        if (c->group_budget > 0 && !c->in_group) {
            // consecutive groups of whole components within the budget
            PruneParams gp;
            mcl_status pst = check_params(c, prm, &gp, true);
            if (pst) return pst;
            std::vector<int32_t> gcut{0};
            int64_t used = 0;
            for (int q = 0; q < ncomp; ++q) {
                const int64_t cost = group_cost(comp_offsets[q + 1] - comp_offsets[q], gp.Krec);
                if (q > gcut.back() && used + cost > (int64_t)c->group_budget) {
                    gcut.push_back(q);
                    used = 0;
                }
                used += cost;
            }
            gcut.push_back(ncomp);
            if (gcut.size() > 2)
                return run_groups(c, A0, comp_offsets, gcut, prm, labels, iters, chaos_hist,
                                  final_out, s);
        }
    }
    if (batched) {
        const size_t n1 = (size_t)A0->n + 1;
        if (!ensure(c, c->comp_off, (size_t)(ncomp + 1) * 4, s) ||
            !ensure(c, c->comp_of_col, n1 * 4, s) || !ensure(c, c->comp_bits, (size_t)ncomp * 8, s) ||
            !ensure(c, c->comp_active, (size_t)ncomp, s) || !ensure(c, c->active, n1, s) ||
            !ensure(c, c->ctr, sizeof(DevCounters), s))
            return fail(c, MCL_ERR_OOM, "batch scratch allocation failed");
        CUDA_TRY(c, cudaMemcpyAsync(c->comp_off.p, comp_offsets, (size_t)(ncomp + 1) * 4,
                                    cudaMemcpyHostToDevice, s));
        CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(DevCounters), s));
        launch_comp_assign(view(A0), (const int32_t*)c->comp_off.p, ncomp,
                           (int32_t*)c->comp_of_col.p, (DevCounters*)c->ctr.p, s);
        if ((st = read_counters(c, s))) return st;
        if (c->hctr->err & ERR_ROW_RANGE)
            return fail(c, MCL_ERR_INVALID, "A0 is not block diagonal over comp_offsets");
        CUDA_TRY(c, cudaMemsetAsync(c->comp_active.p, 1, (size_t)ncomp, s));
    }
    std::vector<unsigned long long> hbits(batched ? ncomp : 0);
    std::vector<uint8_t> hact(batched ? ncomp : 0, 1);
    int nactive = batched ? ncomp : 1;
    mcl_csc cur = *A0;
    bool owned = false;
    int it = 0;
    double ch = 0.0;
    bool converged = false;
    const int saved_iter = c->iteration;
    c->prev_valid = 0;
    PruneParams gpp;
    c->run_exact = 0;
    int gsizing = c->sizing >= 0 ? c->sizing : (prm->use_estimator ? 2 : 0);
    // Estimator fallback: an iteration whose learned estimates fall short on
    // more than 1/20 of the expanded columns (each miss splits windows and
    // redoes their products) hands the rest of the run to the exact sizing.
    auto learned_missed = [&](int64_t misses) -> bool {
        if (gsizing != 2 || c->run_exact) return false;
        int64_t cols = cur.n;
        if (batched) {
            cols = 0;
            for (int q = 0; q < ncomp; ++q)
                if (hact[q]) cols += comp_offsets[q + 1] - comp_offsets[q];
        }
        return misses * 20 > cols;
    };
    bool graph_ok = batched && c->graph_mode && gsizing >= 0 && gsizing <= 3 &&
                    check_params(c, prm, &gpp, true) == MCL_OK;
    GraphRun G;
    int graph_at = -1;  // replay buffer holding cur
    c->stats.graph_replays = 0;
    c->stats.exact_from = 0;
    while (it < prm->max_iters) {
        if (graph_ok && it >= 1) {
            if (graph_at < 0) {
                st = graph_prepare(c, prm, gpp, comp_offsets, ncomp, &cur, gsizing, G, s);
                if (st) {
                    graph_release(c, G, s, -1);
                    if (owned) free_csc(c, &cur, s);  // no-op if graph_prepare took it over
                    c->iteration = saved_iter;
                    c->run_exact = 0;
                    return st;
                }
                graph_at = 0;
                cur = G.buf[0];
                cudaEvent_t e;
                cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
                cudaEventRecord(e, s);
                cudaStreamWaitEvent(G.gs, e, 0);
                cudaEventDestroy(e);
            }
            const int64_t in_nnz = cur.nnz;
            CUDA_TRY(c, cudaGraphLaunch(G.x[graph_at], G.gs));
            count_launches((int)G.kernels);
            CUDA_TRY(c, cudaStreamSynchronize(G.gs));
            ++c->stats.graph_replays;
            const unsigned ef = c->hctr->err;
            const bool refit = !ef && learned_missed((int64_t)c->hctr->misses);
            if (ef & ERR_STAGING) {
                // capacities beyond the replay buffers: this and later iterations run
                // without graphs, from the replay buffer that holds the input
                graph_ok = false;
                int64_t nz = 0;
                CUDA_TRY(c, cudaMemcpy(&nz, cur.colptr + cur.n, 8, cudaMemcpyDeviceToHost));
                cur.nnz = nz;
                CUDA_TRY(c, cudaMemcpy(hact.data(), c->comp_active.p, (size_t)ncomp,
                                       cudaMemcpyDeviceToHost));
                for (int q = 0; q < 2; ++q) {
                    if (G.x[q]) cudaGraphExecDestroy(G.x[q]);
                    if (G.g[q]) cudaGraphDestroy(G.g[q]);
                    G.x[q] = nullptr;
                    G.g[q] = nullptr;
                }
                free_csc(c, &G.buf[graph_at ^ 1], s);
                G.buf[graph_at] = mcl_csc{};
                cudaStreamDestroy(G.gs);
                G.gs = nullptr;
                graph_at = -1;
                owned = true;
                continue;
            }
            if (ef) {
                graph_release(c, G, s, -1);
                c->iteration = saved_iter;
                c->run_exact = 0;
                return err_flags(c, ef);
            }
            graph_at ^= 1;
            cur = G.buf[graph_at];
            cur.nnz = (int64_t)c->hctr->nnz_out;
            G.buf[graph_at].nnz = G.cap;
            ch = chaos_from_bits(c->hctr->chaos_bits);
            nactive = c->hctr->n_active;
            if (refit && nactive > 0) {
                // later replays size exactly: recapture from the buffer holding cur
                c->run_exact = 1;
                c->stats.exact_from = it + 2;
                gsizing = 0;
                CUDA_TRY(c, cudaMemcpy(hact.data(), c->comp_active.p, (size_t)ncomp,
                                       cudaMemcpyDeviceToHost));
                for (int q = 0; q < 2; ++q) {
                    if (G.x[q]) cudaGraphExecDestroy(G.x[q]);
                    if (G.g[q]) cudaGraphDestroy(G.g[q]);
                    G.x[q] = nullptr;
                    G.g[q] = nullptr;
                }
                CUDA_TRY(c, cudaStreamSynchronize(G.gs));
                cudaStreamDestroy(G.gs);
                G.gs = nullptr;
                free_csc(c, &G.buf[graph_at ^ 1], s);
                G.buf[graph_at] = mcl_csc{};
                graph_at = -1;
                owned = true;
            }
            mcl_stats& S = c->stats;
            S.flops = (int64_t)c->hctr->flops;
            S.flops_run += S.flops;
            S.alg_bytes_run += 8 * (in_nnz + S.flops + cur.nnz) + 16 * (int64_t)cur.n;
            S.nnz_in = G.cap;
            S.nnz_b = (int64_t)c->hctr->nnz_b;
            S.nnz_out = cur.nnz;
            S.estimator_misses = (int64_t)c->hctr->misses;
            S.range_splits = (int64_t)c->hctr->splits;
            S.chaos = ch;
            if (chaos_hist) chaos_hist[it] = ch;
            ++it;
            if (nactive == 0) {
                converged = true;
                break;
            }
            continue;
        }
        mcl_csc nxt{};
        c->iteration = it + 1;
        const uint8_t* act = nullptr;
        if (batched) {
            launch_active_from_comp(cur.n, (const int32_t*)c->comp_of_col.p,
                                    (const uint8_t*)c->comp_active.p, (uint8_t*)c->active.p, s);
            act = (const uint8_t*)c->active.p;
        }
        st = expand_impl(c, &cur, prm, &nxt, &ch, s, act);
        const int64_t it_misses = st ? 0 : c->stats.estimator_misses;
        if (!st) {
            mcl_stats& S = c->stats;
            S.flops_run += S.flops;
            S.alg_bytes_run += 8 * (S.nnz_in + S.flops + S.nnz_out) + 16 * (int64_t)cur.n;
        }
        if (!st && batched) {
            // per-component chaos of this iteration; converged components retire
            cudaMemsetAsync(c->comp_bits.p, 0, (size_t)ncomp * 8, s);
            launch_comp_chaos(cur.n, (const int32_t*)c->comp_of_col.p, act,
                              (const double*)c->chaos.p, (unsigned long long*)c->comp_bits.p, s);
            cudaMemcpyAsync(hbits.data(), c->comp_bits.p, (size_t)ncomp * 8, cudaMemcpyDeviceToHost,
                            s);
            if (cudaStreamSynchronize(s) != cudaSuccess)
                st = fail(c, MCL_ERR_CUDA, "component chaos readback failed");
            nactive = 0;
            for (int q = 0; q < ncomp && !st; ++q) {
                if (!hact[q]) continue;
                if (chaos_from_bits(hbits[q]) < prm->chaos_eps)
                    hact[q] = 0;
                else
                    ++nactive;
            }
            if (!st)
                cudaMemcpyAsync(c->comp_active.p, hact.data(), (size_t)ncomp, cudaMemcpyHostToDevice, s);
        }
        if (!st && learned_missed(it_misses)) {
            c->run_exact = 1;
            c->stats.exact_from = it + 2;
            gsizing = 0;
        }
        if (!st && prm->use_estimator) {
            // the compression factor of this iteration feeds the next one's features
            if (ensure(c, c->prev_logcf, ((size_t)cur.n + 1) * 4, s)) {
                launch_logcf(cur.n, (const int64_t*)c->flops.p, (const int64_t*)c->bnnz.p,
                             (float*)c->prev_logcf.p, s);
                c->prev_valid = 1;
            }
        }
        if (st) {
            if (owned) free_csc(c, &cur, s);
            c->iteration = saved_iter;
            c->run_exact = 0;
            c->prev_valid = 0;
            return st;
        }
        if (owned) free_csc(c, &cur, s);
        cur = nxt;
        owned = true;
        if (chaos_hist) chaos_hist[it] = ch;
        ++it;
        if (batched ? nactive == 0 : ch < prm->chaos_eps) {
            converged = true;
            break;
        }
    }
    c->iteration = saved_iter;
    c->run_exact = 0;
    c->prev_valid = 0;
    if (graph_at >= 0) {
        // cur is replay buffer graph_at: keep it (owned, freed below or handed out)
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        cudaEventRecord(e, G.gs);
        cudaStreamWaitEvent(s, e, 0);
        cudaEventDestroy(e);
        graph_release(c, G, s, graph_at);
        owned = true;
    }
    c->stats.iterations = it;
    if (iters) *iters = it;
    st = mcl_components(c, &cur, labels, stream);
    if (st) {
        if (owned) free_csc(c, &cur, s);
        return st;
    }
    if (final_out)
        *final_out = cur;
    else if (owned)
        free_csc(c, &cur, s);
    if (!converged)
        return fail(c, MCL_ERR_NOT_CONVERGED, "max_iters reached with chaos %.3e", ch);
    return MCL_OK;
}

}  // extern "C"
