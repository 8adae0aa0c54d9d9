// Allocation-free variant of the exact symbolic pass.
//
// Some callers cannot allocate device memory at the point where they need
// output sizes: services that reserve the whole GPU memory in a pool at
// start-up and forbid allocation afterwards (cudaMalloc may implicitly
// synchronise the device and can fail under fragmentation), or hosts whose
// memory management owns every device allocation.  For them,
// mcl_symbolic_noalloc computes flops_j and nnz((AA)_*j) with no context
// and no allocation: its scratch is one file-scope device array of
// MCL_NOALLOC_SCRATCH_BYTES, which every GPU that loads this library holds
// until the process exits.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "mcl.h"
#include "mcl_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MCL_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

void put_error(char* buf, size_t len, const char* fmt, ...) {
    if (!buf || len == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, len, fmt, ap);
    va_end(ap);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" mcl_status mcl_symbolic_noalloc(const mcl_csc* A, int64_t* flops, int64_t* nnz_out,
                                           char* errbuf, size_t errlen, void* stream) {
    using namespace mcl;
    if (!A || A->n < 0 || A->nnz < 0 || !A->colptr || (A->nnz > 0 && (!A->rowidx || !A->val))) {
        put_error(errbuf, errlen, "invalid CSC argument");
        return MCL_ERR_INVALID;
    }
    if (A->n > 0 && !flops && !nnz_out) {
        put_error(errbuf, errlen, "flops and nnz_out are both NULL");
        return MCL_ERR_INVALID;
    }
    const size_t n = (size_t)A->n;
    // layout: counters | flops (if not given) | row span lo | hi | capacity | cursors
    const size_t off_flops = align256(sizeof(DevCounters));
    const size_t off_rlo = off_flops + align256(n * 8);
    const size_t off_rhi = off_rlo + align256(n * 4);
    const size_t off_cap = off_rhi + align256(n * 4);
    const size_t off_cur = off_cap + align256(n * 8);
    if (off_cur > (size_t)MCL_NOALLOC_SCRATCH_BYTES) {
        put_error(errbuf, errlen,
                  "n = %lld needs %zu bytes of per-column scratch, above the %d-byte maximum "
                  "(at most about %lld columns)",
                  (long long)A->n, off_cur, MCL_NOALLOC_SCRATCH_BYTES,
                  (long long)((MCL_NOALLOC_SCRATCH_BYTES - 4096) / 24));
        return MCL_ERR_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        put_error(errbuf, errlen, "no usable current CUDA device");
        return MCL_ERR_CUDA;
    }
    // once per device, with that device current: the array's device address
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                put_error(errbuf, errlen, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return MCL_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* sb = static_cast<unsigned char*>(base);
    ExpandBuffers b{};
    b.ctr = reinterpret_cast<DevCounters*>(sb);
    b.flops = flops ? flops : reinterpret_cast<int64_t*>(sb + off_flops);
    b.rlo = reinterpret_cast<int32_t*>(sb + off_rlo);
    b.rhi = reinterpret_cast<int32_t*>(sb + off_rhi);
    b.cap = reinterpret_cast<int64_t*>(sb + off_cap);
    b.active = nullptr;
    int num_sms = 0;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    // the array keeps the previous call's contents: clear the counters
    if (cudaMemsetAsync(b.ctr, 0, sizeof(DevCounters), s) != cudaSuccess) {
        cudaGetLastError();
        put_error(errbuf, errlen, "cudaMemsetAsync failed");
        return MCL_ERR_CUDA;
    }
    const CscView Av{A->n, A->nnz, A->colptr, A->rowidx, A->val};
    PruneParams pp{};
    pp.Krec = 1;
    launch_colstats(Av, pp, b, num_sms > 0 ? num_sms : 1, s);
    unsigned err = 0;
    int max_deg = 0;
    if (cudaMemcpyAsync(&err, &b.ctr->err, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&max_deg, &b.ctr->max_deg, sizeof(max_deg), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        put_error(errbuf, errlen, "column statistics failed: %s", cudaGetErrorString(e));
        return MCL_ERR_CUDA;
    }
    if (err) {
        put_error(errbuf, errlen, "malformed CSC input (flags 0x%x)", err);
        return MCL_ERR_INVALID;
    }
    if (nnz_out && A->n > 0) {
        b.cur_stride = ((max_deg + 31) & ~31) + 32;
        const size_t per_cta = (size_t)b.cur_stride * 2 * 4;
        const size_t room = (size_t)MCL_NOALLOC_SCRATCH_BYTES - off_cur;
        int grid = (int)(room / per_cta);
        if (grid < 1) {
            put_error(errbuf, errlen,
                      "a column with %d entries needs %zu bytes of cursor scratch; %zu remain of "
                      "the %d-byte maximum",
                      max_deg, per_cta, room, MCL_NOALLOC_SCRATCH_BYTES);
            return MCL_ERR_INVALID;
        }
        const int gmax = symbolic_grid(num_sms > 0 ? num_sms : 1);
        if (grid > gmax) grid = gmax;
        b.cursors = reinterpret_cast<int32_t*>(sb + off_cur);
        launch_symbolic(Av, b, nnz_out, num_sms > 0 ? num_sms : 1, grid, s);
        // the pass flags a column longer than its cursor space (not expected:
        // the stride exceeds the longest column) instead of writing its count
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            put_error(errbuf, errlen, "launch failed: %s", cudaGetErrorString(le));
            return MCL_ERR_CUDA;
        }
        err = 0;
        if (cudaMemcpyAsync(&err, &b.ctr->err, sizeof(err), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            const cudaError_t e2 = cudaGetLastError();
            put_error(errbuf, errlen, "symbolic pass failed: %s", cudaGetErrorString(e2));
            return MCL_ERR_CUDA;
        }
        if (err) {
            put_error(errbuf, errlen, "symbolic pass raised flags 0x%x", err);
            return MCL_ERR_INTERNAL;
        }
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        put_error(errbuf, errlen, "launch failed: %s", cudaGetErrorString(e));
        return MCL_ERR_CUDA;
    }
    return MCL_OK;
}
