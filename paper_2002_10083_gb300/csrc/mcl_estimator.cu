// Learned output-size estimator: per-column features, a 16 -> 64 -> 64 -> 2
// MLP (BF16 weights, FP32 accumulation) predicting y0 = log(1 + nnz_j) and
// y1 = log cf_j for every column of A*A, and its training kernels
// (backward pass, Adam).  The prediction replaces the exact symbolic
// SpGEMM (Sections II and V: memory estimation before every iteration)
// for sizing the accumulators; the numeric pass stays exact whatever the
// estimate (an under-estimate only narrows row ranges).
//
// Parameter layout (5378 values): W1 [64 x 16] (row = output unit), b1 [64],
// W2 [64 x 64], b2 [64], W3 [2 x 64], b3 [2].  Inputs are standardised with
// (x - mu) / sigma (norm = mu[16] then sigma[16]).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mcl.h"
#include "mcl_device.cuh"
#include "mcl_internal.h"

namespace mcl {

constexpr int NIN = 16, NH = 64, NOUT = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUT * NH,
              NPARAM = OFF_B3 + NOUT;
static_assert(NPARAM == MCL_MLP_NPARAM, "parameter count");
constexpr int HUGE_DEG = 1024;

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
    return __uint_as_float(((uint32_t)b) << 16);
}

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------

__global__ void k_colmax(CscView A, float* colmax) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < A.n; j += nw) {
        float m = 0.0f;
        for (int64_t p = A.colptr[j] + lane; p < A.colptr[j + 1]; p += 32) m = fmaxf(m, A.val[p]);
        m = warp_max(m);
        if (lane == 0) colmax[j] = m;
    }
}

// Warp per column: the 16 features (see oracle/mlp.py FEATURES for the list).
__global__ void k_features(CscView A, int32_t iteration, const int32_t* iter_dev,
                           const float* prev_logcf, const float* colmax, float* feats) {
    if (iter_dev) iteration = *iter_dev;  // graph replays keep the index on the device
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float logn = logf((float)(A.n > 0 ? A.n : 1));
    const float logit = log1pf((float)iteration);
    for (int64_t j = gw; j < A.n; j += nw) {
        const int64_t cb = A.colptr[j], ce = A.colptr[j + 1];
        const int d = (int)(ce - cb);
        long long sd = 0, sd2 = 0;
        int md = 0, huge = 0, fmin = INT_MAX, lmax = -1;
        double sa = 0.0, sa2 = 0.0, scm = 0.0;
        float ma = 0.0f;
        for (int64_t p = cb + lane; p < ce; p += 32) {
            const int k = A.rowidx[p];
            const float a = A.val[p];
            const int64_t ks = A.colptr[k], ke = A.colptr[k + 1];
            const int dk = (int)(ke - ks);
            sd += dk;
            sd2 += (long long)dk * dk;
            md = max(md, dk);
            huge += dk > HUGE_DEG;
            sa += a;
            sa2 += (double)a * a;
            ma = fmaxf(ma, a);
            scm += colmax[k];
            if (dk > 0) {
                fmin = min(fmin, A.rowidx[ks]);
                lmax = max(lmax, A.rowidx[ke - 1]);
            }
        }
        sd = warp_sum(sd);
        sd2 = warp_sum(sd2);
        md = warp_max(md);
        huge = warp_sum(huge);
        sa = warp_sum(sa);
        sa2 = warp_sum(sa2);
        ma = warp_max(ma);
        scm = warp_sum(scm);
        fmin = warp_min(fmin);
        lmax = warp_max(lmax);
        if (lane < NIN) {
            float f = 0.0f;
            const double dd = (double)d;
            switch (lane) {
                case 0: f = log1pf((float)d); break;
                case 1: f = (float)log1p((double)sd); break;
                case 2: f = d ? log1pf((float)md) : 0.0f; break;
                case 3: f = d ? (float)log1p((double)sd / dd) : 0.0f; break;
                case 4: {
                    if (d) {
                        const double mean = (double)sd / dd;
                        double var = (double)sd2 / dd - mean * mean;
                        f = (float)log1p(var > 0.0 ? var : 0.0);
                    }
                    break;
                }
                case 5: f = ma; break;
                case 6: f = (float)sa; break;
                case 7: f = (float)sa2; break;
                case 8:
                    f = d ? log1pf((float)(A.rowidx[ce - 1] - A.rowidx[cb] + 1)) : 0.0f;
                    break;
                case 9: f = d ? (float)((double)huge / dd) : 0.0f; break;
                case 10: f = logn; break;
                case 11: f = logit; break;
                case 12: f = prev_logcf ? prev_logcf[j] : 0.0f; break;
                case 13: f = d ? (float)(scm / dd) : 0.0f; break;
                case 14: f = (lmax >= 0) ? (float)log1p((double)(lmax - fmin) + 1.0) : 0.0f; break;
                default: f = 1.0f; break;
            }
            feats[j * NIN + lane] = f;
        }
    }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

constexpr int FWD_T = 128;

__device__ __forceinline__ void load_weights(float* W, const uint16_t* wbits) {
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) W[i] = bf16_bits_to_float(wbits[i]);
}

// One sample per thread.  Writes y (out, n x 2) and/or, when est != NULL,
// the size estimate est_j = clamp(ceil(expm1(y0) * safety), 1, min(flops, span)).
__global__ void __launch_bounds__(FWD_T) k_mlp_forward(const float* feats, int64_t n,
                                                       const uint16_t* wbits, const float* norm,
                                                       float* out, int64_t* est, float safety,
                                                       const int64_t* flops, const int32_t* rlo,
                                                       const int32_t* rhi) {
    __shared__ float W[NPARAM];
    __shared__ float mu[NIN], isg[NIN];
    load_weights(W, wbits);
    if (threadIdx.x < NIN) {
        mu[threadIdx.x] = norm[threadIdx.x];
        isg[threadIdx.x] = 1.0f / norm[NIN + threadIdx.x];
    }
    __syncthreads();
    for (int64_t s = (int64_t)blockIdx.x * FWD_T + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * FWD_T) {
        float z[NIN];
#pragma unroll
        for (int i = 0; i < NIN; ++i) z[i] = (feats[s * NIN + i] - mu[i]) * isg[i];
        float h1[NH];
#pragma unroll
        for (int o = 0; o < NH; ++o) {
            float acc = W[OFF_B1 + o];
#pragma unroll
            for (int i = 0; i < NIN; ++i) acc = fmaf(W[OFF_W1 + o * NIN + i], z[i], acc);
            h1[o] = fmaxf(acc, 0.0f);
        }
        float y0 = W[OFF_B3], y1 = W[OFF_B3 + 1];
        for (int o = 0; o < NH; ++o) {
            float acc = W[OFF_B2 + o];
#pragma unroll
            for (int i = 0; i < NH; ++i) acc = fmaf(W[OFF_W2 + o * NH + i], h1[i], acc);
            const float h2 = fmaxf(acc, 0.0f);
            y0 = fmaf(W[OFF_W3 + o], h2, y0);
            y1 = fmaf(W[OFF_W3 + NH + o], h2, y1);
        }
        if (out) {
            out[s * 2] = y0;
            out[s * 2 + 1] = y1;
        }
        if (est) {
            int64_t hi = flops[s];
            const int64_t span = (int64_t)rhi[s] - rlo[s] + 1;
            if (span < hi) hi = span;
            if (hi < 1) hi = 1;
            const double e = ceil(expm1((double)fminf(y0, 40.0f)) * (double)safety);
            int64_t v = e < 1.0 ? 1 : (e > (double)hi ? hi : (int64_t)e);
            est[s] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// backward (training)
// ---------------------------------------------------------------------------

constexpr int BWD_B = 64;     // samples (= threads) per CTA
constexpr int HP = NH + 1;    // padded row stride

struct BwdShared {
    float W[NPARAM];
    float mu[NIN], isg[NIN];
    float Z[BWD_B][NIN + 1];
    float H1[BWD_B][HP];
    float A2[BWD_B][HP];
    float D2[BWD_B][HP];
    float D1[BWD_B][HP];
    float DY[BWD_B][NOUT];
    double red[BWD_B / 32];
};

// Gradient of (scale * sum over samples and outputs of (y - t)^2) with
// respect to the (BF16-valued) weights, added into grad; the loss sum
// (unscaled) is added into *loss.
__global__ void __launch_bounds__(BWD_B) k_mlp_backward(const float* feats, const float* targets,
                                                        int64_t n, const uint16_t* wbits,
                                                        const float* norm, float scale,
                                                        float* grad, double* loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdShared& S = *reinterpret_cast<BwdShared*>(smem_raw);
    const int b = threadIdx.x;
    load_weights(S.W, wbits);
    if (b < NIN) {
        S.mu[b] = norm[b];
        S.isg[b] = 1.0f / norm[NIN + b];
    }
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * BWD_B + b;
    double lsum = 0.0;
    if (s < n) {
        for (int i = 0; i < NIN; ++i) S.Z[b][i] = (feats[s * NIN + i] - S.mu[i]) * S.isg[i];
        for (int o = 0; o < NH; ++o) {
            float acc = S.W[OFF_B1 + o];
            for (int i = 0; i < NIN; ++i) acc = fmaf(S.W[OFF_W1 + o * NIN + i], S.Z[b][i], acc);
            S.H1[b][o] = fmaxf(acc, 0.0f);
        }
        float y0 = S.W[OFF_B3], y1 = S.W[OFF_B3 + 1];
        for (int o = 0; o < NH; ++o) {
            float acc = S.W[OFF_B2 + o];
            for (int i = 0; i < NH; ++i) acc = fmaf(S.W[OFF_W2 + o * NH + i], S.H1[b][i], acc);
            S.A2[b][o] = acc;
            const float h2 = fmaxf(acc, 0.0f);
            y0 = fmaf(S.W[OFF_W3 + o], h2, y0);
            y1 = fmaf(S.W[OFF_W3 + NH + o], h2, y1);
        }
        const float e0 = y0 - targets[s * 2], e1 = y1 - targets[s * 2 + 1];
        lsum = (double)e0 * e0 + (double)e1 * e1;
        const float d0 = 2.0f * e0 * scale, d1 = 2.0f * e1 * scale;
        S.DY[b][0] = d0;
        S.DY[b][1] = d1;
        for (int i = 0; i < NH; ++i) {
            const float g = d0 * S.W[OFF_W3 + i] + d1 * S.W[OFF_W3 + NH + i];
            S.D2[b][i] = S.A2[b][i] > 0.0f ? g : 0.0f;
        }
        for (int i = 0; i < NH; ++i) {
            float g = 0.0f;
            for (int o = 0; o < NH; ++o) g = fmaf(S.D2[b][o], S.W[OFF_W2 + o * NH + i], g);
            S.D1[b][i] = S.H1[b][i] > 0.0f ? g : 0.0f;
        }
    } else {
        for (int i = 0; i < NIN; ++i) S.Z[b][i] = 0.0f;
        for (int i = 0; i < NH; ++i) {
            S.H1[b][i] = 0.0f;
            S.A2[b][i] = 0.0f;
            S.D2[b][i] = 0.0f;
            S.D1[b][i] = 0.0f;
        }
        S.DY[b][0] = 0.0f;
        S.DY[b][1] = 0.0f;
    }
    lsum = warp_sum(lsum);
    if ((b & 31) == 0) S.red[b >> 5] = lsum;
    __syncthreads();
    if (b == 0) {
        double t = 0.0;
        for (int w = 0; w < BWD_B / 32; ++w) t += S.red[w];
        atomicAdd(loss, t);
    }
    // weight gradients: sums over the CTA's samples
    for (int p = b; p < NPARAM; p += BWD_B) {
        float acc = 0.0f;
        if (p < OFF_B1) {
            const int o = p / NIN, i = p % NIN;
            for (int q = 0; q < BWD_B; ++q) acc = fmaf(S.D1[q][o], S.Z[q][i], acc);
        } else if (p < OFF_W2) {
            const int o = p - OFF_B1;
            for (int q = 0; q < BWD_B; ++q) acc += S.D1[q][o];
        } else if (p < OFF_B2) {
            const int o = (p - OFF_W2) / NH, i = (p - OFF_W2) % NH;
            for (int q = 0; q < BWD_B; ++q) acc = fmaf(S.D2[q][o], S.H1[q][i], acc);
        } else if (p < OFF_W3) {
            const int o = p - OFF_B2;
            for (int q = 0; q < BWD_B; ++q) acc += S.D2[q][o];
        } else if (p < OFF_B3) {
            const int o = (p - OFF_W3) / NH, i = (p - OFF_W3) % NH;
            for (int q = 0; q < BWD_B; ++q) acc = fmaf(S.DY[q][o], fmaxf(S.A2[q][i], 0.0f), acc);
        } else {
            const int o = p - OFF_B3;
            for (int q = 0; q < BWD_B; ++q) acc += S.DY[q][o];
        }
        atomicAdd(grad + p, acc);
    }
}

// Adam step on the FP32 master weights; writes their BF16 rounding.
__global__ void k_adam(float* master, float* m, float* v, const float* grad, int64_t step, float lr,
                       float b1, float b2, float eps, uint16_t* wbits) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.0f - b1) * g;
    const float vv = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    const float w = master[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    master[p] = w;
    wbits[p] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

// log cf_j = log(flops_j / max(nnz_j, 1)) from the last numeric pass (input
// to the next iteration's features).
__global__ void k_logcf(int32_t n, const int64_t* flops, const int64_t* bnnz, float* logcf) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t z = bnnz[j] > 0 ? bnnz[j] : 1;
    logcf[j] = flops[j] > 0 ? logf((float)((double)flops[j] / (double)z)) : 0.0f;
}

void launch_colmax_features(const CscView& A, int32_t iteration, const float* prev_logcf,
                            float* colmax, float* feats, cudaStream_t s, const int32_t* iter_dev) {
    if (A.n == 0) return;
    int64_t blocks = ((int64_t)A.n * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_colmax<<<(unsigned)blocks, 256, 0, s>>>(A, colmax);
    count_launches(1);
    k_features<<<(unsigned)blocks, 256, 0, s>>>(A, iteration, iter_dev, prev_logcf, colmax, feats);
    count_launches(1);
}

void launch_mlp_forward(const float* feats, int64_t n, const uint16_t* wbits, const float* norm,
                        float* out, int64_t* est, float safety, const int64_t* flops,
                        const int32_t* rlo, const int32_t* rhi, cudaStream_t s) {
    if (n == 0) return;
    int64_t blocks = (n + FWD_T - 1) / FWD_T;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_mlp_forward<<<(unsigned)blocks, FWD_T, 0, s>>>(feats, n, wbits, norm, out, est, safety,
                                                      flops, rlo, rhi);
    count_launches(1);
}

void launch_mlp_backward(const float* feats, const float* targets, int64_t n,
                         const uint16_t* wbits, const float* norm, float scale, float* grad,
                         double* loss, cudaStream_t s) {
    if (n == 0) return;
    const size_t smem = sizeof(BwdShared);
    cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t blocks = (n + BWD_B - 1) / BWD_B;
    k_mlp_backward<<<(unsigned)blocks, BWD_B, smem, s>>>(feats, targets, n, wbits, norm, scale,
                                                          grad, loss);
    count_launches(1);
}

void launch_adam(float* master, float* m, float* v, const float* grad, int64_t step, float lr,
                 float b1, float b2, float eps, uint16_t* wbits, cudaStream_t s) {
    k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(master, m, v, grad, step, lr, b1, b2, eps, wbits);
    count_launches(1);
}

__global__ void k_iter_bump(int32_t* it) {
    if (threadIdx.x == 0) ++*it;
}

void launch_iter_bump(int32_t* it, cudaStream_t s) {
    k_iter_bump<<<1, 32, 0, s>>>(it);
    count_launches(1);
}

void launch_logcf(int32_t n, const int64_t* flops, const int64_t* bnnz, float* logcf,
                  cudaStream_t s) {
    if (n == 0) return;
    k_logcf<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, flops, bnnz, logcf);
    count_launches(1);
}

}  // namespace mcl
