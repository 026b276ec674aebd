// Learned output sizing: a small MLP that predicts, per output row, the
// fraction r_i = nnz(C_i) / ub_i of its intermediate products that land on
// distinct columns (the paper sizes nothing by learning: this serves the
// numeric phase's capacity choice, with exact fallback on overflow).
//
// Features f_i = log1p(nnz(A_i), ub_i, max_k nnz(B_k), mean_k nnz(B_k)).
// Network 4 -> 64 -> 64 -> 1, ReLU, r = sigmoid(z).  BF16 weights and
// activations (features, h1, h2 rounded to BF16), FP32 accumulation.
// Loss per row: pinball (quantile tau) on log r:  u = log(target) - log r,
// L = tau u (u > 0, under-prediction) else (tau - 1) u.
//
// Parameters (kParams floats): W1[64][4] b1[64] W2[64][64] b2[64] W3[64] b3.
// Training: forward with activations kept, per-row backward, parameter
// gradients as reductions over the batch, Adam on FP32 master weights.
#include <cuda_bf16.h>

#include "../../include/spgemm.h"
#include "plan.h"
#include "rowwork.cuh"

namespace spg {

constexpr int kIn = 4, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH,
              kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH,
              kParams = kOffB3 + 1;
static_assert(kParams == SPGEMM_MLP_PARAMS, "parameter layout of the C ABI");

SPG_DEV float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---- features -----------------------------------------------------------------

// f = log1p(nnz(A_i), ub_i, max nnz(B_k), mean nnz(B_k)), one 16-byte store per
// row.  Pass 1: 32 consecutive rows per warp, long rows to a list; pass 2: a
// warp per listed row.
SPG_DEV void store_features(float* feat, int64_t* ub_out, int64_t g, int64_t na, int64_t s,
                            int64_t mx) {
    const float4 f = make_float4(log1pf((float)na), log1pf((float)s), log1pf((float)mx),
                                 log1pf(na > 0 ? (float)s / (float)na : 0.f));
    reinterpret_cast<float4*>(feat)[g] = f;
    if (ub_out) ub_out[g] = s;
}

__global__ void k_row_features(const Prob* __restrict__ probs, int nprob, int64_t R,
                               float* __restrict__ feat, int64_t* __restrict__ ub_out,
                               int32_t* long_rows, Counters* ctr) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id()) * 32; g0 < R;
         g0 += nw * 32) {
        const int64_t g = g0 + lane;
        bool is_long = false;
        if (g < R) {
            const RowRange rr = row_range(probs, nprob, g);
            const int64_t na = rr.a1 - rr.a0;
            if (na > kRowShort) {
                is_long = true;
            } else {
                int64_t s, mx;
                lane_row_counts(probs[rr.pi], rr.a0, na, s, mx);
                store_features(feat, ub_out, g, na, s, mx);
            }
        }
        append_rows(is_long, g, long_rows, ctr);
    }
}

__global__ void k_row_features_long(const Prob* __restrict__ probs, int nprob,
                                    float* __restrict__ feat, int64_t* __restrict__ ub_out,
                                    const int32_t* __restrict__ long_rows, const Counters* ctr) {
    const int n = ctr->claim[kClLongRows];
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + warp_id(); r < n; r += nw) {
        const int64_t g = long_rows[r];
        const RowRange rr = row_range(probs, nprob, g);
        int64_t s, mx;
        warp_row_long(probs[rr.pi], rr.a0, rr.a1, s, mx);
        if (lane_id() == 0) store_features(feat, ub_out, g, rr.a1 - rr.a0, s, mx);
    }
}

// ---- forward (inference) ----------------------------------------------------------

// one thread per row; parameters (BF16) staged in shared memory as float.
// With ub != null, rows with ub <= min_ub are skipped (z left unwritten).
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ feat, int64_t R,
                                                     const __nv_bfloat16* __restrict__ params,
                                                     float* __restrict__ z_out,
                                                     const int64_t* __restrict__ ub,
                                                     int64_t min_ub) {
    __shared__ float w[kParams];
    for (int t = threadIdx.x; t < kParams; t += blockDim.x) w[t] = __bfloat162float(params[t]);
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (ub && ub[r] <= min_ub) continue;
        float f[kIn];
#pragma unroll
        for (int m = 0; m < kIn; ++m) f[m] = bf(feat[r * 4 + m]);
        float h1[kH];
#pragma unroll
        for (int k = 0; k < kH; ++k) {
            float a = w[kOffB1 + k];
#pragma unroll
            for (int m = 0; m < kIn; ++m) a = fmaf(w[kOffW1 + k * kIn + m], f[m], a);
            h1[k] = bf(fmaxf(a, 0.f));
        }
        float z = w[kOffB3];
        for (int j = 0; j < kH; ++j) {
            float a = w[kOffB2 + j];
#pragma unroll
            for (int k = 0; k < kH; ++k) a = fmaf(w[kOffW2 + j * kH + k], h1[k], a);
            z = fmaf(w[kOffW3 + j], bf(fmaxf(a, 0.f)), z);
        }
        z_out[r] = z;
    }
}

// ---- training -----------------------------------------------------------------------

// forward with activations kept (H1 post-ReLU BF16-rounded, H2 pre-activation),
// and dz = dL/dz of the pinball loss; loss summed into *loss
__global__ void __launch_bounds__(128) k_mlp_train_fwd(const float* __restrict__ feat,
                                                       const float* __restrict__ logt, int64_t B,
                                                       float tau,
                                                       const __nv_bfloat16* __restrict__ params,
                                                       float* __restrict__ H1, float* __restrict__ H2,
                                                       float* __restrict__ dz, float* loss) {
    __shared__ float w[kParams];
    for (int t = threadIdx.x; t < kParams; t += blockDim.x) w[t] = __bfloat162float(params[t]);
    __syncthreads();
    float lsum = 0.f;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < B;
         r += (int64_t)gridDim.x * blockDim.x) {
        float f[kIn];
#pragma unroll
        for (int m = 0; m < kIn; ++m) f[m] = bf(feat[r * 4 + m]);
        float h1[kH];
#pragma unroll
        for (int k = 0; k < kH; ++k) {
            float a = w[kOffB1 + k];
#pragma unroll
            for (int m = 0; m < kIn; ++m) a = fmaf(w[kOffW1 + k * kIn + m], f[m], a);
            h1[k] = bf(fmaxf(a, 0.f));
            H1[r * kH + k] = h1[k];
        }
        float z = w[kOffB3];
        for (int j = 0; j < kH; ++j) {
            float a = w[kOffB2 + j];
#pragma unroll
            for (int k = 0; k < kH; ++k) a = fmaf(w[kOffW2 + j * kH + k], h1[k], a);
            H2[r * kH + j] = a;
            z = fmaf(w[kOffW3 + j], bf(fmaxf(a, 0.f)), z);
        }
        // log r = log sigmoid(z) = -softplus(-z)
        const float logr = -(fmaxf(-z, 0.f) + log1pf(expf(-fabsf(z))));
        const float u = logt[r] - logr;
        const float dLdu = u > 0.f ? tau : tau - 1.f;
        lsum += u > 0.f ? tau * u : (tau - 1.f) * u;
        const float sig = 1.f / (1.f + expf(-z));
        dz[r] = -dLdu * (1.f - sig) / (float)B;   // mean over the batch
    }
    lsum = warp_sum(lsum);
    if (lane_id() == 0) atomicAdd(loss, lsum / (float)B);
}

// per row: dH2[j] = W3[j] [H2 > 0] dz,  dH1[k] = (sum_j W2[j][k] dH2[j]) [H1 > 0]
__global__ void __launch_bounds__(128) k_mlp_train_bwd(const float* __restrict__ H1,
                                                       const float* __restrict__ H2,
                                                       const float* __restrict__ dz, int64_t B,
                                                       const __nv_bfloat16* __restrict__ params,
                                                       float* __restrict__ dH1,
                                                       float* __restrict__ dH2) {
    __shared__ float w[kParams];
    for (int t = threadIdx.x; t < kParams; t += blockDim.x) w[t] = __bfloat162float(params[t]);
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < B;
         r += (int64_t)gridDim.x * blockDim.x) {
        const float d = dz[r];
        float g2[kH];
#pragma unroll
        for (int j = 0; j < kH; ++j) {
            g2[j] = H2[r * kH + j] > 0.f ? w[kOffW3 + j] * d : 0.f;
            dH2[r * kH + j] = g2[j];
        }
        for (int k = 0; k < kH; ++k) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < kH; ++j) a = fmaf(w[kOffW2 + j * kH + k], g2[j], a);
            dH1[r * kH + k] = H1[r * kH + k] > 0.f ? a : 0.f;
        }
    }
}

// parameter gradients as reductions over the batch; one CTA per output group:
//   blocks [0, 64)   : W2 row j (64 threads = k) and b2[j] (thread 0)
//   blocks [64, 128) : W1 row k (4 threads) and b1[k]
//   block 128        : W3 (64 threads) and b3
__global__ void __launch_bounds__(64) k_mlp_train_wgrad(const float* __restrict__ feat,
                                                        const float* __restrict__ H1,
                                                        const float* __restrict__ H2,
                                                        const float* __restrict__ dz,
                                                        const float* __restrict__ dH1,
                                                        const float* __restrict__ dH2, int64_t B,
                                                        float* __restrict__ grad) {
    const int t = threadIdx.x;
    const int b = blockIdx.x;
    if (b < kH) {
        const int j = b;
        float gw = 0.f, gb = 0.f;
        for (int64_t r = 0; r < B; ++r) {
            const float g = dH2[r * kH + j];
            gw = fmaf(g, H1[r * kH + t], gw);
            gb += g;
        }
        grad[kOffW2 + j * kH + t] = gw;
        if (t == 0) grad[kOffB2 + j] = gb;
    } else if (b < 2 * kH) {
        const int k = b - kH;
        if (t < kIn) {
            float gw = 0.f;
            for (int64_t r = 0; r < B; ++r) gw = fmaf(dH1[r * kH + k], bf(feat[r * 4 + t]), gw);
            grad[kOffW1 + k * kIn + t] = gw;
        } else if (t == kIn) {
            float gb = 0.f;
            for (int64_t r = 0; r < B; ++r) gb += dH1[r * kH + k];
            grad[kOffB1 + k] = gb;
        }
    } else {
        float gw = 0.f, gb = 0.f;
        for (int64_t r = 0; r < B; ++r) {
            const float d = dz[r];
            gw = fmaf(d, bf(fmaxf(H2[r * kH + t], 0.f)), gw);
            gb += d;
        }
        grad[kOffW3 + t] = gw;
        if (t == 0) grad[kOffB3] = gb;
    }
}

// Adam on FP32 master weights, BF16 copy for the forward
__global__ void k_mlp_adam(float* __restrict__ master, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, __nv_bfloat16* __restrict__ params,
                           float lr, float b1, float b2, float eps, int step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)step));
    const float vh = vi / (1.f - powf(b2, (float)step));
    const float w = master[i] - lr * mh / (sqrtf(vh) + eps);
    master[i] = w;
    params[i] = __float2bfloat16_rn(w);
}

__global__ void k_mlp_to_bf16(const float* __restrict__ master, __nv_bfloat16* __restrict__ params) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kParams) params[i] = __float2bfloat16_rn(master[i]);
}

// ---- launchers ---------------------------------------------------------------------

int mlp_param_count() { return kParams; }

size_t mlp_train_ws_bytes(int64_t B) {
    // H1, H2, dH1, dH2 (B x 64 floats each), dz (B), grad (kParams)
    return sizeof(float) * ((size_t)B * kH * 4 + (size_t)B + kParams + 64);
}

cudaError_t launch_row_features(const Prob* probs, int nprob, int64_t R, float* feat,
                                int64_t* ub, int32_t* long_rows, Counters* ctr,
                                const DevInfo& dev, cudaStream_t st) {
    if (R <= 0) return cudaSuccess;
    int64_t blocks = (R + 255) / 256;    // 8 warps x 32 rows
    if (blocks > (int64_t)dev.sms * 16) blocks = (int64_t)dev.sms * 16;
    cudaError_t e = cudaMemsetAsync(&ctr->claim[kClLongRows], 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    k_row_features<<<(unsigned)blocks, 256, 0, st>>>(probs, nprob, R, feat, ub, long_rows, ctr);
    k_row_features_long<<<(unsigned)(dev.sms * 8), 256, 0, st>>>(probs, nprob, feat, ub,
                                                                  long_rows, ctr);
    count_launch(dev, 2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* feat, int64_t R, const void* params, float* z,
                               const int64_t* ub, int64_t min_ub, const DevInfo& dev,
                               cudaStream_t st) {
    if (R <= 0) return cudaSuccess;
    int64_t blocks = (R + 127) / 128;
    if (blocks > (int64_t)dev.sms * 8) blocks = (int64_t)dev.sms * 8;
    k_mlp_forward<<<(unsigned)blocks, 128, 0, st>>>(feat, R, (const __nv_bfloat16*)params, z,
                                                    ub, min_ub);
    count_launch(dev);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* feat, const float* logt, int64_t B, float tau,
                            const void* params, float* grad, float* loss, void* ws,
                            const DevInfo& dev, cudaStream_t st) {
    float* H1 = (float*)ws;
    float* H2 = H1 + (size_t)B * kH;
    float* dH1 = H2 + (size_t)B * kH;
    float* dH2 = dH1 + (size_t)B * kH;
    float* dz = dH2 + (size_t)B * kH;
    int64_t blocks = (B + 127) / 128;
    if (blocks > (int64_t)dev.sms * 8) blocks = (int64_t)dev.sms * 8;
    if (blocks < 1) blocks = 1;
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    k_mlp_train_fwd<<<(unsigned)blocks, 128, 0, st>>>(feat, logt, B, tau,
                                                      (const __nv_bfloat16*)params, H1, H2, dz, loss);
    k_mlp_train_bwd<<<(unsigned)blocks, 128, 0, st>>>(H1, H2, dz, B, (const __nv_bfloat16*)params,
                                                      dH1, dH2);
    k_mlp_train_wgrad<<<2 * kH + 1, 64, 0, st>>>(feat, H1, H2, dz, dH1, dH2, B, grad);
    count_launch(dev, 3);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* master, float* m, float* v, const float* grad, void* params,
                            float lr, int step, const DevInfo& dev, cudaStream_t st) {
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, st>>>(master, m, v, grad, (__nv_bfloat16*)params,
                                                       lr, 0.9f, 0.999f, 1e-8f, step);
    count_launch(dev);
    return cudaGetLastError();
}

cudaError_t launch_mlp_to_bf16(const float* master, void* params, cudaStream_t st) {
    k_mlp_to_bf16<<<(kParams + 255) / 256, 256, 0, st>>>(master, (__nv_bfloat16*)params);
    return cudaGetLastError();
}

}  // namespace spg
