// Learned opening angle: a 6-32-32-1 multilayer perceptron that predicts a
// group's log10 RMS relative force error from statistics of its interaction
// list and a candidate opening angle.  The paper controls accuracy with the
// absolute MAC parameter Delta (Section II-B, Eq. SW_MAC; Section III-F); this
// network replaces that control by choosing an angle per group.
//
// Kernels
//   k_mlp_forward   one thread per row, bf16 weights widened to FP32 in shared
//                   memory, FP32 accumulation, tanhf activations.
//   k_mlp_backward  one CTA per 128 rows: each thread runs its row forward and
//                   backward, the per-row deltas go to shared memory, then the
//                   threads sum the rows' outer products in fixed row order
//                   into a per-CTA gradient partial (deterministic).
//   k_mlp_adam      one thread per parameter: sums the CTA partials in CTA
//                   order, applies Adam to the FP32 master weight and rounds
//                   the bf16 copy (round to nearest even).
//   k_select_theta  one thread per group: the largest grid angle whose
//                   predicted error meets the target.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../common.h"

using namespace otoo;

namespace {

constexpr int NI = OTOO_MLP_IN;
constexpr int NH = OTOO_MLP_H;
constexpr int NP = OTOO_MLP_NPARAM;
// parameter offsets
constexpr int OW1 = 0;
constexpr int OB1 = OW1 + NH * NI;
constexpr int OW2 = OB1 + NH;
constexpr int OB2 = OW2 + NH * NH;
constexpr int OW3 = OB2 + NH;
constexpr int OB3 = OW3 + NH;
static_assert(OB3 + 1 == NP, "parameter layout");

constexpr int kRowsPerCta = 128;
// per-row record kept in shared memory by the backward kernel
constexpr int kRec = NI + NH + NH + NH + NH + 1;  // x, h1, h2, d1, d2, dy

__device__ __forceinline__ float bf16_to_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ void load_weights(const uint16_t* __restrict__ wbf16, float* s_w)
{
    for (int k = threadIdx.x; k < NP; k += blockDim.x) s_w[k] = bf16_to_f(wbf16[k]);
    __syncthreads();
}

// Forward pass of one row; keeps the activations.
__device__ __forceinline__ float forward_row(const float* __restrict__ w, const float x[NI], float h1[NH], float h2[NH])
{
#pragma unroll
    for (int i = 0; i < NH; ++i) {
        float z = w[OB1 + i];
#pragma unroll
        for (int k = 0; k < NI; ++k) z = fmaf(w[OW1 + i * NI + k], x[k], z);
        h1[i] = tanhf(z);
    }
#pragma unroll 4
    for (int i = 0; i < NH; ++i) {
        float z = w[OB2 + i];
#pragma unroll
        for (int j = 0; j < NH; ++j) z = fmaf(w[OW2 + i * NH + j], h1[j], z);
        h2[i] = tanhf(z);
    }
    float y = w[OB3];
#pragma unroll
    for (int j = 0; j < NH; ++j) y = fmaf(w[OW3 + j], h2[j], y);
    return y;
}

__global__ void k_mlp_forward(const uint16_t* __restrict__ wbf16, const float* __restrict__ x, float* __restrict__ y,
                              int64_t n)
{
    __shared__ float s_w[NP];
    load_weights(wbf16, s_w);
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float xr[NI], h1[NH], h2[NH];
#pragma unroll
    for (int k = 0; k < NI; ++k) xr[k] = x[r * NI + k];
    y[r] = forward_row(s_w, xr, h1, h2);
}

// Loss L = (1/n) sum_r (y_r - t_r)^2 and its gradient, per-CTA partials:
// part[cta][0..NP) = gradient sum over the CTA's rows, part[cta][NP] = sum of
// squared residuals / n.
__global__ void __launch_bounds__(kRowsPerCta) k_mlp_backward(const uint16_t* __restrict__ wbf16,
                                                              const float* __restrict__ x,
                                                              const float* __restrict__ tgt, int64_t n,
                                                              float* __restrict__ part)
{
    extern __shared__ float smem[];
    float* s_w = smem;                 // NP
    float* s_rec = smem + NP;          // kRowsPerCta * kRec
    load_weights(wbf16, s_w);
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerCta;
    const int tid = threadIdx.x;
    const int64_t r = r0 + tid;
    float* rec = s_rec + tid * kRec;
    const float inv_n = 1.0f / (float)n;
    if (r < n) {
        float xr[NI], h1[NH], h2[NH];
#pragma unroll
        for (int k = 0; k < NI; ++k) xr[k] = x[r * NI + k];
        const float yv = forward_row(s_w, xr, h1, h2);
        const float dy = 2.0f * (yv - tgt[r]) * inv_n;
        float d2[NH];
#pragma unroll
        for (int i = 0; i < NH; ++i) d2[i] = dy * s_w[OW3 + i] * (1.0f - h2[i] * h2[i]);
#pragma unroll 4
        for (int j = 0; j < NH; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < NH; ++i) s = fmaf(s_w[OW2 + i * NH + j], d2[i], s);
            rec[NI + 3 * NH + j] = s * (1.0f - h1[j] * h1[j]);  // d1
        }
#pragma unroll
        for (int k = 0; k < NI; ++k) rec[k] = xr[k];
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            rec[NI + i] = h1[i];
            rec[NI + NH + i] = h2[i];
            rec[NI + 2 * NH + i] = d2[i];
        }
        rec[NI + 4 * NH] = dy;
    }
    __syncthreads();
    const int nrows = (n - r0) < kRowsPerCta ? (int)(n - r0) : kRowsPerCta;
    float* out = part + (int64_t)blockIdx.x * (NP + 1);
    for (int p = tid; p < NP; p += blockDim.x) {
        float g = 0.f;
        if (p < OB1) {
            const int i = p / NI, k = p % NI;
            for (int q = 0; q < nrows; ++q) g = fmaf(s_rec[q * kRec + NI + 3 * NH + i], s_rec[q * kRec + k], g);
        } else if (p < OW2) {
            const int i = p - OB1;
            for (int q = 0; q < nrows; ++q) g += s_rec[q * kRec + NI + 3 * NH + i];
        } else if (p < OB2) {
            const int i = (p - OW2) / NH, j = (p - OW2) % NH;
            for (int q = 0; q < nrows; ++q) g = fmaf(s_rec[q * kRec + NI + 2 * NH + i], s_rec[q * kRec + NI + j], g);
        } else if (p < OW3) {
            const int i = p - OB2;
            for (int q = 0; q < nrows; ++q) g += s_rec[q * kRec + NI + 2 * NH + i];
        } else if (p < OB3) {
            const int j = p - OW3;
            for (int q = 0; q < nrows; ++q) g = fmaf(s_rec[q * kRec + NI + 4 * NH], s_rec[q * kRec + NI + NH + j], g);
        } else {
            for (int q = 0; q < nrows; ++q) g += s_rec[q * kRec + NI + 4 * NH];
        }
        out[p] = g;
    }
    // loss partial: recompute residuals from dy (res = dy * n / 2)
    if (tid == 0) {
        float l = 0.f;
        for (int q = 0; q < nrows; ++q) {
            const float res = s_rec[q * kRec + NI + 4 * NH] * (0.5f * (float)n);
            l = fmaf(res, res, l);
        }
        out[NP] = l * inv_n;
    }
}

// Sum the CTA partials (in CTA order) into grad and loss.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, float* __restrict__ grad, float* __restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += part[(int64_t)b * (NP + 1) + p];
    if (p < NP)
        grad[p] = g;
    else if (loss)
        loss[0] = g;
}

// Adam (Kingma & Ba 2015) on the FP32 master weights, bias-corrected, then
// the bf16 copy is refreshed.
__global__ void k_mlp_adam(float* __restrict__ w, uint16_t* __restrict__ wbf16, float* __restrict__ m,
                           float* __restrict__ v, const float* __restrict__ part, int nblk, float lr, float b1,
                           float b2, float eps, float c1, float c2, float* __restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += part[(int64_t)b * (NP + 1) + p];
    if (p == NP) {
        if (loss) loss[0] = g;
        return;
    }
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / c1, vh = vv / c2;
    const float nw = w[p] - lr * mh / (sqrtf(vh) + eps);
    w[p] = nw;
    wbf16[p] = __bfloat16_as_ushort(__float2bfloat16_rn(nw));
}

__global__ void k_to_bf16(const float* __restrict__ w, uint16_t* __restrict__ o, int n)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) o[p] = __bfloat16_as_ushort(__float2bfloat16_rn(w[p]));
}

__global__ void k_select_theta(const uint16_t* __restrict__ wbf16, const float* __restrict__ x,
                               const float* __restrict__ grid, int nth, int64_t ng, float target,
                               const float* __restrict__ target_g, float fallback, float* __restrict__ out)
{
    __shared__ float s_w[NP];
    load_weights(wbf16, s_w);
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    if (target_g) target = target_g[g];
    float best = grid[0];
    bool bad = false;
    for (int k = 0; k < nth; ++k) {
        float xr[NI], h1[NH], h2[NH];
        const float* xs = x + (g * nth + k) * NI;
#pragma unroll
        for (int c = 0; c < NI; ++c) xr[c] = xs[c];
        const float y = forward_row(s_w, xr, h1, h2);
        if (!isfinite(y)) bad = true;
        if (y <= target) best = fmaxf(best, grid[k]);
    }
    out[g] = bad ? fallback : best;
}

#define CUDA_TRY(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return set_error(OTOO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

int backward(const uint16_t* wbf16, const float* x, const float* t, int64_t n, float* scratch, cudaStream_t s,
             int* nblk_out)
{
    const int64_t nb = (n + kRowsPerCta - 1) / kRowsPerCta;
    OTOO_REQUIRE(nb <= (1 << 20), OTOO_EINVAL, "too many rows");
    const size_t sm = sizeof(float) * (NP + (size_t)kRowsPerCta * kRec);
    CUDA_TRY(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_mlp_backward<<<(unsigned)nb, kRowsPerCta, sm, s>>>(wbf16, x, t, n, scratch);
    CUDA_TRY(cudaGetLastError());
    *nblk_out = (int)nb;
    return OTOO_OK;
}

}  // namespace

extern "C" {

int64_t otoo_mlp_scratch_floats(int64_t n_rows)
{
    if (n_rows < 1) return 0;
    return ((n_rows + kRowsPerCta - 1) / kRowsPerCta) * (NP + 1);
}

int otoo_mlp_predict(const uint16_t* wbf16, const float* x, float* y, int64_t n_rows, void* stream)
{
    OTOO_REQUIRE(wbf16 && x && y, OTOO_EINVAL, "otoo_mlp_predict: NULL pointer");
    OTOO_REQUIRE(n_rows >= 0, OTOO_EINVAL, "otoo_mlp_predict: n_rows < 0");
    if (n_rows == 0) return OTOO_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_mlp_forward<<<(unsigned)((n_rows + 127) / 128), 128, 0, s>>>(wbf16, x, y, n_rows);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_mlp_grad(const uint16_t* wbf16, const float* x, const float* target, int64_t n_rows, float* scratch,
                  float* grad, float* loss, void* stream)
{
    OTOO_REQUIRE(wbf16 && x && target && scratch && grad, OTOO_EINVAL, "otoo_mlp_grad: NULL pointer");
    OTOO_REQUIRE(n_rows >= 1, OTOO_EINVAL, "otoo_mlp_grad: n_rows < 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int nb = 0;
    int rc = backward(wbf16, x, target, n_rows, scratch, s, &nb);
    if (rc) return rc;
    k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, s>>>(scratch, nb, grad, loss);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_mlp_train_step(float* w, uint16_t* wbf16, float* m, float* v, float* scratch, const float* x,
                        const float* target, int64_t n_rows, float lr, float beta1, float beta2, float eps_adam,
                        int32_t t, float* loss, void* stream)
{
    otoo::Range range_("otoo_mlp_train_step");
    OTOO_REQUIRE(w && wbf16 && m && v && scratch && x && target, OTOO_EINVAL, "otoo_mlp_train_step: NULL pointer");
    OTOO_REQUIRE(n_rows >= 1 && t >= 1, OTOO_EINVAL, "otoo_mlp_train_step: n_rows and t must be >= 1");
    OTOO_REQUIRE(lr > 0 && beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps_adam > 0, OTOO_EINVAL,
                 "otoo_mlp_train_step: bad Adam hyper-parameters");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int nb = 0;
    int rc = backward(wbf16, x, target, n_rows, scratch, s, &nb);
    if (rc) return rc;
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    k_mlp_adam<<<(NP + 1 + 255) / 256, 256, 0, s>>>(w, wbf16, m, v, scratch, nb, lr, beta1, beta2, eps_adam, c1, c2,
                                                     loss);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_mlp_to_bf16(const float* w, uint16_t* wbf16, int32_t n, void* stream)
{
    OTOO_REQUIRE(w && wbf16 && n >= 0, OTOO_EINVAL, "otoo_mlp_to_bf16: bad argument");
    if (n == 0) return OTOO_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_to_bf16<<<(n + 255) / 256, 256, 0, s>>>(w, wbf16, n);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_select_theta(const uint16_t* wbf16, const float* x, const float* theta_grid, int32_t n_theta,
                      int64_t n_groups, float log10_target, const float* log10_target_per_group, float fallback,
                      float* theta_out, void* stream)
{
    otoo::Range range_("otoo_select_theta");
    OTOO_REQUIRE(wbf16 && x && theta_grid && theta_out, OTOO_EINVAL, "otoo_select_theta: NULL pointer");
    OTOO_REQUIRE(n_theta >= 1 && n_groups >= 0, OTOO_EINVAL, "otoo_select_theta: bad sizes");
    if (n_groups == 0) return OTOO_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_select_theta<<<(unsigned)((n_groups + 127) / 128), 128, 0, s>>>(wbf16, x, theta_grid, n_theta, n_groups,
                                                                      log10_target, log10_target_per_group, fallback,
                                                                      theta_out);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

}  // extern "C"
