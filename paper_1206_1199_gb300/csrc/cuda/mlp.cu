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
//   k_theta_weights, k_theta_lambda, k_theta_choose
//                   the whole per-group selection from raw list statistics
//                   (otoo_learned_theta): range check, standardisation,
//                   budgeted per-group targets normalised to the global RMS
//                   target, the choice over the angle grid.
//   k_group_rms     per-group RMS relative acceleration error (labels).
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

// ---- learned angle from raw list statistics ---------------------------------

constexpr int kThetaBlock = 128;

struct ThetaArgs {
    const uint16_t* wbf16;
    const float* mean;
    const float* std;
    const float* lo;
    const float* hi;
    const float* feat;     // [n][NI - 1]
    const int32_t* count;  // [n]
    int64_t n;
    float theta0, alpha, beta;
};

// Standardised row of group g's statistics with angle th.
__device__ __forceinline__ void theta_row(const ThetaArgs& a, int64_t g, float th, float x[NI])
{
#pragma unroll
    for (int k = 0; k < NI - 1; ++k) x[k] = __fdiv_rn(__fsub_rn(a.feat[g * (NI - 1) + k], a.mean[k]), a.std[k]);
    x[NI - 1] = __fdiv_rn(__fsub_rn(th, a.mean[NI - 1]), a.std[NI - 1]);
}

// Budget weight of every group (0 outside the training range or for a
// non-finite prediction): w = 10^(alpha y0 + beta log10 L), y0 the predicted
// log10 error at theta0, L = 2^feat[0] the list length at theta0; and the
// block's sums of count * w^2 and count over the groups that have a weight,
// in a fixed order (FP64).
__global__ void __launch_bounds__(kThetaBlock) k_theta_weights(const ThetaArgs a, float* __restrict__ wg,
                                                               double* __restrict__ part)
{
    __shared__ float s_w[NP];
    __shared__ double s_a[kThetaBlock], s_b[kThetaBlock];
    load_weights(a.wbf16, s_w);
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double nw2 = 0.0, nn = 0.0;
    if (g < a.n) {
        bool ok = true;
#pragma unroll
        for (int k = 0; k < NI - 1; ++k) {
            const float f = a.feat[g * (NI - 1) + k];
            ok = ok && isfinite(f);
            if (a.lo) ok = ok && f >= a.lo[k] && f <= a.hi[k];
        }
        float w = 0.f;
        if (ok) {
            float x[NI], h1[NH], h2[NH];
            theta_row(a, g, a.theta0, x);
            const float y0 = forward_row(s_w, x, h1, h2);
            // log10 L = feat[0] log10(2)
            const float e = fmaf(a.alpha, y0, a.beta * a.feat[g * (NI - 1)] * 0.30102999566398120f);
            w = isfinite(e) ? exp10f(e) : 0.f;
            if (!(w > 0.f) || !isfinite(w)) w = 0.f;
        }
        wg[g] = w;
        if (w > 0.f) {
            const double c = (double)a.count[g];
            nw2 = c * (double)w * (double)w;
            nn = c;
        }
    }
    s_a[threadIdx.x] = nw2;
    s_b[threadIdx.x] = nn;
    __syncthreads();
    for (int h = kThetaBlock / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_a[threadIdx.x] += s_a[threadIdx.x + h];
            s_b[threadIdx.x] += s_b[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s_a[0];
        part[2 * blockIdx.x + 1] = s_b[0];
    }
}

// lambda = target / sqrt(sum count w^2 / sum count): the common factor that
// makes the particle-weighted RMS of the group targets equal to target.
// One thread sums the block partials in block order.
__global__ void k_theta_lambda(const double* __restrict__ part, int nblk, double target, double* __restrict__ lambda)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblk; ++k) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    lambda[0] = (a > 0.0 && b > 0.0) ? target / sqrt(a / b) : target;
}

// The choice: groups with a weight aim at log10(lambda w), the largest grid
// angle whose prediction is at most that (grid[0] when none); the others,
// and groups with a non-finite prediction, take the fallback angle.
__global__ void __launch_bounds__(kThetaBlock) k_theta_choose(const ThetaArgs a, const float* __restrict__ wg,
                                                              const double* __restrict__ lambda,
                                                              const float* __restrict__ grid, int nth,
                                                              float fallback, float* __restrict__ tgt_out,
                                                              float* __restrict__ out)
{
    __shared__ float s_w[NP];
    load_weights(a.wbf16, s_w);
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    const float w = wg[g];
    if (!(w > 0.f)) {
        if (tgt_out) tgt_out[g] = __int_as_float(0x7fc00000);  // no target: NaN
        out[g] = fallback;
        return;
    }
    const float target = (float)log10(lambda[0] * (double)w);
    if (tgt_out) tgt_out[g] = target;
    float best = grid[0];
    bool bad = false;
    for (int k = 0; k < nth; ++k) {
        float x[NI], h1[NH], h2[NH];
        theta_row(a, g, grid[k], x);
        const float y = forward_row(s_w, x, h1, h2);
        if (!isfinite(y)) bad = true;
        if (y <= target) best = fmaxf(best, grid[k]);
    }
    out[g] = bad ? fallback : best;
}

// Rows standardised with the training set's statistics: (x - mean) / std.
__global__ void k_standardise(const float* __restrict__ x, int64_t n, const float* __restrict__ mean,
                              const float* __restrict__ std, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * NI) return;
    const int k = (int)(i % NI);
    out[i] = __fdiv_rn(__fsub_rn(x[i], mean[k]), std[k]);
}

// Per-group RMS of the relative acceleration error |a - ref| / |ref| over the
// targets [off[g], off[g + 1]) (one warp per group, lanes in a fixed order):
// out[g] = log10(max(rms, floor)).
__global__ void k_group_rms(const double* __restrict__ acc, const double* __restrict__ ref,
                            const int64_t* __restrict__ off, int64_t ng, float floor_v, float* __restrict__ out,
                            uint32_t* __restrict__ status)
{
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= ng) return;
    const int64_t b = off[g], e = off[g + 1];
    if (b < 0 || e <= b) {
        if (lane == 0) {
            atomicOr(status, 1u);
            out[g] = __int_as_float(0x7fc00000);
        }
        return;
    }
    double s = 0.0;
    for (int64_t t = b + lane; t < e; t += 32) {
        double d2 = 0.0, r2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double d = acc[3 * t + c] - ref[3 * t + c];
            d2 = fma(d, d, d2);
            r2 = fma(ref[3 * t + c], ref[3 * t + c], r2);
        }
        s += d2 / r2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[g] = (float)log10(fmax(sqrt(s / (double)(e - b)), (double)floor_v));
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

int otoo_mlp_standardise(const float* x, int64_t n_rows, const float* mean, const float* std, float* out,
                         void* stream)
{
    OTOO_REQUIRE(x && mean && std && out && n_rows >= 0, OTOO_EINVAL, "otoo_mlp_standardise: bad argument");
    if (n_rows == 0) return OTOO_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = n_rows * NI;
    k_standardise<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n_rows, mean, std, out);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int64_t otoo_learned_theta_scratch_floats(int64_t n_groups)
{
    if (n_groups < 1) return 0;
    const int64_t nblk = (n_groups + kThetaBlock - 1) / kThetaBlock;
    // weights, then (aligned to 8 bytes) 2 doubles per block and lambda
    return ((n_groups + 1) & ~(int64_t)1) + 4 * nblk + 2;
}

int otoo_learned_theta(const otoo_theta_net* net, const otoo_theta_rule* rule, const float* feat,
                       const int32_t* count, int64_t n_groups, const float* grid, int32_t n_theta, float* scratch,
                       float* log10_target, float* theta_out, void* stream)
{
    otoo::Range range_("otoo_learned_theta");
    OTOO_REQUIRE(net && rule && feat && count && grid && scratch && theta_out, OTOO_EINVAL,
                 "otoo_learned_theta: NULL pointer");
    OTOO_REQUIRE(net->wbf16 && net->mean && net->std && ((net->lo == nullptr) == (net->hi == nullptr)), OTOO_EINVAL,
                 "otoo_learned_theta: network arrays missing (lo and hi are both set or both NULL)");
    OTOO_REQUIRE(n_theta >= 1 && n_groups >= 0 && n_groups < ((int64_t)1 << 31), OTOO_EINVAL,
                 "otoo_learned_theta: bad sizes");
    OTOO_REQUIRE(rule->target_rms > 0.f && rule->calib > 0.f && rule->theta0 > 0.f && std::isfinite(rule->alpha) &&
                     std::isfinite(rule->beta) && std::isfinite(rule->target_rms * rule->calib),
                 OTOO_EINVAL, "otoo_learned_theta: bad rule");
    OTOO_REQUIRE((reinterpret_cast<uintptr_t>(scratch) & 7) == 0, OTOO_EINVAL,
                 "otoo_learned_theta: scratch must be 8-byte aligned");
    if (n_groups == 0) return OTOO_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ThetaArgs a;
    a.wbf16 = net->wbf16;
    a.mean = net->mean;
    a.std = net->std;
    a.lo = net->lo;
    a.hi = net->hi;
    a.feat = feat;
    a.count = count;
    a.n = n_groups;
    a.theta0 = rule->theta0;
    a.alpha = rule->alpha;
    a.beta = rule->beta;
    const int nblk = (int)((n_groups + kThetaBlock - 1) / kThetaBlock);
    float* wg = scratch;
    double* part = reinterpret_cast<double*>(scratch + ((n_groups + 1) & ~(int64_t)1));
    double* lambda = part + 2 * nblk;
    k_theta_weights<<<nblk, kThetaBlock, 0, s>>>(a, wg, part);
    CUDA_TRY(cudaGetLastError());
    k_theta_lambda<<<1, 32, 0, s>>>(part, nblk, (double)rule->target_rms * (double)rule->calib, lambda);
    CUDA_TRY(cudaGetLastError());
    k_theta_choose<<<nblk, kThetaBlock, 0, s>>>(a, wg, lambda, grid, n_theta, rule->fallback, log10_target,
                                                 theta_out);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_group_rms_error(const double* acc, const double* ref, const int64_t* group_off, int64_t n_groups,
                         float floor_value, float* log10_rms, uint32_t* status, void* stream)
{
    otoo::Range range_("otoo_group_rms_error");
    OTOO_REQUIRE(acc && ref && group_off && log10_rms && status, OTOO_EINVAL, "otoo_group_rms_error: NULL pointer");
    OTOO_REQUIRE(n_groups >= 0 && floor_value > 0.f, OTOO_EINVAL, "otoo_group_rms_error: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    if (n_groups == 0) return OTOO_OK;
    const int64_t threads = 32 * n_groups;
    k_group_rms<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(acc, ref, group_off, n_groups, floor_value,
                                                                  log10_rms, status);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

}  // extern "C"
