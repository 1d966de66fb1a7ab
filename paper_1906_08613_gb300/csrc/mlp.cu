// The learned selector's network: a 3-layer MLP cost model, forward,
// backward and Adam in CUDA (FP32).
//
//   h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3
//   x  : SS_MLP_IN features (op one-hot, log2 n, log2 batch, mode one-hot)
//   y  : SS_MLP_OUT predicted log2(milliseconds), one per kernel configuration
//   loss = sum_r,k mask[r,k] (y[r,k] - t[r,k])^2 / max(1, sum mask)
// Parameters are one flat float array: W1 (H x IN, row-major), b1, W2 (H x H),
// b2, W3 (OUT x H), b3.  The paper names model-based selection as future work
// ("Limitations and future work"); nothing in it fixes the model, so this one
// is the smallest that fits the autotuner's table.
#include <math.h>

#include "ss_internal.h"

namespace ss {
namespace {

constexpr int IN = SS_MLP_IN, H = SS_MLP_HIDDEN, OUT = SS_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + OUT * H, NPARAM = OFF_B3 + OUT;
static_assert(NPARAM == SS_MLP_PARAMS, "parameter layout");

// Per-row record kept for the gradient: h1, h2, dh1 (pre-activation), dh2
// (pre-activation), dy, loss term.
constexpr int REC = H + H + H + H + OUT + 1;
constexpr int WARPS = 4;

// One warp per row: lanes own hidden units j = lane and lane + 32.
__device__ void row_forward(const float *p, const float *x, float *h1, float *h2, float *y)
{
    const int lane = threadIdx.x & 31;
    for (int j = lane; j < H; j += 32) {
        float s = p[OFF_B1 + j];
        for (int i = 0; i < IN; ++i) s = fmaf(p[OFF_W1 + j * IN + i], x[i], s);
        h1[j] = fmaxf(s, 0.0f);
    }
    __syncwarp();
    for (int j = lane; j < H; j += 32) {
        float s = p[OFF_B2 + j];
        for (int i = 0; i < H; ++i) s = fmaf(p[OFF_W2 + j * H + i], h1[i], s);
        h2[j] = fmaxf(s, 0.0f);
    }
    __syncwarp();
    if (lane < OUT) {
        float s = p[OFF_B3 + lane];
        for (int i = 0; i < H; ++i) s = fmaf(p[OFF_W3 + lane * H + i], h2[i], s);
        y[lane] = s;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32 * WARPS) mlp_forward_kernel(const float *p, int nrows, const float *X,
                                                                 float *Y)
{
    __shared__ float s_h[WARPS][2 * H + OUT];
    const int w = threadIdx.x >> 5;
    for (int r = blockIdx.x * WARPS + w; r < nrows; r += gridDim.x * WARPS) {
        float *h1 = s_h[w], *h2 = h1 + H, *y = h2 + H;
        row_forward(p, X + (long)r * IN, h1, h2, y);
        const int lane = threadIdx.x & 31;
        if (lane < OUT) Y[(long)r * OUT + lane] = y[lane];
        __syncwarp();
    }
}

// Forward and backward per row; writes the row's record to rec.
__global__ void __launch_bounds__(32 * WARPS) mlp_rows_kernel(const float *p, int nrows, const float *X,
                                                              const float *T, const float *M, float inv_n,
                                                              float *rec)
{
    __shared__ float s_h[WARPS][2 * H + OUT];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = blockIdx.x * WARPS + w; r < nrows; r += gridDim.x * WARPS) {
        float *h1 = s_h[w], *h2 = h1 + H, *y = h2 + H;
        row_forward(p, X + (long)r * IN, h1, h2, y);
        float *R = rec + (long)r * REC;
        float *Rh1 = R, *Rh2 = R + H, *Rd1 = R + 2 * H, *Rd2 = R + 3 * H, *Rdy = R + 4 * H;
        // dy = 2 m (y - t) / N ; loss term
        float lt = 0.0f;
        if (lane < OUT) {
            const float m = M[(long)r * OUT + lane];
            const float d = y[lane] - T[(long)r * OUT + lane];
            Rdy[lane] = 2.0f * m * d * inv_n;
            lt = m * d * d * inv_n;
        }
        for (int o = 16; o > 0; o >>= 1) lt += __shfl_xor_sync(0xffffffffu, lt, o);
        if (lane == 0) R[4 * H + OUT] = lt;
        __syncwarp();
        // dh2 (pre-activation) = (W3^T dy) * [h2 > 0]
        for (int j = lane; j < H; j += 32) {
            float s = 0.0f;
            for (int k = 0; k < OUT; ++k) s = fmaf(p[OFF_W3 + k * H + j], Rdy[k], s);
            Rd2[j] = h2[j] > 0.0f ? s : 0.0f;
            Rh1[j] = h1[j];
            Rh2[j] = h2[j];
        }
        __syncwarp();
        // dh1 (pre-activation) = (W2^T dh2) * [h1 > 0]
        for (int j = lane; j < H; j += 32) {
            float s = 0.0f;
            for (int k = 0; k < H; ++k) s = fmaf(p[OFF_W2 + k * H + j], Rd2[k], s);
            Rd1[j] = h1[j] > 0.0f ? s : 0.0f;
        }
        __syncwarp();
    }
}

// One thread per parameter: the gradient as a sum over rows (fixed order,
// deterministic).  Thread NPARAM sums the loss.
__global__ void mlp_grad_kernel(int nrows, const float *X, const float *rec, float *G, float *loss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > NPARAM) return;
    float g = 0.0f;
    if (q == NPARAM) {
        for (int r = 0; r < nrows; ++r) g += rec[(long)r * REC + 4 * H + OUT];
        *loss = g;
        return;
    }
    for (int r = 0; r < nrows; ++r) {
        const float *R = rec + (long)r * REC;
        const float *Rh1 = R, *Rh2 = R + H, *Rd1 = R + 2 * H, *Rd2 = R + 3 * H, *Rdy = R + 4 * H;
        const float *x = X + (long)r * IN;
        float v;
        if (q < OFF_B1)      v = Rd1[(q - OFF_W1) / IN] * x[(q - OFF_W1) % IN];
        else if (q < OFF_W2) v = Rd1[q - OFF_B1];
        else if (q < OFF_B2) v = Rd2[(q - OFF_W2) / H] * Rh1[(q - OFF_W2) % H];
        else if (q < OFF_W3) v = Rd2[q - OFF_B2];
        else if (q < OFF_B3) v = Rdy[(q - OFF_W3) / H] * Rh2[(q - OFF_W3) % H];
        else                 v = Rdy[q - OFF_B3];
        g += v;
    }
    G[q] = g;
}

__global__ void mlp_adam_kernel(float *P, const float *G, float *Mm, float *Vv, float c1, float c2,
                                float lr, float b1, float b2, float eps)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    const float g = G[q];
    const float m = b1 * Mm[q] + (1.0f - b1) * g;
    const float v = b2 * Vv[q] + (1.0f - b2) * g * g;
    Mm[q] = m;
    Vv[q] = v;
    const float mh = m / c1, vh = v / c2;
    P[q] -= lr * mh / (sqrtf(vh) + eps);
}

int grid_rows(int nrows)
{
    int g = (nrows + WARPS - 1) / WARPS;
    const int cap = 4 * sm_count();
    return g < 1 ? 1 : (g > cap ? cap : g);
}

}  // namespace
}  // namespace ss

using namespace ss;

extern "C" {

int ss_mlp_workspace_size(int nrows, size_t *bytes)
{
    if (nrows < 0) return -1;
    if (!bytes) return -2;
    *bytes = (size_t)nrows * REC * sizeof(float);
    return 0;
}

int ss_mlp_forward(const float *d_params, int nrows, const float *d_x, float *d_y, void *stream)
{
    if (!d_params) return -1;
    if (nrows < 0) return -2;
    if (nrows > 0 && !d_x) return -3;
    if (nrows > 0 && !d_y) return -4;
    if (nrows == 0) return 0;
    mlp_forward_kernel<<<grid_rows(nrows), 32 * WARPS, 0, static_cast<cudaStream_t>(stream)>>>(d_params, nrows, d_x, d_y);
    return cudaGetLastError() == cudaSuccess ? 0 : SS_ERR_CUDA;
}

int ss_mlp_grad(const float *d_params, int nrows, const float *d_x, const float *d_t, const float *d_mask,
                float mask_total, float *d_grad, float *d_loss, void *d_work, size_t work_bytes, void *stream)
{
    if (!d_params) return -1;
    if (nrows < 1) return -2;
    if (!d_x) return -3;
    if (!d_t) return -4;
    if (!d_mask) return -5;
    if (!(mask_total > 0.0f)) return -6;
    if (!d_grad) return -7;
    if (!d_loss) return -8;
    if (!d_work) return -9;
    if (work_bytes < (size_t)nrows * REC * sizeof(float)) return -10;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *rec = static_cast<float *>(d_work);
    mlp_rows_kernel<<<grid_rows(nrows), 32 * WARPS, 0, st>>>(d_params, nrows, d_x, d_t, d_mask, 1.0f / mask_total, rec);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    mlp_grad_kernel<<<(NPARAM + 1 + 127) / 128, 128, 0, st>>>(nrows, d_x, rec, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? 0 : SS_ERR_CUDA;
}

int ss_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int step, float lr,
                float beta1, float beta2, float eps, void *stream)
{
    if (!d_params) return -1;
    if (!d_grad) return -2;
    if (!d_m) return -3;
    if (!d_v) return -4;
    if (step < 1) return -5;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    mlp_adam_kernel<<<(NPARAM + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        d_params, d_grad, d_m, d_v, c1, c2, lr, beta1, beta2, eps);
    return cudaGetLastError() == cudaSuccess ? 0 : SS_ERR_CUDA;
}

}  // extern "C"
