// learned.cu -- the C ABI of the learned scattering proposal: network state
// (FP32 master parameters, Adam moments, BF16 inference copy), evaluation and
// training entry points.  Kernels live in mlp.cu; the tracer's use of the
// network is in trace.cu / api.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "mcrt_internal.h"

using namespace mcrt;

namespace {

int lfail(mcrt_ctx* ctx, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

#define LCK(ctx, call)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return lfail((ctx), e_ == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA,     \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);     \
    } while (0)

// Xavier-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)), zero
// biases; the uniform of parameter i is Philox(counter (i, 0, "MLP", 0),
// key (seed lo, seed hi)) word 0.
__global__ void xavier_kernel(float* p, uint2 key)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    // layer boundaries of the parameter vector
    const int sizes[8] = {64 * 9, 64, 64 * 64, 64, 64 * 64, 64, 40 * 64, 40};
    const int fan[8][2] = {{9, 64}, {0, 0}, {64, 64}, {0, 0}, {64, 64}, {0, 0}, {64, 40}, {0, 0}};
    int off = 0, L = 0;
    while (L < 7 && i >= off + sizes[L]) { off += sizes[L]; ++L; }
    if (fan[L][0] == 0) { p[i] = 0.0f; return; }
    const float a = sqrtf(6.0f / (float)(fan[L][0] + fan[L][1]));
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 0u, 0x4D4C5000u, 0u), key);
    p[i] = (2.0f * u01(r.x) - 1.0f) * a;
}

// FP32 rows (n x cols) -> BF16 rows of stride ld, zero padded.
__global__ void f32_to_bf16_rows_kernel(const float* __restrict__ src, int n, int cols, __nv_bfloat16* dst, int ld)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * ld) return;
    const int r = (int)(i / ld), c = (int)(i % ld);
    dst[i] = __float2bfloat16_rn(c < cols ? src[(size_t)r * cols + c] : 0.0f);
}

int alloc_proposal(mcrt_ctx* ctx, mcrt_proposal* P)
{
    const size_t np = kMlpParams * sizeof(float);
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&P->d_params), np, ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&P->d_m), np, ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&P->d_v), np, ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&P->d_grad), np, ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&P->d_loss), sizeof(float), ctx->stream));
    LCK(ctx, cudaMallocAsync(&P->d_wbf, mlp_packed_bf16_elems() * 2, ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&P->d_bias), mlp_packed_bias_elems() * sizeof(float),
                             ctx->stream));
    LCK(ctx, cudaMemsetAsync(P->d_m, 0, np, ctx->stream));
    LCK(ctx, cudaMemsetAsync(P->d_v, 0, np, ctx->stream));
    return MCRT_OK;
}

}  // namespace

namespace mcrt {

cudaError_t launch_xavier(float* p, uint64_t seed, cudaStream_t st)
{
    xavier_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16_rows(const float* src, int n, int cols, void* dst, int ld, cudaStream_t st)
{
    const long long tot = (long long)n * ld;
    if (tot == 0) return cudaSuccess;
    f32_to_bf16_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, n, cols,
                                                                          static_cast<__nv_bfloat16*>(dst), ld);
    return cudaGetLastError();
}

}  // namespace mcrt

extern "C" {

int mcrt_proposal_create(mcrt_ctx* ctx, uint64_t seed, mcrt_proposal** out)
{
    if (!ctx || !out) return lfail(ctx, MCRT_ERR_ARG, "mcrt_proposal_create: NULL argument");
    *out = nullptr;
    LCK(ctx, cudaSetDevice(ctx->device));
    mcrt_proposal* P = new (std::nothrow) mcrt_proposal();
    if (!P) return lfail(ctx, MCRT_ERR_OOM, "mcrt_proposal_create: host allocation failed");
    P->ctx = ctx;
    int rc = alloc_proposal(ctx, P);
    if (rc) { delete P; return rc; }
    ctx->launches += 2;
    LCK(ctx, launch_xavier(P->d_params, seed, ctx->stream));
    LCK(ctx, launch_pack(P->d_params, P->d_wbf, P->d_bias, ctx->stream));
    LCK(ctx, cudaStreamSynchronize(ctx->stream));
    *out = P;
    return MCRT_OK;
}

int mcrt_proposal_destroy(mcrt_proposal* P)
{
    if (!P) return lfail(nullptr, MCRT_ERR_ARG, "mcrt_proposal_destroy: NULL");
    mcrt_ctx* ctx = P->ctx;
    for (void* p : {(void*)P->d_params, (void*)P->d_m, (void*)P->d_v, (void*)P->d_grad, (void*)P->d_loss, P->d_wbf,
                    (void*)P->d_bias})
        if (p) cudaFreeAsync(p, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    delete P;
    return MCRT_OK;
}

int mcrt_proposal_nparams(int32_t* n)
{
    if (!n) return MCRT_ERR_ARG;
    *n = kMlpParams;
    return MCRT_OK;
}

int mcrt_proposal_set_params(mcrt_proposal* P, const float* host, size_t n)
{
    if (!P || !host) return lfail(P ? P->ctx : nullptr, MCRT_ERR_ARG, "mcrt_proposal_set_params: NULL argument");
    mcrt_ctx* ctx = P->ctx;
    if (n != (size_t)kMlpParams) return lfail(ctx, MCRT_ERR_ARG, "mcrt_proposal_set_params: need %d values", kMlpParams);
    LCK(ctx, cudaSetDevice(ctx->device));
    LCK(ctx, cudaMemcpyAsync(P->d_params, host, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    LCK(ctx, cudaMemsetAsync(P->d_m, 0, n * sizeof(float), ctx->stream));
    LCK(ctx, cudaMemsetAsync(P->d_v, 0, n * sizeof(float), ctx->stream));
    P->step = 0;
    ctx->launches++;
    LCK(ctx, launch_pack(P->d_params, P->d_wbf, P->d_bias, ctx->stream));
    LCK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

int mcrt_proposal_set_training(mcrt_proposal* P, int32_t mode)
{
    if (!P) return lfail(nullptr, MCRT_ERR_ARG, "mcrt_proposal_set_training: NULL proposal");
    if (mode != MCRT_TRAIN_TENSOR && mode != MCRT_TRAIN_FP32)
        return lfail(P->ctx, MCRT_ERR_ARG, "mcrt_proposal_set_training: bad mode %d", mode);
    P->train_mode = mode;
    return MCRT_OK;
}

int mcrt_proposal_get_params(const mcrt_proposal* P, float* host, size_t n)
{
    if (!P || !host) return lfail(P ? P->ctx : nullptr, MCRT_ERR_ARG, "mcrt_proposal_get_params: NULL argument");
    mcrt_ctx* ctx = P->ctx;
    if (n < (size_t)kMlpParams) return lfail(ctx, MCRT_ERR_BOUNDS, "mcrt_proposal_get_params: need %d values", kMlpParams);
    LCK(ctx, cudaMemcpyAsync(host, P->d_params, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    LCK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

int mcrt_proposal_get_adam(const mcrt_proposal* P, float* host_m, float* host_v, size_t n, int64_t* step)
{
    const char* who = "mcrt_proposal_get_adam";
    if (!P || !host_m || !host_v || !step) return lfail(P ? P->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = P->ctx;
    if (n < (size_t)kMlpParams) return lfail(ctx, MCRT_ERR_BOUNDS, "%s: need %d values", who, kMlpParams);
    LCK(ctx, cudaSetDevice(ctx->device));
    LCK(ctx, cudaMemcpyAsync(host_m, P->d_m, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    LCK(ctx, cudaMemcpyAsync(host_v, P->d_v, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    LCK(ctx, cudaStreamSynchronize(ctx->stream));
    *step = P->step;
    return MCRT_OK;
}

int mcrt_proposal_set_adam(mcrt_proposal* P, const float* host_m, const float* host_v, size_t n, int64_t step)
{
    const char* who = "mcrt_proposal_set_adam";
    if (!P || !host_m || !host_v) return lfail(P ? P->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = P->ctx;
    if (n < (size_t)kMlpParams) return lfail(ctx, MCRT_ERR_BOUNDS, "%s: need %d values", who, kMlpParams);
    if (step < 0 || step > (int64_t)1 << 30) return lfail(ctx, MCRT_ERR_ARG, "%s: bad step count", who);
    for (int i = 0; i < kMlpParams; ++i)
        if (!std::isfinite(host_m[i]) || !(host_v[i] >= 0.0f) || !std::isfinite(host_v[i]))
            return lfail(ctx, MCRT_ERR_ARG, "%s: moment %d not finite (or second moment < 0)", who, i);
    LCK(ctx, cudaSetDevice(ctx->device));
    LCK(ctx, cudaMemcpyAsync(P->d_m, host_m, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    LCK(ctx, cudaMemcpyAsync(P->d_v, host_v, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    LCK(ctx, cudaStreamSynchronize(ctx->stream));
    P->step = (int)step;
    return MCRT_OK;
}

int mcrt_proposal_eval(mcrt_proposal* P, const float* host_feat, size_t n, float* host_mix, float* host_raw)
{
    NvtxRange nvtx_range("mcrt_proposal_eval");
    if (!P || !host_feat || !host_mix) return lfail(P ? P->ctx : nullptr, MCRT_ERR_ARG, "mcrt_proposal_eval: NULL argument");
    mcrt_ctx* ctx = P->ctx;
    if (n == 0) return MCRT_OK;
    if (n > (size_t)(1 << 28)) return lfail(ctx, MCRT_ERR_ARG, "mcrt_proposal_eval: too many rows");
    LCK(ctx, cudaSetDevice(ctx->device));
    float* d_f32 = nullptr;
    void* d_feat = nullptr;
    float *d_mix = nullptr, *d_raw = nullptr;
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&d_f32), n * 9 * sizeof(float), ctx->stream));
    LCK(ctx, cudaMallocAsync(&d_feat, n * 16 * 2, ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&d_mix), n * 40 * sizeof(float), ctx->stream));
    if (host_raw) LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&d_raw), n * 40 * sizeof(float), ctx->stream));
    cudaError_t e = cudaMemcpyAsync(d_f32, host_feat, n * 9 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) { ctx->launches++; e = launch_f32_to_bf16_rows(d_f32, (int)n, 9, d_feat, 16, ctx->stream); }
    if (e == cudaSuccess) {
        ctx->launches++;
        e = launch_mlp_infer(P->d_wbf, P->d_bias, d_feat, (int)n, d_mix, d_raw, ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_mix, d_mix, n * 40 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && host_raw)
        e = cudaMemcpyAsync(host_raw, d_raw, n * 40 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFreeAsync(d_f32, ctx->stream);
    cudaFreeAsync(d_feat, ctx->stream);
    cudaFreeAsync(d_mix, ctx->stream);
    if (d_raw) cudaFreeAsync(d_raw, ctx->stream);
    LCK(ctx, e);
    int terr = 0;
    LCK(ctx, tc5_take_error(&terr, ctx->stream));
    if (terr) return lfail(ctx, MCRT_ERR_TIMEOUT, "mcrt_proposal_eval: a tensor-core wait ran out");
    return MCRT_OK;
}

int mcrt_proposal_train_step(mcrt_proposal* P, const float* host_feat, const float* host_dirs,
                             const float* host_targets, size_t n, float lr, float* loss_out, float* host_grad)
{
    NvtxRange nvtx_range("mcrt_proposal_train_step");
    if (!P || !host_feat || !host_dirs || !host_targets)
        return lfail(P ? P->ctx : nullptr, MCRT_ERR_ARG, "mcrt_proposal_train_step: NULL argument");
    mcrt_ctx* ctx = P->ctx;
    if (n == 0 || n > (size_t)(1 << 26)) return lfail(ctx, MCRT_ERR_ARG, "mcrt_proposal_train_step: bad record count");
    if (!(lr >= 0.0f)) return lfail(ctx, MCRT_ERR_ARG, "mcrt_proposal_train_step: lr must be >= 0");
    LCK(ctx, cudaSetDevice(ctx->device));
    float *d_f32 = nullptr, *d_dirs = nullptr, *d_t = nullptr;
    void* d_feat = nullptr;
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&d_f32), n * 9 * sizeof(float), ctx->stream));
    LCK(ctx, cudaMallocAsync(&d_feat, n * 16 * 2, ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&d_dirs), n * 3 * sizeof(float), ctx->stream));
    LCK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&d_t), n * sizeof(float), ctx->stream));
    cudaError_t e = cudaMemcpyAsync(d_f32, host_feat, n * 9 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_dirs, host_dirs, n * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, host_targets, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) { ctx->launches++; e = launch_f32_to_bf16_rows(d_f32, (int)n, 9, d_feat, 16, ctx->stream); }
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_grad, 0, kMlpParams * sizeof(float), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_loss, 0, sizeof(float), ctx->stream);
    if (e == cudaSuccess) {
        ctx->launches++;
        e = P->train_mode == MCRT_TRAIN_FP32
                ? launch_mlp_train(P->d_params, d_feat, d_dirs, d_t, (int)n, 1.0f / (float)n, P->d_grad, P->d_loss,
                                   ctx->sm_count, ctx->stream)
                : launch_mlp_train_tc(P->d_wbf, P->d_bias, P->d_params, d_feat, d_dirs, d_t, (int)n, 1.0f / (float)n,
                                      P->d_grad, P->d_loss, ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess && host_grad)
        e = cudaMemcpyAsync(host_grad, P->d_grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    float loss = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, P->d_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && lr > 0.0f) {
        P->step++;
        ctx->launches += 2;
        e = launch_adam(P->d_params, P->d_m, P->d_v, P->d_grad, kMlpParams, lr, 0.9f, 0.999f, 1e-8f, P->step,
                        ctx->stream);
        if (e == cudaSuccess) e = launch_pack(P->d_params, P->d_wbf, P->d_bias, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFreeAsync(d_f32, ctx->stream);
    cudaFreeAsync(d_feat, ctx->stream);
    cudaFreeAsync(d_dirs, ctx->stream);
    cudaFreeAsync(d_t, ctx->stream);
    LCK(ctx, e);
    int terr = 0;
    LCK(ctx, tc5_take_error(&terr, ctx->stream));
    if (terr) return lfail(ctx, MCRT_ERR_TIMEOUT, "mcrt_proposal_train_step: a tensor-core wait ran out");
    if (loss_out) *loss_out = loss;
    return MCRT_OK;
}

int mcrt_proposal_apply_gradient(mcrt_proposal* P, const float* host_grad, float lr)
{
    NvtxRange nvtx_range("mcrt_proposal_apply_gradient");
    const char* who = "mcrt_proposal_apply_gradient";
    if (!P || !host_grad) return lfail(P ? P->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = P->ctx;
    if (!(lr > 0.0f)) return lfail(ctx, MCRT_ERR_ARG, "%s: lr must be > 0", who);
    for (int i = 0; i < kMlpParams; ++i)
        if (!std::isfinite(host_grad[i])) return lfail(ctx, MCRT_ERR_ARG, "%s: gradient entry %d not finite", who, i);
    LCK(ctx, cudaSetDevice(ctx->device));
    cudaError_t e = cudaMemcpyAsync(P->d_grad, host_grad, kMlpParams * sizeof(float), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess) {
        P->step++;
        ctx->launches += 2;
        e = launch_adam(P->d_params, P->d_m, P->d_v, P->d_grad, kMlpParams, lr, 0.9f, 0.999f, 1e-8f, P->step,
                        ctx->stream);
        if (e == cudaSuccess) e = launch_pack(P->d_params, P->d_wbf, P->d_bias, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    LCK(ctx, e);
    return MCRT_OK;
}

}  // extern "C"
