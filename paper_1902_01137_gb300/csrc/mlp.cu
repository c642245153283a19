// mlp.cu -- the learned scattering proposal's network (sm_103a): the FP32
// reference path of its training, the optimiser and the weight packing.
//
// A 9-64-64-64-40 perceptron (GELU, tanh form) maps vertex features to the
// parameters of an 8-lobe von Mises-Fisher mixture that is mixed with the HG
// phase function by one-sample MIS in the tracer (a project addition with no
// counterpart in the paper).  Inference and the default training kernel run
// on the tensor cores (mlp_tc5.cu); this file holds
//  * mlp_train_kernel -- forward, KL-loss gradient and backward pass in FP32
//    on CUDA cores over tiles of 32 records; weight gradients accumulate in
//    shared memory and are added to the global gradient once per block
//    (the exact-arithmetic path, MCRT_TRAIN_FP32);
//  * adam_kernel / pack_kernel -- the optimiser step on FP32 master weights
//    and the BF16 copy the tensor-core kernels read.
#include <cuda_bf16.h>

#include "mcrt_internal.h"
#include "mlp_layout.h"

namespace mcrt {

namespace {

using namespace mlp;
static_assert(kNumParams == kMlpParams, "parameter count");

__device__ __forceinline__ float gelu(float x)
{
    const float c = 0.7978845608028654f;
    return 0.5f * x * (1.0f + tanhf(c * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_grad(float x)
{
    const float c = 0.7978845608028654f;
    const float t = tanhf(c * (x + 0.044715f * x * x * x));
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * x * x);
}

// ---------------------------------------------------------------------------
// Training: forward + KL gradient + backward in FP32, tiles of 32 records
// ---------------------------------------------------------------------------
constexpr int kTR = 32;   // records per tile

struct TrainSmem {
    float W[kMlpParams];
    float G[kMlpParams];
    float X0[kTR][kIn];
    float Z[3][kTR][kH];
    float A[3][kTR][kH];
    float O[kTR][kOut];
    float dO[kTR][kOut];
    float dA[kTR][kH];
    float dir[kTR][3];
    float tgt[kTR];
    float loss;
};

// y[r][o] = b[o] + sum_i W[o][i] x[r][i] for kTR rows; 128 threads.
__device__ __forceinline__ void tdense(const float* W, const float* b, const float* x, int nin, int ldx, int nout,
                                       float* y, int ldy)
{
    for (int idx = threadIdx.x; idx < kTR * nout; idx += blockDim.x) {
        const int r = idx / nout, o = idx % nout;
        float s = b[o];
        const float* wr = W + o * nin;
        const float* xr = x + r * ldx;
        for (int i = 0; i < nin; ++i) s = fmaf(wr[i], xr[i], s);
        y[r * ldy + o] = s;
    }
}

__global__ void __launch_bounds__(128) mlp_train_kernel(const float* __restrict__ params,
                                                       const __nv_bfloat16* __restrict__ feat,
                                                       const float* __restrict__ dirs, const float* __restrict__ tgt,
                                                       int n, float scale, float* __restrict__ grad,
                                                       float* __restrict__ loss_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) { S.W[i] = params[i]; S.G[i] = 0.0f; }
    if (threadIdx.x == 0) S.loss = 0.0f;
    __syncthreads();
    const float* W1 = S.W + kOffW1; const float* b1 = S.W + kOffB1;
    const float* W2 = S.W + kOffW2; const float* b2 = S.W + kOffB2;
    const float* W3 = S.W + kOffW3; const float* b3 = S.W + kOffB3;
    const float* W4 = S.W + kOffW4; const float* b4 = S.W + kOffB4;
    const int tiles = (n + kTR - 1) / kTR;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int row0 = tile * kTR;
        for (int idx = threadIdx.x; idx < kTR * kIn; idx += blockDim.x) {
            const int r = idx / kIn, i = idx % kIn;
            S.X0[r][i] = (row0 + r < n) ? __bfloat162float(feat[(size_t)(row0 + r) * 16 + i]) : 0.0f;
        }
        for (int idx = threadIdx.x; idx < kTR * 3; idx += blockDim.x) {
            const int r = idx / 3, a = idx % 3;
            S.dir[r][a] = (row0 + r < n) ? dirs[(size_t)(row0 + r) * 3 + a] : 0.0f;
        }
        for (int r = threadIdx.x; r < kTR; r += blockDim.x) S.tgt[r] = (row0 + r < n) ? tgt[row0 + r] * scale : 0.0f;
        __syncthreads();
        // forward
        tdense(W1, b1, &S.X0[0][0], kIn, kIn, kH, &S.Z[0][0][0], kH);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kTR * kH; idx += blockDim.x) (&S.A[0][0][0])[idx] = gelu((&S.Z[0][0][0])[idx]);
        __syncthreads();
        tdense(W2, b2, &S.A[0][0][0], kH, kH, kH, &S.Z[1][0][0], kH);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kTR * kH; idx += blockDim.x) (&S.A[1][0][0])[idx] = gelu((&S.Z[1][0][0])[idx]);
        __syncthreads();
        tdense(W3, b3, &S.A[1][0][0], kH, kH, kH, &S.Z[2][0][0], kH);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kTR * kH; idx += blockDim.x) (&S.A[2][0][0])[idx] = gelu((&S.Z[2][0][0])[idx]);
        __syncthreads();
        tdense(W4, b4, &S.A[2][0][0], kH, kH, kOut, &S.O[0][0], kOut);
        __syncthreads();
        // d(-t log q_vMF)/d outputs, one thread per record
        if (threadIdx.x < kTR) {
            const int r = threadIdx.x;
            const float* raw = S.O[r];
            const float* w = S.dir[r];
            float mx = -3.0e38f;
            for (int j = 0; j < kLobes; ++j) mx = fmaxf(mx, raw[5 * j + 4]);
            float pi[kLobes], f[kLobes], s = 0.0f;
            for (int j = 0; j < kLobes; ++j) { pi[j] = expf(raw[5 * j + 4] - mx); s += pi[j]; }
            float q = 0.0f;
            float mu[kLobes][3], kap[kLobes], nrm[kLobes], cc[kLobes];
            for (int j = 0; j < kLobes; ++j) {
                pi[j] /= s;
                const float x = raw[5 * j], y = raw[5 * j + 1], z = raw[5 * j + 2];
                nrm[j] = sqrtf(x * x + y * y + z * z);
                if (nrm[j] < 1e-12f) { mu[j][0] = 0.0f; mu[j][1] = 0.0f; mu[j][2] = 1.0f; }
                else { mu[j][0] = x / nrm[j]; mu[j][1] = y / nrm[j]; mu[j][2] = z / nrm[j]; }
                kap[j] = (raw[5 * j + 3] > 20.0f ? raw[5 * j + 3] : log1pf(expf(raw[5 * j + 3]))) + 1e-3f;
                cc[j] = mu[j][0] * w[0] + mu[j][1] * w[1] + mu[j][2] * w[2];
                f[j] = kap[j] / (2.0f * kPi * (-expm1f(-2.0f * kap[j]))) * expf(kap[j] * (cc[j] - 1.0f));
                q += pi[j] * f[j];
            }
            const float tr = S.tgt[r];
            const float qs = fmaxf(q, 1e-30f);
            if (tr != 0.0f) atomicAdd(&S.loss, -tr * logf(qs));
            for (int j = 0; j < kLobes; ++j) {
                const float resp = pi[j] * f[j] / qs;
                const float k = kap[j];
                for (int a = 0; a < 3; ++a) {
                    const float dmu = nrm[j] < 1e-12f ? 0.0f : k * (w[a] - cc[j] * mu[j][a]) / nrm[j];
                    S.dO[r][5 * j + a] = -tr * resp * dmu;
                }
                const float e2 = expf(-2.0f * k);
                const float dk = 1.0f / k - 2.0f * e2 / (-expm1f(-2.0f * k)) + (cc[j] - 1.0f);
                const float sig = 1.0f / (1.0f + expf(-raw[5 * j + 3]));
                S.dO[r][5 * j + 3] = -tr * resp * dk * sig;
                S.dO[r][5 * j + 4] = -tr * (resp - pi[j]);
            }
        }
        __syncthreads();
        // layer 4 gradients and dA3
        for (int idx = threadIdx.x; idx < kOut * kH; idx += blockDim.x) {
            const int o = idx / kH, i = idx % kH;
            float s = 0.0f;
            for (int r = 0; r < kTR; ++r) s = fmaf(S.dO[r][o], S.A[2][r][i], s);
            S.G[kOffW4 + idx] += s;
        }
        for (int o = threadIdx.x; o < kOut; o += blockDim.x) {
            float s = 0.0f;
            for (int r = 0; r < kTR; ++r) s += S.dO[r][o];
            S.G[kOffB4 + o] += s;
        }
        for (int idx = threadIdx.x; idx < kTR * kH; idx += blockDim.x) {
            const int r = idx / kH, i = idx % kH;
            float s = 0.0f;
            for (int o = 0; o < kOut; ++o) s = fmaf(W4[o * kH + i], S.dO[r][o], s);
            S.dA[r][i] = s * gelu_grad(S.Z[2][r][i]);          // dZ3
        }
        __syncthreads();
        // layers 3, 2, 1
        for (int L = 2; L >= 0; --L) {
            const int nin = (L == 0) ? kIn : kH;
            const float* inp = (L == 0) ? &S.X0[0][0] : &S.A[L - 1][0][0];
            const int ldin = (L == 0) ? kIn : kH;
            const int offW = (L == 0) ? kOffW1 : (L == 1 ? kOffW2 : kOffW3);
            const int offB = (L == 0) ? kOffB1 : (L == 1 ? kOffB2 : kOffB3);
            for (int idx = threadIdx.x; idx < kH * nin; idx += blockDim.x) {
                const int o = idx / nin, i = idx % nin;
                float s = 0.0f;
                for (int r = 0; r < kTR; ++r) s = fmaf(S.dA[r][o], inp[r * ldin + i], s);
                S.G[offW + idx] += s;
            }
            for (int o = threadIdx.x; o < kH; o += blockDim.x) {
                float s = 0.0f;
                for (int r = 0; r < kTR; ++r) s += S.dA[r][o];
                S.G[offB + o] += s;
            }
            if (L > 0) {
                __syncthreads();
                // dZ of the previous layer into Z[L-1] (its pre-activations are no longer needed after)
                for (int idx = threadIdx.x; idx < kTR * kH; idx += blockDim.x) {
                    const int r = idx / kH, i = idx % kH;
                    float s = 0.0f;
                    const float* Wl = S.W + offW;
                    for (int o = 0; o < kH; ++o) s = fmaf(Wl[o * kH + i], S.dA[r][o], s);
                    S.Z[L - 1][r][i] = s * gelu_grad(S.Z[L - 1][r][i]);
                }
                __syncthreads();
                for (int idx = threadIdx.x; idx < kTR * kH; idx += blockDim.x)
                    (&S.dA[0][0])[idx] = (&S.Z[L - 1][0][0])[idx];
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
        if (S.G[i] != 0.0f) atomicAdd(grad + i, S.G[i]);
    if (threadIdx.x == 0 && loss_out) atomicAdd(loss_out, S.loss);
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FP32 master parameters -> padded BF16 weights (nearest) and FP32 biases.
__global__ void pack_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ w, float* __restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kPackedBf16) {
        float v = 0.0f;
        if (i < kPW2) {                                    // layer 1: 64 x 24
            const int o = i / kLd1, k = i % kLd1;
            if (k < kIn) v = p[kOffW1 + o * kIn + k];
        } else if (i < kPW3) {
            const int j = i - kPW2, o = j / kLd, k = j % kLd;
            if (k < kH) v = p[kOffW2 + o * kH + k];
        } else if (i < kPW4) {
            const int j = i - kPW3, o = j / kLd, k = j % kLd;
            if (k < kH) v = p[kOffW3 + o * kH + k];
        } else {
            const int j = i - kPW4, o = j / kLd, k = j % kLd;
            if (k < kH && o < kOut) v = p[kOffW4 + o * kH + k];
        }
        w[i] = __float2bfloat16_rn(v);
    }
    if (i < kPackedBias) {
        float v = 0.0f;
        if (i < 64) v = p[kOffB1 + i];
        else if (i < 128) v = p[kOffB2 + i - 64];
        else if (i < 192) v = p[kOffB3 + i - 128];
        else if (i - 192 < kOut) v = p[kOffB4 + i - 192];
        b[i] = v;
    }
}

}  // namespace

size_t mlp_packed_bf16_elems() { return kPackedBf16; }
size_t mlp_packed_bias_elems() { return kPackedBias; }

cudaError_t launch_mlp_train(const float* params, const void* feat, const float* dirs, const float* tgt, int n,
                             float scale, float* grad, float* loss, int sm_count, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(TrainSmem);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int tiles = (n + kTR - 1) / kTR;
    const int grid = tiles < sm_count ? tiles : sm_count;
    mlp_train_kernel<<<grid, 128, smem, st>>>(params, static_cast<const __nv_bfloat16*>(feat), dirs, tgt, n, scale,
                                               grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps,
                        int t, cudaStream_t st)
{
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(p, m, v, g, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float* p, void* w, float* b, cudaStream_t st)
{
    pack_kernel<<<(kPackedBf16 + 255) / 256, 256, 0, st>>>(p, static_cast<__nv_bfloat16*>(w), b);
    return cudaGetLastError();
}

}  // namespace mcrt
