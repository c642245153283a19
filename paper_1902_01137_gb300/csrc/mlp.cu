// mlp.cu -- the learned scattering proposal's network (sm_103a).
//
// A 9-64-64-64-40 perceptron (GELU, tanh form) maps vertex features to the
// parameters of an 8-lobe von Mises-Fisher mixture that is mixed with the HG
// phase function by one-sample MIS in the tracer (a project addition with no
// counterpart in the paper).
//
//  * mlp_infer_kernel -- tensor cores: mma.sync m16n8k16, BF16 operands,
//    FP32 accumulation.  A warp owns 32 rows; the FP32 accumulator fragment
//    of one layer is re-packed in registers as the BF16 A fragment of the
//    next (no shared-memory round trip); weights are staged once per block
//    in shared memory with padded rows (conflict-free fragment loads).  The
//    epilogue turns the 40 outputs of a row into unit axes, concentrations
//    and softmax weights.
//  * mlp_train_kernel -- forward, KL-loss gradient and backward pass in FP32
//    on CUDA cores over tiles of 32 records; weight gradients accumulate in
//    shared memory and are added to the global gradient once per block.
//    (2^20 records cost about 7e10 flops per step.)
//  * adam_kernel / pack_kernel -- the optimiser step on FP32 master weights
//    and the BF16 copy used for inference.
//
// Parameter vector (11,560 floats, shared convention with the host API):
// W1[64][9], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[40][64], b4[40].
#include <cuda_bf16.h>

#include "mcrt_internal.h"

namespace mcrt {

namespace {

constexpr int kIn = 9, kH = 64, kOut = 40, kLobes = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kOut * kH;
static_assert(kOffB4 + kOut == kMlpParams, "parameter count");

// Padded BF16 inference layout: rows of k values, row strides 24 (layer 1,
// k padded 9 -> 16) and 72 (k = 64), layer 4 padded to 48 rows.
constexpr int kLd1 = 24, kLd = 72;
constexpr int kPW1 = 0, kPW2 = kPW1 + 64 * kLd1, kPW3 = kPW2 + 64 * kLd, kPW4 = kPW3 + 64 * kLd;
constexpr int kPackedBf16 = kPW4 + 48 * kLd;                // 14,208 bf16
constexpr int kPackedBias = 64 * 3 + 48;                      // fp32

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

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float softplus_f(float x) { return x > 20.0f ? x : log1pf(__expf(x)); }

// ---------------------------------------------------------------------------
// Inference
// ---------------------------------------------------------------------------
// One dense layer on a warp's 32 rows (2 m-tiles): acc[m][j][4] = bias +
// A (32 x 16*KT) * W^T for NT n-tiles; A fragments are given per m-tile and
// k-tile.
template <int KT, int NT>
__device__ __forceinline__ void dense_mma(const __nv_bfloat16* W, int ld, const float* bias, const uint32_t (*A)[KT][4],
                                          float (*acc)[NT][4], int g, int t)
{
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
            acc[m][j][0] = b0; acc[m][j][1] = b1; acc[m][j][2] = b0; acc[m][j][3] = b1;
        }
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            const uint32_t* wr = reinterpret_cast<const uint32_t*>(W + (8 * j + g) * ld + 16 * kk + 2 * t);
            const uint32_t b0 = wr[0], b1 = wr[4];
#pragma unroll
            for (int m = 0; m < 2; ++m) mma_bf16(acc[m][j], A[m][kk][0], A[m][kk][1], A[m][kk][2], A[m][kk][3], b0, b1);
        }
}

// GELU and re-pack of a 64-wide accumulator as the next layer's A fragments.
__device__ __forceinline__ void gelu_pack(float (*acc)[8][4], uint32_t (*A)[4][4])
{
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const float* c0 = acc[m][2 * kk];
            const float* c1 = acc[m][2 * kk + 1];
            A[m][kk][0] = pack_bf16(gelu(c0[0]), gelu(c0[1]));
            A[m][kk][1] = pack_bf16(gelu(c0[2]), gelu(c0[3]));
            A[m][kk][2] = pack_bf16(gelu(c1[0]), gelu(c1[1]));
            A[m][kk][3] = pack_bf16(gelu(c1[2]), gelu(c1[3]));
        }
}

__global__ void __launch_bounds__(128) mlp_infer_kernel(const __nv_bfloat16* __restrict__ wpacked,
                                                       const float* __restrict__ bpacked,
                                                       const __nv_bfloat16* __restrict__ feat, int n,
                                                       float* __restrict__ mix, float* __restrict__ raw_out)
{
    __shared__ __align__(16) __nv_bfloat16 sW[kPackedBf16];
    __shared__ float sB[kPackedBias];
    __shared__ float sOut[4][16][41];
    for (int i = threadIdx.x; i < kPackedBf16 / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(sW)[i] = reinterpret_cast<const uint32_t*>(wpacked)[i];
    for (int i = threadIdx.x; i < kPackedBias; i += blockDim.x) sB[i] = bpacked[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int tiles = (n + 31) / 32;
    for (int tile = blockIdx.x * 4 + warp; tile < tiles; tile += gridDim.x * 4) {
        const int row0 = tile * 32;
        // layer 1: A fragments straight from the feature rows (16 bf16 each)
        uint32_t A1[2][1][4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int r0 = row0 + 16 * m + g, r1 = r0 + 8;
            const uint32_t* f0 = reinterpret_cast<const uint32_t*>(feat + (size_t)r0 * 16);
            const uint32_t* f1 = reinterpret_cast<const uint32_t*>(feat + (size_t)r1 * 16);
            A1[m][0][0] = r0 < n ? f0[t] : 0u;
            A1[m][0][1] = r1 < n ? f1[t] : 0u;
            A1[m][0][2] = r0 < n ? f0[t + 4] : 0u;
            A1[m][0][3] = r1 < n ? f1[t + 4] : 0u;
        }
        float acc[2][8][4];
        uint32_t A[2][4][4];
        dense_mma<1, 8>(sW + kPW1, kLd1, sB, A1, acc, g, t);
        gelu_pack(acc, A);
        dense_mma<4, 8>(sW + kPW2, kLd, sB + 64, A, acc, g, t);
        gelu_pack(acc, A);
        dense_mma<4, 8>(sW + kPW3, kLd, sB + 128, A, acc, g, t);
        gelu_pack(acc, A);
        float out[2][6][4];
        dense_mma<4, 6>(sW + kPW4, kLd, sB + 192, A, out, g, t);
        // stage the 40 outputs of 16 rows at a time, then one lane per row
#pragma unroll
        for (int m = 0; m < 2; ++m) {
#pragma unroll
            for (int j = 0; j < 5; ++j) {      // columns 40..47 are padding
                sOut[warp][g][8 * j + 2 * t] = out[m][j][0];
                sOut[warp][g][8 * j + 2 * t + 1] = out[m][j][1];
                sOut[warp][g + 8][8 * j + 2 * t] = out[m][j][2];
                sOut[warp][g + 8][8 * j + 2 * t + 1] = out[m][j][3];
            }
            __syncwarp();
            const int row = row0 + 16 * m + lane;
            if (lane < 16 && row < n) {
                const float* r = sOut[warp][lane];
                if (raw_out)
                    for (int i = 0; i < kOut; ++i) raw_out[(size_t)row * kOut + i] = r[i];
                float mx = -3.0e38f;
#pragma unroll
                for (int j = 0; j < kLobes; ++j) mx = fmaxf(mx, r[5 * j + 4]);
                float e[kLobes], s = 0.0f;
#pragma unroll
                for (int j = 0; j < kLobes; ++j) { e[j] = __expf(r[5 * j + 4] - mx); s += e[j]; }
                const float inv_s = 1.0f / s;
                float* o = mix + (size_t)row * kOut;
#pragma unroll
                for (int j = 0; j < kLobes; ++j) {
                    const float x = r[5 * j], y = r[5 * j + 1], z = r[5 * j + 2];
                    const float nn = x * x + y * y + z * z;
                    const float inv = nn > 1e-24f ? rsqrtf(nn) : 0.0f;
                    o[5 * j] = nn > 1e-24f ? x * inv : 0.0f;
                    o[5 * j + 1] = nn > 1e-24f ? y * inv : 0.0f;
                    o[5 * j + 2] = nn > 1e-24f ? z * inv : 1.0f;
                    o[5 * j + 3] = softplus_f(r[5 * j + 3]) + 1e-3f;
                    o[5 * j + 4] = e[j] * inv_s;
                }
            }
            __syncwarp();
        }
    }
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

// ---------------------------------------------------------------------------
// Training on the tensor cores: the same loss and gradient with every dense
// product on mma.sync (BF16 operands, FP32 accumulation).  A warp takes 32
// records: the forward pass keeps each layer's GELU output and GELU
// derivative (BF16) in its shared-memory slab; the loss gradient of the 40
// outputs is computed per record on the CUDA cores (FP32); the backward
// pass runs dA = dZ W (weights transposed once per block) and
// dW += dZ^T A (the records are the reduction dimension) on mma.sync, and
// the block's FP32 gradient accumulates in shared memory before one global
// add.  It is kept transposed (rows = inputs, stride 68 = 4 mod 32 words):
// the 32 lanes of an accumulator fragment then hit 32 different banks.
// ---------------------------------------------------------------------------
constexpr int kTcWarps = 2;
constexpr int kLdA0 = 24;     // feature rows: 16 bf16 + pad
constexpr int kLdT4 = 56;     // W4^T rows: 48 outputs (40 + zero pad) + pad
constexpr int kLdG = 68;      // transposed gradient rows (outputs), 68 = 4 mod 32
// transposed gradient blocks: W1^T (16 rows), W2^T, W3^T, W4^T (64 rows each), biases
constexpr int kG1 = 0, kG2 = kG1 + 16 * kLdG, kG3 = kG2 + 64 * kLdG, kG4 = kG3 + 64 * kLdG;
constexpr int kGb = kG4 + 64 * kLdG, kGsize = kGb + kPackedBias;

struct TcWarpSmem {
    __nv_bfloat16 A0[32 * kLdA0];
    __nv_bfloat16 A[3][32 * kLd];     // GELU outputs of layers 1..3
    __nv_bfloat16 GD[3][32 * kLd];    // GELU derivatives of layers 1..3
    __nv_bfloat16 dZ[2][32 * kLd];    // gradients w.r.t. pre-activations (ping-pong)
    float O[32][41];
    float dO[32][41];                 // output gradient in FP32 (bias 4)
    float dir[32][3];
    float tgt[32];
};

struct TcSmem {
    __nv_bfloat16 W[kPackedBf16];     // forward weights (inference layout)
    __nv_bfloat16 T2[64 * kLd], T3[64 * kLd], T4[64 * kLdT4];   // W^T: rows = inputs
    float B[kPackedBias];
    float G[kGsize];                  // transposed gradient blocks (see kG*)
    TcWarpSmem w[kTcWarps];
    float loss;
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16* lo, const __nv_bfloat16* hi)
{
    return (uint32_t)__bfloat16_as_ushort(*lo) | ((uint32_t)__bfloat16_as_ushort(*hi) << 16);
}

// A fragment (16 x 16 at rows m0, cols k0) of a row-major [m][k] matrix.
__device__ __forceinline__ void frag_a(const __nv_bfloat16* M, int ld, int m0, int k0, int g, int t, uint32_t a[4])
{
    a[0] = ld_pair(M + (m0 + g) * ld + k0 + 2 * t);
    a[1] = ld_pair(M + (m0 + g + 8) * ld + k0 + 2 * t);
    a[2] = ld_pair(M + (m0 + g) * ld + k0 + 2 * t + 8);
    a[3] = ld_pair(M + (m0 + g + 8) * ld + k0 + 2 * t + 8);
}

// A fragment of the transpose of a row-major [k][m] matrix (A[m][k] = M[k][m]).
__device__ __forceinline__ void frag_a_t(const __nv_bfloat16* M, int ld, int m0, int k0, int g, int t, uint32_t a[4])
{
    const __nv_bfloat16* c0 = M + (k0 + 2 * t) * ld;
    const __nv_bfloat16* c8 = M + (k0 + 2 * t + 8) * ld;
    a[0] = pack2(c0 + m0 + g, c0 + ld + m0 + g);
    a[1] = pack2(c0 + m0 + g + 8, c0 + ld + m0 + g + 8);
    a[2] = pack2(c8 + m0 + g, c8 + ld + m0 + g);
    a[3] = pack2(c8 + m0 + g + 8, c8 + ld + m0 + g + 8);
}

// B fragment (16 x 8: k0.., n0..) of B[k][n] stored as rows n ([n][k]).
__device__ __forceinline__ void frag_b_nk(const __nv_bfloat16* M, int ld, int n0, int k0, int g, int t, uint32_t b[2])
{
    b[0] = ld_pair(M + (n0 + g) * ld + k0 + 2 * t);
    b[1] = ld_pair(M + (n0 + g) * ld + k0 + 2 * t + 8);
}

// B fragment of B[k][n] stored as rows k ([k][n]).
__device__ __forceinline__ void frag_b_kn(const __nv_bfloat16* M, int ld, int n0, int k0, int g, int t, uint32_t b[2])
{
    const __nv_bfloat16* c0 = M + (k0 + 2 * t) * ld + n0 + g;
    const __nv_bfloat16* c8 = M + (k0 + 2 * t + 8) * ld + n0 + g;
    b[0] = pack2(c0, c0 + ld);
    b[1] = pack2(c8, c8 + ld);
}

// Forward epilogue of a 64-wide layer: GELU output and derivative to the
// warp's slab, and the GELU output as the next layer's A fragments.
__device__ __forceinline__ void tc_forward_store(float (*acc)[8][4], uint32_t (*An)[4][4], __nv_bfloat16* As,
                                                 __nv_bfloat16* GDs, int g, int t)
{
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float* c = acc[m][2 * kk + h];
                const int col = 8 * (2 * kk + h) + 2 * t;
                const uint32_t top = pack_bf16(gelu(c[0]), gelu(c[1]));
                const uint32_t bot = pack_bf16(gelu(c[2]), gelu(c[3]));
                *reinterpret_cast<uint32_t*>(As + (16 * m + g) * kLd + col) = top;
                *reinterpret_cast<uint32_t*>(As + (16 * m + g + 8) * kLd + col) = bot;
                *reinterpret_cast<uint32_t*>(GDs + (16 * m + g) * kLd + col) = pack_bf16(gelu_grad(c[0]), gelu_grad(c[1]));
                *reinterpret_cast<uint32_t*>(GDs + (16 * m + g + 8) * kLd + col) =
                    pack_bf16(gelu_grad(c[2]), gelu_grad(c[3]));
                An[m][kk][2 * h] = top;
                An[m][kk][2 * h + 1] = bot;
            }
}

// dW[o][i] += sum_r dZ[r][o] X[r][i] over the warp's 32 records, added into
// the block's transposed FP32 gradient Gt[i][o] (stride kLdG; o < nout,
// i < nin).
template <int MT, int NT>
__device__ __forceinline__ void tc_weight_grad(const __nv_bfloat16* dZ, const __nv_bfloat16* X, int ldx, float* Gt,
                                               int nin, int nout, int g, int t)
{
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
        uint32_t a[2][4];
        frag_a_t(dZ, kLd, 16 * mt, 0, g, t, a[0]);
        frag_a_t(dZ, kLd, 16 * mt, 16, g, t, a[1]);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t b[2];
                frag_b_kn(X, ldx, 8 * j, 16 * ks, g, t, b);
                mma_bf16(c, a[ks][0], a[ks][1], a[ks][2], a[ks][3], b[0], b[1]);
            }
            const int o0 = 16 * mt + g, o1 = o0 + 8, i0 = 8 * j + 2 * t;
            if (o0 < nout) {
                if (i0 < nin) atomicAdd(Gt + i0 * kLdG + o0, c[0]);
                if (i0 + 1 < nin) atomicAdd(Gt + (i0 + 1) * kLdG + o0, c[1]);
            }
            if (o1 < nout) {
                if (i0 < nin) atomicAdd(Gt + i0 * kLdG + o1, c[2]);
                if (i0 + 1 < nin) atomicAdd(Gt + (i0 + 1) * kLdG + o1, c[3]);
            }
        }
    }
}

// dZprev[r][i] = (sum_o dZ[r][o] W[o][i]) * GD[r][i], with W^T in T (rows i,
// KS k-steps of 16 outputs); the column sums of dZ (bias gradient of the
// layer the gradient came from) are added to Gb.
template <int KS>
__device__ __forceinline__ void tc_back_input(const __nv_bfloat16* dZ, const __nv_bfloat16* T, int ldt,
                                              const __nv_bfloat16* GD, __nv_bfloat16* dZprev, int g, int t)
{
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        uint32_t a[KS][4];
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) frag_a(dZ, kLd, 16 * m, 16 * ks, g, t, a[ks]);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                uint32_t b[2];
                frag_b_nk(T, ldt, 8 * j, 16 * ks, g, t, b);
                mma_bf16(c, a[ks][0], a[ks][1], a[ks][2], a[ks][3], b[0], b[1]);
            }
            const int col = 8 * j + 2 * t, r0 = 16 * m + g, r1 = r0 + 8;
            const __nv_bfloat16* gd0 = GD + r0 * kLd + col;
            const __nv_bfloat16* gd1 = GD + r1 * kLd + col;
            *reinterpret_cast<uint32_t*>(dZprev + r0 * kLd + col) =
                pack_bf16(c[0] * __bfloat162float(gd0[0]), c[1] * __bfloat162float(gd0[1]));
            *reinterpret_cast<uint32_t*>(dZprev + r1 * kLd + col) =
                pack_bf16(c[2] * __bfloat162float(gd1[0]), c[3] * __bfloat162float(gd1[1]));
        }
    }
}

// Bias gradient: column sums of a warp's dZ (32 x ncols) into Gb.
__device__ __forceinline__ void tc_bias_grad(const __nv_bfloat16* dZ, int ncols, float* Gb, int lane)
{
    for (int c = lane; c < ncols; c += 32) {
        float s = 0.0f;
        for (int r = 0; r < 32; ++r) s += __bfloat162float(dZ[r * kLd + c]);
        atomicAdd(Gb + c, s);
    }
}

// The same over the FP32 output gradient (bias 4).
__device__ __forceinline__ void tc_bias_grad_f32(const float (*dO)[41], float* Gb, int lane)
{
    for (int c = lane; c < kOut; c += 32) {
        float s = 0.0f;
        for (int r = 0; r < 32; ++r) s += dO[r][c];
        atomicAdd(Gb + c, s);
    }
}

__global__ void __launch_bounds__(32 * kTcWarps) mlp_train_tc_kernel(
    const __nv_bfloat16* __restrict__ wpacked, const float* __restrict__ bpacked, const float* __restrict__ params,
    const __nv_bfloat16* __restrict__ feat, const float* __restrict__ dirs, const float* __restrict__ tgt, int n,
    float scale, float* __restrict__ grad, float* __restrict__ loss_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    for (int i = threadIdx.x; i < kPackedBf16 / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(S.W)[i] = reinterpret_cast<const uint32_t*>(wpacked)[i];
    for (int i = threadIdx.x; i < kPackedBias; i += blockDim.x) S.B[i] = bpacked[i];
    for (int i = threadIdx.x; i < kGsize; i += blockDim.x) S.G[i] = 0.0f;
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
        const int i = idx / 64, o = idx % 64;       // T[i][o] = W[o][i]
        S.T2[i * kLd + o] = __float2bfloat16_rn(params[kOffW2 + o * kH + i]);
        S.T3[i * kLd + o] = __float2bfloat16_rn(params[kOffW3 + o * kH + i]);
    }
    for (int idx = threadIdx.x; idx < 64 * 48; idx += blockDim.x) {
        const int i = idx / 48, o = idx % 48;
        S.T4[i * kLdT4 + o] = __float2bfloat16_rn(o < kOut ? params[kOffW4 + o * kH + i] : 0.0f);
    }
    if (threadIdx.x == 0) S.loss = 0.0f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    TcWarpSmem& X = S.w[warp];
    const int tiles = (n + 31) / 32;
    for (int tile = blockIdx.x * kTcWarps + warp; tile < tiles; tile += gridDim.x * kTcWarps) {
        const int row = tile * 32 + lane;
        const bool ok = row < n;
        {   // the lane's record: features (16 bf16), direction, target
            const uint32_t* f = reinterpret_cast<const uint32_t*>(feat + (size_t)row * 16);
            uint32_t* a0 = reinterpret_cast<uint32_t*>(X.A0 + lane * kLdA0);
#pragma unroll
            for (int q = 0; q < 8; ++q) a0[q] = ok ? f[q] : 0u;
            for (int a = 0; a < 3; ++a) X.dir[lane][a] = ok ? dirs[(size_t)row * 3 + a] : 0.0f;
            X.tgt[lane] = ok ? tgt[row] * scale : 0.0f;
        }
        __syncwarp();
        // ---- forward
        uint32_t A1[2][1][4];
        frag_a(X.A0, kLdA0, 0, 0, g, t, A1[0][0]);
        frag_a(X.A0, kLdA0, 16, 0, g, t, A1[1][0]);
        float acc[2][8][4];
        uint32_t A[2][4][4];
        dense_mma<1, 8>(S.W + kPW1, kLd1, S.B, A1, acc, g, t);
        tc_forward_store(acc, A, X.A[0], X.GD[0], g, t);
        dense_mma<4, 8>(S.W + kPW2, kLd, S.B + 64, A, acc, g, t);
        tc_forward_store(acc, A, X.A[1], X.GD[1], g, t);
        dense_mma<4, 8>(S.W + kPW3, kLd, S.B + 128, A, acc, g, t);
        tc_forward_store(acc, A, X.A[2], X.GD[2], g, t);
        float out[2][6][4];
        dense_mma<4, 6>(S.W + kPW4, kLd, S.B + 192, A, out, g, t);
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                X.O[16 * m + g][8 * j + 2 * t] = out[m][j][0];
                X.O[16 * m + g][8 * j + 2 * t + 1] = out[m][j][1];
                X.O[16 * m + g + 8][8 * j + 2 * t] = out[m][j][2];
                X.O[16 * m + g + 8][8 * j + 2 * t + 1] = out[m][j][3];
            }
        __syncwarp();
        // ---- d(-t log q_vMF)/d outputs: one lane per record, FP32
        {
            const float* raw = X.O[lane];
            const float* w = X.dir[lane];
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
            const float tr = X.tgt[lane];
            const float qs = fmaxf(q, 1e-30f);
            if (tr != 0.0f) atomicAdd(&S.loss, -tr * logf(qs));
            __nv_bfloat16* d = X.dZ[0] + lane * kLd;
            for (int j = 0; j < kLobes; ++j) {
                const float resp = pi[j] * f[j] / qs;
                const float k = kap[j];
                float v[5];
                for (int a = 0; a < 3; ++a)
                    v[a] = -tr * resp * (nrm[j] < 1e-12f ? 0.0f : k * (w[a] - cc[j] * mu[j][a]) / nrm[j]);
                const float e2 = expf(-2.0f * k);
                const float dk = 1.0f / k - 2.0f * e2 / (-expm1f(-2.0f * k)) + (cc[j] - 1.0f);
                const float sig = 1.0f / (1.0f + expf(-raw[5 * j + 3]));
                v[3] = -tr * resp * dk * sig;
                v[4] = -tr * (resp - pi[j]);
                for (int a = 0; a < 5; ++a) {
                    d[5 * j + a] = __float2bfloat16_rn(v[a]);
                    X.dO[lane][5 * j + a] = v[a];
                }
            }
            for (int c = kOut; c < 48; ++c) d[c] = __float2bfloat16_rn(0.0f);
        }
        __syncwarp();
        // ---- backward: layer 4, then 3, 2, 1
        tc_bias_grad_f32(X.dO, S.G + kGb + 192, lane);                 // bias 4 (exact FP32)
        tc_weight_grad<3, 8>(X.dZ[0], X.A[2], kLd, S.G + kG4, kH, kOut, g, t);
        tc_back_input<3>(X.dZ[0], S.T4, kLdT4, X.GD[2], X.dZ[1], g, t);
        __syncwarp();
        tc_bias_grad(X.dZ[1], kH, S.G + kGb + 128, lane);
        tc_weight_grad<4, 8>(X.dZ[1], X.A[1], kLd, S.G + kG3, kH, kH, g, t);
        tc_back_input<4>(X.dZ[1], S.T3, kLd, X.GD[1], X.dZ[0], g, t);
        __syncwarp();
        tc_bias_grad(X.dZ[0], kH, S.G + kGb + 64, lane);
        tc_weight_grad<4, 8>(X.dZ[0], X.A[0], kLd, S.G + kG2, kH, kH, g, t);
        tc_back_input<4>(X.dZ[0], S.T2, kLd, X.GD[0], X.dZ[1], g, t);
        __syncwarp();
        tc_bias_grad(X.dZ[1], kH, S.G + kGb, lane);
        tc_weight_grad<4, 2>(X.dZ[1], X.A0, kLdA0, S.G + kG1, kIn, kH, g, t);
        __syncwarp();
    }
    __syncthreads();
    // transposed blocks -> the parameter layout (W[o][i], row = output unit)
    for (int idx = threadIdx.x; idx < kMlpParams; idx += blockDim.x) {
        float v;
        if (idx < kOffB1) { const int o = idx / kIn, i = idx % kIn; v = S.G[kG1 + i * kLdG + o]; }
        else if (idx < kOffW2) v = S.G[kGb + idx - kOffB1];
        else if (idx < kOffB2) { const int q = idx - kOffW2, o = q / kH, i = q % kH; v = S.G[kG2 + i * kLdG + o]; }
        else if (idx < kOffW3) v = S.G[kGb + 64 + idx - kOffB2];
        else if (idx < kOffB3) { const int q = idx - kOffW3, o = q / kH, i = q % kH; v = S.G[kG3 + i * kLdG + o]; }
        else if (idx < kOffW4) v = S.G[kGb + 128 + idx - kOffB3];
        else if (idx < kOffB4) { const int q = idx - kOffW4, o = q / kH, i = q % kH; v = S.G[kG4 + i * kLdG + o]; }
        else v = S.G[kGb + 192 + idx - kOffB4];
        if (v != 0.0f) atomicAdd(grad + idx, v);
    }
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

cudaError_t launch_mlp_infer(const void* wpacked, const float* bpacked, const void* feat, int n, float* mix,
                             float* raw, int sm_count, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int tiles = (n + 31) / 32;
    int grid = (tiles + 3) / 4;
    if (grid > sm_count * 8) grid = sm_count * 8;
    mlp_infer_kernel<<<grid, 128, 0, st>>>(static_cast<const __nv_bfloat16*>(wpacked), bpacked,
                                           static_cast<const __nv_bfloat16*>(feat), n, mix, raw);
    return cudaGetLastError();
}

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

cudaError_t launch_mlp_train_tc(const void* wpacked, const float* bpacked, const float* params, const void* feat,
                                const float* dirs, const float* tgt, int n, float scale, float* grad, float* loss,
                                int sm_count, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(TcSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = (n + 31) / 32;
    const int want = (tiles + kTcWarps - 1) / kTcWarps;
    const int grid = want < sm_count ? want : sm_count;
    mlp_train_tc_kernel<<<grid, 32 * kTcWarps, smem, st>>>(static_cast<const __nv_bfloat16*>(wpacked), bpacked, params,
                                                            static_cast<const __nv_bfloat16*>(feat), dirs, tgt, n, scale,
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
