// mlp_tc5.cu -- the learned proposal's network on the 5th-generation tensor
// cores of sm_103a (tcgen05 MMA with tensor-memory accumulators).
//
// Both kernels take tiles of 128 rows (records or queued vertices); thread
// r of the CTA's 128 owns row r: it writes the row's operands to shared
// memory and reads the row's accumulators back from TMEM lane r.  One
// thread issues the MMAs of a step and commits them to an mbarrier that
// every thread waits on (a bounded wait: a wait that runs out sets an
// error word, the CTA frees its tensor memory and leaves).  Operands are
// BF16 in the no-swizzle core-matrix layout of tc5.cuh, accumulation FP32.
//
//  * mlp_infer_tc5_kernel -- forward pass; the epilogue turns the 40 outputs
//    of a row into unit lobe axes, concentrations and softmax weights.
//  * mlp_train_tc5_kernel -- forward, gradient of the KL loss with respect
//    to the 40 outputs (FP32, CUDA cores), and the backward pass:
//      dA_{l-1} = dZ_l W_l          M = 128 rows, N = 64, from TMEM
//      dW_l    += dZ_l^T [A_{l-1} 1] M = 64 units, K = 128 rows
//    The weight-gradient accumulators stay in TMEM across all of a CTA's
//    tiles (the records are their reduction dimension) and are added to the
//    global gradient once; the constant-1 column appended to each layer's
//    input gives the bias gradient in the same product.  The GELU
//    derivatives wait in TMEM between the forward and backward passes.
#include <cuda_bf16.h>

#include "mcrt_internal.h"
#include "mlp_layout.h"
#include "tc5.cuh"

namespace mcrt {

namespace {

using namespace mlp;
using namespace tc5;

__device__ int g_tc5_error;        // 1: an MMA wait ran out in some CTA

constexpr int kRows = 128;         // rows per tile (the MMA's M)
constexpr int kCX = 16;            // feature columns (9 used, a ones column at 9 in training)
constexpr int kCH = 72;            // training activations: 64 + a ones column + pad
constexpr int kCD = 64;            // output / pre-activation gradient columns

// shared-memory operand buffers (bytes)
constexpr uint32_t kSzW1 = 64 * 16 * 2, kSzW = 64 * 64 * 2, kSzW4 = 48 * 64 * 2;
constexpr uint32_t kOffSW1 = 0, kOffSW2 = kOffSW1 + kSzW1, kOffSW3 = kOffSW2 + kSzW, kOffSW4 = kOffSW3 + kSzW;
constexpr uint32_t kOffSX = kOffSW4 + kSzW4;                       // 24,576
constexpr uint32_t kSzX = kRows * kCX * 2;

// tensor-memory columns of the training kernel (512 allocated)
constexpr uint32_t cACC = 0;                                      // 64: forward Z, output, dA
constexpr uint32_t cGP1 = 64, cGP2 = 128, cGP3 = 192;             // GELU derivatives, FP32
constexpr uint32_t cG1 = 256, cG2 = 272, cG3 = 344, cG4 = 416;    // dW (M = 64 layout), 16 / 72 / 72 / 72 columns

__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU (tanh form), h = x/2 (1 + tanh u) with u = c (x + a x^3), and its
// derivative h' = (1 + t)/2 + x/2 (1 - t^2) c (1 + 3 a x^2), t = tanh u,
// written as a chain of fused multiply-adds.
constexpr float kGeluC = 0.7978845608028654f;                 // sqrt(2 / pi)
constexpr float kGeluAC = 0.044715f * 0.7978845608028654f;      // a c
constexpr float kGelu3AC = 3.0f * 0.044715f * 0.7978845608028654f;

__device__ __forceinline__ void gelu2(float x, float& h, float& gp)
{
    const float x2 = x * x;
    const float t = tanh_fast(x * fmaf(kGeluAC, x2, kGeluC));
    const float hx = 0.5f * x;
    h = fmaf(hx, t, hx);
    gp = fmaf(hx * fmaf(-t, t, 1.0f), fmaf(kGelu3AC, x2, kGeluC), fmaf(0.5f, t, 0.5f));
}

__device__ __forceinline__ float gelu1(float x)
{
    const float t = tanh_fast(x * fmaf(kGeluAC, x * x, kGeluC));
    const float hx = 0.5f * x;
    return fmaf(hx, t, hx);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void st16(uint8_t* base, uint32_t off, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    *reinterpret_cast<uint4*>(base + off) = make_uint4(a, b, c, d);
}

// The BF16 inference weights (padded row layout) to K-major core-matrix
// operands: W1 64 x 16, W2 and W3 64 x 64, W4 48 x 64 (rows = output units).
__device__ void stage_weights(uint8_t* sm, const __nv_bfloat16* __restrict__ wp, int tid, int nthreads)
{
    const uint4* w = reinterpret_cast<const uint4*>(wp);
    for (int i = tid; i < 64 * 2; i += nthreads) {                 // W1: 64 rows x 2 chunks
        const int o = i >> 1, k = (i & 1) * 8;
        *reinterpret_cast<uint4*>(sm + kOffSW1 + core_off(o, k, 16)) = w[(kPW1 + o * kLd1 + k) / 8];
    }
    for (int i = tid; i < 64 * 8; i += nthreads) {                 // W2, W3: 64 rows x 8 chunks
        const int o = i >> 3, k = (i & 7) * 8;
        *reinterpret_cast<uint4*>(sm + kOffSW2 + core_off(o, k, 64)) = w[(kPW2 + o * kLd + k) / 8];
        *reinterpret_cast<uint4*>(sm + kOffSW3 + core_off(o, k, 64)) = w[(kPW3 + o * kLd + k) / 8];
    }
    for (int i = tid; i < 48 * 8; i += nthreads) {                 // W4: 48 rows x 8 chunks
        const int o = i >> 3, k = (i & 7) * 8;
        *reinterpret_cast<uint4*>(sm + kOffSW4 + core_off(o, k, 64)) = w[(kPW4 + o * kLd + k) / 8];
    }
}

// Make this thread's shared-memory writes visible to the tensor cores, then
// synchronise the CTA (tensor-memory accesses before it are ordered too).
__device__ __forceinline__ void to_mma()
{
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// Every thread waits for the committed MMAs; the result is made uniform so
// that the whole CTA leaves together when a wait ran out.
__device__ __forceinline__ bool from_mma(uint64_t* bar, uint32_t& phase)
{
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    fence_after_sync();
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Mixture parameters of one row's 40 raw outputs: unit axis mu_j,
// concentration kappa_j = softplus + 1e-3, softmax weight pi_j.  The API
// layout holds (mu, kappa, pi) per lobe (40 floats); the tracer's layout
// (kTracerMix floats) holds (mu, kappa, CDF of the weights up to lobe j,
// pi_j C(kappa_j)) with the vMF normalisation C(k) = k / (2 pi (1 - e^-2k)),
// so that a resumed vertex evaluates the mixture density with one
// exponential per lobe.
constexpr int kTracerMix = 48;

__device__ __forceinline__ void mixture_out(const float* r, float* __restrict__ o, bool tracer)
{
    float mx = -3.0e38f;
#pragma unroll
    for (int j = 0; j < kLobes; ++j) mx = fmaxf(mx, r[5 * j + 4]);
    float e[kLobes], s = 0.0f;
#pragma unroll
    for (int j = 0; j < kLobes; ++j) { e[j] = __expf(r[5 * j + 4] - mx); s += e[j]; }
    const float inv_s = 1.0f / s;
    float cdf = 0.0f;
#pragma unroll
    for (int j = 0; j < kLobes; ++j) {
        const float x = r[5 * j], y = r[5 * j + 1], z = r[5 * j + 2];
        const float nn = x * x + y * y + z * z;
        const float inv = nn > 1e-24f ? rsqrtf(nn) : 0.0f;
        const float k = r[5 * j + 3];
        const float kap = (k > 20.0f ? k : log1pf(__expf(k))) + 1e-3f;
        const float pi = e[j] * inv_s;
        const int b = tracer ? 6 * j : 5 * j;
        o[b] = nn > 1e-24f ? x * inv : 0.0f;
        o[b + 1] = nn > 1e-24f ? y * inv : 0.0f;
        o[b + 2] = nn > 1e-24f ? z * inv : 1.0f;
        o[b + 3] = kap;
        if (tracer) {
            cdf += pi;
            o[b + 4] = cdf;
            o[b + 5] = pi * kap / (2.0f * kPi * (-expm1f(-2.0f * kap)));
        } else {
            o[b + 4] = pi;
        }
    }
}

// ---------------------------------------------------------------------------
// Inference
// ---------------------------------------------------------------------------
constexpr uint32_t kInfOffHa = kOffSX + kSzX, kInfOffHb = kInfOffHa + kRows * 64 * 2;
constexpr uint32_t kInfSmem = kInfOffHb + kRows * 64 * 2;          // 61,440 bytes
constexpr uint32_t kInfCols = 64;
static_assert(kRows * (48 + 1) * 4 <= kInfSmem - kInfOffHa, "output staging fits in the two activation buffers");

// One forward epilogue: bias + GELU of the 64 accumulator columns, BF16 to
// the next layer's operand rows.
__device__ __forceinline__ void infer_hidden(uint32_t tacc, const float* __restrict__ bias, uint8_t* H, int row)
{
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tacc + c0, v);
        tmem_wait_ld(v);
        uint32_t p[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            p[j] = pack2(gelu1(__uint_as_float(v[2 * j]) + bias[c0 + 2 * j]),
                         gelu1(__uint_as_float(v[2 * j + 1]) + bias[c0 + 2 * j + 1]));
        st16(H, core_off(row, c0, 64), p[0], p[1], p[2], p[3]);
        st16(H, core_off(row, c0 + 8, 64), p[4], p[5], p[6], p[7]);
    }
}

__global__ void __launch_bounds__(128) mlp_infer_tc5_kernel(const __nv_bfloat16* __restrict__ wpacked,
                                                           const float* __restrict__ bpacked,
                                                           const __nv_bfloat16* __restrict__ feat, int n,
                                                           float* __restrict__ mix, float* __restrict__ raw_out,
                                                           int tracer_layout)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ float sB[kPackedBias];
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    stage_weights(sm, wpacked, tid, 128);
    for (int i = tid; i < kPackedBias; i += 128) sB[i] = bpacked[i];
    if (tid == 0) { mbar_init(&bar, 1); fence_mbar_init(); }
    if (warp == 0) { tmem_alloc(&tbase, kInfCols); tmem_relinquish(); }
    to_mma();
    const uint32_t T = tbase;
    const uint32_t tacc = T + ((uint32_t)(32 * warp) << 16);
    const uint32_t aW1 = smem_addr(sm + kOffSW1), aW2 = smem_addr(sm + kOffSW2), aW3 = smem_addr(sm + kOffSW3);
    const uint32_t aW4 = smem_addr(sm + kOffSW4), aX = smem_addr(sm + kOffSX);
    const uint32_t aHa = smem_addr(sm + kInfOffHa), aHb = smem_addr(sm + kInfOffHb);
    constexpr uint32_t id64 = idesc_bf16(128, 64, false, false), id48 = idesc_bf16(128, 48, false, false);
    uint32_t phase = 0;
    bool ok = true;
    const int tiles = (n + kRows - 1) / kRows;
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int row = tile * kRows + tid;
        uint4 f0 = make_uint4(0u, 0u, 0u, 0u), f1 = f0;
        if (row < n) {
            const uint4* fp = reinterpret_cast<const uint4*>(feat + (size_t)row * 16);
            f0 = __ldg(fp);
            f1 = __ldg(fp + 1);
        }
        *reinterpret_cast<uint4*>(sm + kOffSX + core_off(tid, 0, kCX)) = f0;
        *reinterpret_cast<uint4*>(sm + kOffSX + core_off(tid, 8, kCX)) = f1;
        // layer 1: X (K = 16) -> ACC
        to_mma();
        if (tid == 0) {
            mma_bf16(T, sdesc_kmajor(aX, kCX), sdesc_kmajor(aW1, 16), id64, 0u);
            mma_commit(&bar);
        }
        if (!(ok = from_mma(&bar, phase))) break;
        infer_hidden(tacc, sB, sm + kInfOffHa, tid);
        // layers 2 and 3: K = 64 in four steps, operands alternating between Ha and Hb
        for (int L = 0; L < 2 && ok; ++L) {
            const uint32_t aIn = L == 0 ? aHa : aHb, aWl = L == 0 ? aW2 : aW3;
            to_mma();
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    mma_bf16(T, sdesc_kmajor(aIn + 256u * k, 64), sdesc_kmajor(aWl + 256u * k, 64), id64, k ? 1u : 0u);
                mma_commit(&bar);
            }
            if (!(ok = from_mma(&bar, phase))) break;
            infer_hidden(tacc, sB + 64 * (L + 1), sm + (L == 0 ? kInfOffHb : kInfOffHa), tid);
        }
        if (!ok) break;
        // layer 4: Ha (K = 64) -> 48 output columns (40 used)
        to_mma();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_bf16(T, sdesc_kmajor(aHa + 256u * k, 64), sdesc_kmajor(aW4 + 256u * k, 64), id48, k ? 1u : 0u);
            mma_commit(&bar);
        }
        if (!(ok = from_mma(&bar, phase))) break;
        float r[48];
#pragma unroll
        for (int c0 = 0; c0 < 48; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tacc + c0, v);
            tmem_wait_ld(v);
#pragma unroll
            for (int j = 0; j < 16; ++j) r[c0 + j] = __uint_as_float(v[j]) + sB[192 + c0 + j];
        }
        // the rows' mixtures go through shared memory (the activation
        // buffers are free once layer 4 has run; stride W + 1 words: no bank
        // conflicts) and out with a warp per row, so the stores coalesce
        const int W = tracer_layout ? kTracerMix : kOut;
        float* stage = reinterpret_cast<float*>(sm + kInfOffHa);
        if (row < n) {
            if (raw_out)
                for (int i = 0; i < kOut; ++i) raw_out[(size_t)row * kOut + i] = r[i];
            mixture_out(r, stage + tid * (W + 1), tracer_layout != 0);
        }
        __syncthreads();
        const int nrows = min(kRows, n - tile * kRows);
        for (int rr = warp; rr < nrows; rr += 4)
            for (int c = lane; c < W; c += 32)
                mix[(size_t)(tile * kRows + rr) * W + c] = stage[rr * (W + 1) + c];
    }
    if (!ok && tid == 0) atomicExch(&g_tc5_error, 1);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(T, kInfCols);
    }
}

// ---------------------------------------------------------------------------
// Training
// ---------------------------------------------------------------------------
constexpr uint32_t kTrOffH1 = kOffSX + kSzX, kSzH = kRows * kCH * 2;
constexpr uint32_t kTrOffH2 = kTrOffH1 + kSzH, kTrOffH3 = kTrOffH2 + kSzH;
constexpr uint32_t kTrOffDO = kTrOffH3 + kSzH, kTrOffDZ = kTrOffDO + kRows * kCD * 2;
constexpr uint32_t kTrainSmem = kTrOffDZ + kRows * kCD * 2;        // 116,736 bytes: one CTA per SM
constexpr uint32_t kTrCols = 512;
constexpr int kTrThreads = 256;    // two threads per row: warps w and w + 4 share TMEM lane quarter w

// Forward epilogue of hidden layer l over the thread's 32 columns
// [c1, c1 + 32) (one TMEM load, one wait): bias + GELU to the operand rows
// (BF16), the GELU derivative to TMEM.
__device__ __forceinline__ void train_hidden(uint32_t tl, uint32_t cgp, int c1, const float* __restrict__ bias,
                                             uint8_t* H, int row)
{
    uint32_t v[32];
    tmem_ld32(tl + cACC + c1, v);
    tmem_wait_ld32(v);
    uint32_t p[16], g[32];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float h0, h1, g0, g1;
        gelu2(__uint_as_float(v[2 * j]) + bias[c1 + 2 * j], h0, g0);
        gelu2(__uint_as_float(v[2 * j + 1]) + bias[c1 + 2 * j + 1], h1, g1);
        p[j] = pack2(h0, h1);
        g[2 * j] = __float_as_uint(g0);
        g[2 * j + 1] = __float_as_uint(g1);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) st16(H, core_off(row, c1 + 8 * q, kCH), p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
    tmem_st32(tl + cgp + c1, g);
    tmem_wait_st();
}

// Backward epilogue over the thread's 32 columns (the two TMEM loads in
// flight together): dZ = dA * GELU'(Z) to the operand rows (BF16).
__device__ __forceinline__ void train_dz(uint32_t tl, uint32_t cgp, int c1, uint8_t* DZ, int row)
{
    uint32_t a[32], g[32];
    tmem_ld32(tl + cACC + c1, a);
    tmem_ld32(tl + cgp + c1, g);
    tmem_wait_ld32(a);
    tmem_after_wait32(g);
    uint32_t p[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
        p[j] = pack2(__uint_as_float(a[2 * j]) * __uint_as_float(g[2 * j]),
                     __uint_as_float(a[2 * j + 1]) * __uint_as_float(g[2 * j + 1]));
#pragma unroll
    for (int q = 0; q < 4; ++q) st16(DZ, core_off(row, c1 + 8 * q, kCD), p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
}

// Gradient of -t log q_vMF(w) with respect to the 20 raw outputs of lobes
// 4h .. 4h + 3 of one row (the row's other lobes are the other thread's):
// the softmax maximum and sum and the mixture density are combined through
// shared memory (xch[step][half][row]; every thread of the CTA passes the
// same two barriers); the 20 gradients go to the output-gradient rows as
// BF16.  Returns this half's loss term (the first half carries it).
__device__ __forceinline__ float train_loss_half(uint32_t tl, const float* __restrict__ sB, float (*xch)[2][kRows],
                                                 int row, int h, const float w[3], float t, uint8_t* DO)
{
    const int C0 = 20 * h;
    float raw[20];
    {
        float r48[48];
#pragma unroll
        for (int c0 = 0; c0 < 48; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tl + cACC + c0, v);
            tmem_wait_ld(v);
#pragma unroll
            for (int j = 0; j < 16; ++j) r48[c0 + j] = __uint_as_float(v[j]);
        }
#pragma unroll
        for (int c = 0; c < 20; ++c) raw[c] = (h ? r48[20 + c] : r48[c]) + sB[192 + C0 + c];
    }
    float mx = -3.0e38f;
#pragma unroll
    for (int j = 0; j < 4; ++j) mx = fmaxf(mx, raw[5 * j + 4]);
    xch[0][h][row] = mx;
    __syncthreads();
    mx = fmaxf(xch[0][0][row], xch[0][1][row]);
    float pi[4], s = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) { pi[j] = __expf(raw[5 * j + 4] - mx); s += pi[j]; }
    float mu[4][3], kap[4], nrm[4], cc[4], f[4];
    float q = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float x = raw[5 * j], y = raw[5 * j + 1], z = raw[5 * j + 2];
        nrm[j] = sqrtf(x * x + y * y + z * z);
        const float in = nrm[j] < 1e-12f ? 0.0f : 1.0f / nrm[j];
        mu[j][0] = x * in; mu[j][1] = y * in; mu[j][2] = nrm[j] < 1e-12f ? 1.0f : z * in;
        const float r3 = raw[5 * j + 3];
        kap[j] = (r3 > 20.0f ? r3 : log1pf(__expf(r3))) + 1e-3f;
        cc[j] = mu[j][0] * w[0] + mu[j][1] * w[1] + mu[j][2] * w[2];
        f[j] = kap[j] / (2.0f * kPi * (-expm1f(-2.0f * kap[j]))) * __expf(kap[j] * (cc[j] - 1.0f));
        q += pi[j] * f[j];                      // weights not yet normalised
    }
    xch[1][h][row] = s;
    xch[2][h][row] = q;
    __syncthreads();
    const float inv_s = 1.0f / (xch[1][0][row] + xch[1][1][row]);
    const float qs = fmaxf((xch[2][0][row] + xch[2][1][row]) * inv_s, 1e-30f);
    float d[20];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        pi[j] *= inv_s;
        const float resp = pi[j] * f[j] / qs;
        const float k = kap[j];
        const float sc = nrm[j] < 1e-12f ? 0.0f : -t * resp * k / nrm[j];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[5 * j + a] = sc * (w[a] - cc[j] * mu[j][a]);
        const float e2 = __expf(-2.0f * k);
        const float dk = 1.0f / k - 2.0f * e2 / (-expm1f(-2.0f * k)) + (cc[j] - 1.0f);
        const float sig = 1.0f / (1.0f + __expf(-raw[5 * j + 3]));
        d[5 * j + 3] = -t * resp * dk * sig;
        d[5 * j + 4] = -t * (resp - pi[j]);
    }
#pragma unroll
    for (int c = 0; c < 20; c += 2)      // even columns: a pair never crosses a core matrix
        *reinterpret_cast<uint32_t*>(DO + core_off(row, C0 + c, kCD)) = pack2(d[c], d[c + 1]);
    return (h == 0 && t != 0.0f) ? -t * __logf(qs) : 0.0f;
}

// Add one M = 64 gradient block (rows 16q + lane of lane quarter q's lanes
// 0..15) to the global gradient: W[m][c] for c < ncols at wofs + m * ncols,
// and the bias (column bcol) at bofs + m, for rows m < nrows; the thread
// loads the 16-column chunks [cfrom, cto).
__device__ __forceinline__ void flush_block(uint32_t tl, uint32_t col, int cfrom, int cto, int ncols, int bcol,
                                            int nrows, int wofs, int bofs, float* __restrict__ grad, int quarter,
                                            int lane)
{
    const int m = 16 * quarter + lane;
    for (int c0 = cfrom; c0 < cto; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tl + col + c0, v);
        tmem_wait_ld(v);
        if (lane < 16 && m < nrows) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = c0 + j;
                const float x = __uint_as_float(v[j]);
                if (c < ncols) atomicAdd(grad + wofs + m * ncols + c, x);
                else if (c == bcol) atomicAdd(grad + bofs + m, x);
            }
        }
    }
}

__global__ void __launch_bounds__(kTrThreads, 1) mlp_train_tc5_kernel(const __nv_bfloat16* __restrict__ wpacked,
                                                                     const float* __restrict__ bpacked,
                                                                     const __nv_bfloat16* __restrict__ feat,
                                                                     const float* __restrict__ dirs,
                                                                     const float* __restrict__ tgt, int n, float scale,
                                                                     float* __restrict__ grad,
                                                                     float* __restrict__ loss_out)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ float sB[kPackedBias];
    __shared__ float xch[3][2][kRows];
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    __shared__ float sloss;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row = 32 * quarter + lane;           // this thread's row (= TMEM lane)
    const int c1 = 32 * half;                      // its 32 columns of a 64-column block
    stage_weights(sm, wpacked, tid, kTrThreads);
    for (int i = tid; i < kPackedBias; i += kTrThreads) sB[i] = bpacked[i];
    // constant columns: a one after each hidden layer's 64 outputs (bias
    // gradients); zeros in the output-gradient columns 40..63
    if (half == 0) {
        const uint32_t one = 0x3F80u;                              // BF16 1.0
        st16(sm + kTrOffH1, core_off(row, 64, kCH), one, 0u, 0u, 0u);
        st16(sm + kTrOffH2, core_off(row, 64, kCH), one, 0u, 0u, 0u);
        st16(sm + kTrOffH3, core_off(row, 64, kCH), one, 0u, 0u, 0u);
    } else {
        st16(sm + kTrOffDO, core_off(row, 40, kCD), 0u, 0u, 0u, 0u);
        st16(sm + kTrOffDO, core_off(row, 48, kCD), 0u, 0u, 0u, 0u);
        st16(sm + kTrOffDO, core_off(row, 56, kCD), 0u, 0u, 0u, 0u);
    }
    if (tid == 0) { sloss = 0.0f; mbar_init(&bar, 1); fence_mbar_init(); }
    if (warp == 0) { tmem_alloc(&tbase, kTrCols); tmem_relinquish(); }
    to_mma();
    const uint32_t T = tbase;
    const uint32_t tl = T + ((uint32_t)(32 * quarter) << 16);    // this warp's lane quarter
    const uint32_t aW1 = smem_addr(sm + kOffSW1), aW2 = smem_addr(sm + kOffSW2), aW3 = smem_addr(sm + kOffSW3);
    const uint32_t aW4 = smem_addr(sm + kOffSW4), aX = smem_addr(sm + kOffSX);
    const uint32_t aH1 = smem_addr(sm + kTrOffH1), aH2 = smem_addr(sm + kTrOffH2), aH3 = smem_addr(sm + kTrOffH3);
    const uint32_t aDO = smem_addr(sm + kTrOffDO), aDZ = smem_addr(sm + kTrOffDZ);
    constexpr uint32_t id64 = idesc_bf16(128, 64, false, false), id48 = idesc_bf16(128, 48, false, false);
    constexpr uint32_t idBack = idesc_bf16(128, 64, false, true);    // dZ (K-major) x W (read along its rows)
    constexpr uint32_t idG = idesc_bf16(64, 72, true, true);         // dZ^T x [A 1], both read along rows
    constexpr uint32_t idG1 = idesc_bf16(64, 16, true, true);
    uint32_t phase = 0;
    bool ok = true;
    uint32_t acc_g = 0u;              // 0 on a CTA's first tile: the gradient blocks start from zero
    float lsum = 0.0f;
    const int tiles = (n + kRows - 1) / kRows;
    // the row's record of a tile: its half of the features (the one of
    // feature 9 set: bias of layer 1), the sampled direction, the target
    auto load_record = [&](int tl_, uint4& fq, float (&w)[3], float& t) {
        const int r = tl_ * kRows + row;
        fq = make_uint4(0u, 0u, 0u, 0u);
        w[0] = 0.0f; w[1] = 0.0f; w[2] = 1.0f;
        t = 0.0f;
        if (tl_ < tiles && r < n) {
            fq = __ldg(reinterpret_cast<const uint4*>(feat + (size_t)r * 16) + half);
            if (half) fq.x = (fq.x & 0xFFFFu) | (0x3F80u << 16);
            w[0] = __ldg(dirs + 3 * (size_t)r);
            w[1] = __ldg(dirs + 3 * (size_t)r + 1);
            w[2] = __ldg(dirs + 3 * (size_t)r + 2);
            t = __ldg(tgt + r) * scale;
        }
    };
    uint4 nfq;
    float nw[3], nt;
    load_record(blockIdx.x, nfq, nw, nt);
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint4 fq = nfq;
        const float w[3] = {nw[0], nw[1], nw[2]}, t = nt;
        load_record(tile + gridDim.x, nfq, nw, nt);     // the next tile's, in flight during this one
        *reinterpret_cast<uint4*>(sm + kOffSX + core_off(row, 8 * half, kCX)) = fq;
        // ---- forward
        to_mma();
        if (tid == 0) {
            mma_bf16(T + cACC, sdesc_kmajor(aX, kCX), sdesc_kmajor(aW1, 16), id64, 0u);
            mma_commit(&bar);
        }
        if (!(ok = from_mma(&bar, phase))) break;
        train_hidden(tl, cGP1, c1, sB, sm + kTrOffH1, row);
        for (int L = 0; L < 2 && ok; ++L) {
            const uint32_t aIn = L == 0 ? aH1 : aH2, aWl = L == 0 ? aW2 : aW3;
            to_mma();
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    mma_bf16(T + cACC, sdesc_kmajor(aIn + 256u * k, kCH), sdesc_kmajor(aWl + 256u * k, 64), id64,
                             k ? 1u : 0u);
                mma_commit(&bar);
            }
            if (!(ok = from_mma(&bar, phase))) break;
            train_hidden(tl, L == 0 ? cGP2 : cGP3, c1, sB + 64 * (L + 1), sm + (L == 0 ? kTrOffH2 : kTrOffH3), row);
        }
        if (!ok) break;
        to_mma();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_bf16(T + cACC, sdesc_kmajor(aH3 + 256u * k, kCH), sdesc_kmajor(aW4 + 256u * k, 64), id48,
                         k ? 1u : 0u);
            mma_commit(&bar);
        }
        if (!(ok = from_mma(&bar, phase))) break;
        // ---- d(-t log q_vMF)/d outputs, FP32, half the lobes of a row per thread
        lsum += train_loss_half(tl, sB, xch, row, half, w, t, sm + kTrOffDO);
        // ---- backward, layer 4: dW4 += dO^T [H3 1]; dA3 = dO W4 (K = 48)
        to_mma();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma_bf16(T + cG4, sdesc_mnmajor(aDO + 2u * kCD * 16u * k, kCD), sdesc_mnmajor(aH3 + 2u * kCH * 16u * k, kCH),
                         idG, (acc_g | k) ? 1u : 0u);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                mma_bf16(T + cACC, sdesc_kmajor(aDO + 256u * k, kCD), sdesc_mnmajor(aW4 + 2u * 64u * 16u * k, 64), idBack,
                         k ? 1u : 0u);
            mma_commit(&bar);
        }
        if (!(ok = from_mma(&bar, phase))) break;
        train_dz(tl, cGP3, c1, sm + kTrOffDZ, row);
        // ---- layers 3 and 2: dW_l += dZ^T [A_{l-1} 1]; dA_{l-1} = dZ W_l
        for (int L = 0; L < 2 && ok; ++L) {
            const uint32_t aIn = L == 0 ? aH2 : aH1, aWl = L == 0 ? aW3 : aW2, cG = L == 0 ? cG3 : cG2;
            to_mma();
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    mma_bf16(T + cG, sdesc_mnmajor(aDZ + 2u * kCD * 16u * k, kCD),
                             sdesc_mnmajor(aIn + 2u * kCH * 16u * k, kCH), idG, (acc_g | k) ? 1u : 0u);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    mma_bf16(T + cACC, sdesc_kmajor(aDZ + 256u * k, kCD), sdesc_mnmajor(aWl + 2u * 64u * 16u * k, 64),
                             idBack, k ? 1u : 0u);
                mma_commit(&bar);
            }
            if (!(ok = from_mma(&bar, phase))) break;
            train_dz(tl, L == 0 ? cGP2 : cGP1, c1, sm + kTrOffDZ, row);
        }
        if (!ok) break;
        // ---- layer 1: dW1 += dZ1^T [X 1] (features 0..8, the one at 9)
        to_mma();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma_bf16(T + cG1, sdesc_mnmajor(aDZ + 2u * kCD * 16u * k, kCD), sdesc_mnmajor(aX + 2u * kCX * 16u * k, kCX),
                         idG1, (acc_g | k) ? 1u : 0u);
            mma_commit(&bar);
        }
        if (!(ok = from_mma(&bar, phase))) break;   // the next tile overwrites X, H, dO and dZ
        acc_g = 1u;
    }
    // ---- loss and gradient blocks to global memory (the two threads of a
    // lane split the column chunks of each block)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) atomicAdd(&sloss, lsum);
    if (ok && acc_g) {
        if (half == 0) flush_block(tl, cG1, 0, 16, kIn, 9, 64, kOffW1, kOffB1, grad, quarter, lane);
        flush_block(tl, cG2, half ? 48 : 0, half ? 80 : 48, kH, 64, 64, kOffW2, kOffB2, grad, quarter, lane);
        flush_block(tl, cG3, half ? 48 : 0, half ? 80 : 48, kH, 64, 64, kOffW3, kOffB3, grad, quarter, lane);
        flush_block(tl, cG4, half ? 48 : 0, half ? 80 : 48, kH, 64, kOut, kOffW4, kOffB4, grad, quarter, lane);
    }
    if (!ok && tid == 0) atomicExch(&g_tc5_error, 1);
    fence_before_sync();
    __syncthreads();
    if (tid == 0 && loss_out) atomicAdd(loss_out, sloss);
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(T, kTrCols);
    }
}

}  // namespace

cudaError_t launch_mlp_infer(const void* wpacked, const float* bpacked, const void* feat, int n, float* mix,
                             float* raw, int sm_count, cudaStream_t st, bool tracer_layout)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_infer_tc5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kInfSmem);
    if (e != cudaSuccess) return e;
    const int tiles = (n + kRows - 1) / kRows;
    const int grid = tiles < 3 * sm_count ? tiles : 3 * sm_count;
    mlp_infer_tc5_kernel<<<grid, 128, kInfSmem, st>>>(static_cast<const __nv_bfloat16*>(wpacked), bpacked,
                                                      static_cast<const __nv_bfloat16*>(feat), n, mix, raw,
                                                      tracer_layout ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_tc(const void* wpacked, const float* bpacked, const float* /*params: the BF16 copy is used*/,
                                const void* feat, const float* dirs, const float* tgt, int n, float scale, float* grad,
                                float* loss, int sm_count, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_train_tc5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTrainSmem);
    if (e != cudaSuccess) return e;
    const int tiles = (n + kRows - 1) / kRows;
    const int grid = tiles < sm_count ? tiles : sm_count;
    mlp_train_tc5_kernel<<<grid, kTrThreads, kTrainSmem, st>>>(static_cast<const __nv_bfloat16*>(wpacked), bpacked,
                                                         static_cast<const __nv_bfloat16*>(feat), dirs, tgt, n, scale,
                                                         grad, loss);
    return cudaGetLastError();
}

// The error word of the tensor-core kernels: 1 if an MMA wait ran out since
// the last call (then cleared).  Synchronises the stream.
cudaError_t tc5_take_error(int* err, cudaStream_t st)
{
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_tc5_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v) {
        const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_tc5_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    *err = v;
    return e;
}

}  // namespace mcrt
