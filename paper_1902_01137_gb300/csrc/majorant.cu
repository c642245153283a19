// majorant.cu -- field ingest and the majorant pyramid (sm_103a).
//
// K2+K1 fused (relayout_l1): the row-major extinction field is rewritten into
// 8x8x8 bricks (Sec. 3.1.2: voxels kept in fixed-size spatially coherent
// blocks) and, in the same pass, the max of every brick -- the level-1 cell of
// the pyramid -- is reduced.  One pass over HBM: 4 B read + 4 B (or 2 B) written
// per voxel plus 4 B per 512 voxels.
// K1 (reduce_level): level L >= 2 cells take the exact max of their (up to)
// 8x8x8 children (Sec. 3.1.1: merged voxels store the max).  Max is exact and
// order-free, so the result is bit-identical to any other evaluation order.
// Octree (oct_level1, oct_reduce2): the paper's own grid, Sec. 3.1.1 --
// groups of 2^3 cells merged recursively, each cell keeping the max and the
// min of the voxels it covers.  Level 1 reads the stored voxels (bricks);
// level L >= 2 reduces 2^3 cells of level L - 1.
// Leaf map (either grid): for each level-1 cell, the coarsest ancestor whose
// majorant times its height is <= tau~ (Sec. 4.2's merge criterion), with
// its majorant, its minorant (the min levels, built alongside the max) and
// its size as a voxel shift.
#include <cuda_bf16.h>

#include "mcrt_internal.h"

namespace mcrt {

namespace {

// One block of 256 threads = 4 consecutive bricks along x.  Thread t holds
// row r = t >> 2 (y & 7 = r & 7, z & 7 = r >> 3) of brick q = t & 3.
template <bool BF16>
__global__ void __launch_bounds__(256) relayout_l1_kernel(const float* __restrict__ src, int nx, int ny, int nz,
                                                          int nbx, int nby, void* __restrict__ dst,
                                                          float* __restrict__ l1, float* __restrict__ l1min)
{
    const int t = threadIdx.x;
    const int q = t & 3;
    const int r = t >> 2;
    const int bx = blockIdx.x * 4 + q;
    const int by = blockIdx.y;
    const int bz = blockIdx.z;
    const int y = by * 8 + (r & 7);
    const int z = bz * 8 + (r >> 3);
    const int x0 = bx * 8;
    float v[8];
    const bool row_ok = (bx < nbx) && (y < ny) && (z < nz);
    const size_t row = ((size_t)z * ny + y) * (size_t)nx;
    if (row_ok && x0 + 8 <= nx && (nx & 3) == 0 &&
        ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(src + row + x0));
        const float4 b = __ldcs(reinterpret_cast<const float4*>(src + row + x0 + 4));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (row_ok && x0 + i < nx) ? src[row + x0 + i] : 0.0f;
    }
    float m = 0.0f;
    float mn = __int_as_float(0x7f800000);   // min over the existing voxels (as stored)
    if (BF16) {
        // stored voxels: nearest bf16; majorant: smallest bf16 >= the FP32 max,
        // which bounds every nearest-rounded voxel of the brick
        uint32_t packed[4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[i]));
            const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[i + 1]));
            packed[i / 2] = lo | (hi << 16);
            m = fmaxf(m, fmaxf(v[i], v[i + 1]));
            if (row_ok && x0 + i < nx) mn = fminf(mn, __uint_as_float(lo << 16));
            if (row_ok && x0 + i + 1 < nx) mn = fminf(mn, __uint_as_float(hi << 16));
        }
        m = __bfloat162float(__float2bfloat16_ru(m));
        if (bx < nbx) {
            const size_t brick = ((size_t)bz * nby + by) * (size_t)nbx + bx;
            uint4* o = reinterpret_cast<uint4*>(static_cast<uint16_t*>(dst) + brick * 512 + r * 8);
            __stcs(o, make_uint4(packed[0], packed[1], packed[2], packed[3]));
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            m = fmaxf(m, v[i]);
            if (row_ok && x0 + i < nx) mn = fminf(mn, v[i]);
        }
        if (bx < nbx) {
            const size_t brick = ((size_t)bz * nby + by) * (size_t)nbx + bx;
            float4* o = reinterpret_cast<float4*>(static_cast<float*>(dst) + brick * 512 + r * 8);
            __stcs(o, make_float4(v[0], v[1], v[2], v[3]));
            __stcs(o + 1, make_float4(v[4], v[5], v[6], v[7]));
        }
    }
    // max over the 64 rows of each brick: lanes sharing q differ in bits 2..4
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 4));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 8));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 16));
    __shared__ float part[8][4], partmin[8][4];
    if ((t & 31) < 4) { part[t >> 5][q] = m; partmin[t >> 5][q] = mn; }
    __syncthreads();
    if (t < 4) {
        float mm = part[0][t], mmn = partmin[0][t];
#pragma unroll
        for (int w = 1; w < 8; ++w) { mm = fmaxf(mm, part[w][t]); mmn = fminf(mmn, partmin[w][t]); }
        const int bxx = blockIdx.x * 4 + t;
        if (bxx < nbx) {
            l1[((size_t)bz * nby + by) * (size_t)nbx + bxx] = mm;
            l1min[((size_t)bz * nby + by) * (size_t)nbx + bxx] = mmn;
        }
    }
}

// One warp per coarse cell; lane l takes children l, l + 32, ... of 512.
// MIN: the minorant level (min over the existing children) instead.
template <bool MIN>
__global__ void __launch_bounds__(256) reduce_level_kernel(const float* __restrict__ prev, int px, int py, int pz,
                                                           float* __restrict__ out, int cx, int cy, int cz)
{
    const long long cell = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (cell >= (long long)cx * cy * cz) return;
    const int ix = (int)(cell % cx);
    const int iy = (int)((cell / cx) % cy);
    const int iz = (int)(cell / ((long long)cx * cy));
    float m = MIN ? __int_as_float(0x7f800000) : 0.0f;
#pragma unroll 4
    for (int c = lane; c < 512; c += 32) {
        const int x = ix * 8 + (c & 7), y = iy * 8 + ((c >> 3) & 7), z = iz * 8 + (c >> 6);
        if (x < px && y < py && z < pz) {
            const float v = prev[((size_t)z * py + y) * (size_t)px + x];
            m = MIN ? fminf(m, v) : fmaxf(m, v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, m, o);
        m = MIN ? fminf(m, w) : fmaxf(m, w);
    }
    if (lane == 0) out[cell] = m;
}

struct LevelTable {
    const float* p[kMaxGridLevels + 1];
    const float* pmin[kMaxGridLevels + 1];
    int dims[kMaxGridLevels + 1][3];
    float hz[kMaxGridLevels + 1];
};

// Leaf of each level-1 cell: search from the top level down to finest + 1.
// lb: log2 of the branching per axis (3 pyramid, 1 octree); a level-L cell
// spans 2^(lb L) voxels per axis, which is the shift the entry records.
__global__ void __launch_bounds__(256) leafmap_kernel(LevelTable T, int levels, int finest, float tau, int lb,
                                                      int n1x, int n1y, int n1z, uint2* __restrict__ leaf)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n1x * n1y * n1z) return;
    const int cx = (int)(i % n1x), cy = (int)((i / n1x) % n1y), cz = (int)(i / ((long long)n1x * n1y));
    for (int L = levels; L > finest; --L) {
        const int s = lb * (L - 1);
        const int ax = cx >> s, ay = cy >> s, az = cz >> s;
        const size_t c = ((size_t)az * T.dims[L][1] + ay) * T.dims[L][0] + ax;
        const float M = T.p[L][c];
        if (__fmul_rn(M, T.hz[L]) <= tau) {
            // .y: the minorant rounded down to bfloat16 (high half) | the shift
            leaf[i] = make_uint2(__float_as_uint(M),
                                 (__float_as_uint(T.pmin[L][c]) & 0xFFFF0000u) | (unsigned)(lb * L));
            return;
        }
    }
    if (finest == 0) {
        leaf[i] = make_uint2(0u, 0u);
    } else {
        const int s = lb * (finest - 1);
        const size_t c = ((size_t)(cz >> s) * T.dims[finest][1] + (cy >> s)) * T.dims[finest][0] + (cx >> s);
        const float M = T.p[finest][c];
        leaf[i] = make_uint2(__float_as_uint(M),
                             (__float_as_uint(T.pmin[finest][c]) & 0xFFFF0000u) | (unsigned)(lb * finest));
    }
}

// Octree level 1: max and min of each 2^3 voxel group, read from the bricks
// (the stored values: FP32, or the nearest-bfloat16 voxels of a BF16 field,
// whose max bounds exactly what the tracer reads).
template <bool BF16>
__global__ void __launch_bounds__(256) oct_level1_kernel(DevScene S, int dx, int dy, int dz, float* __restrict__ omax,
                                                         float* __restrict__ omin)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)dx * dy * dz) return;
    const int cx = (int)(i % dx), cy = (int)((i / dx) % dy), cz = (int)(i / ((long long)dx * dy));
    float m = 0.0f, mn = __int_as_float(0x7f800000);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int x = 2 * cx + (c & 1), y = 2 * cy + ((c >> 1) & 1), z = 2 * cz + (c >> 2);
        if (x < S.n[0] && y < S.n[1] && z < S.n[2]) {
            const float v = kfetch<BF16>(S, x, y, z);
            m = fmaxf(m, v);
            mn = fminf(mn, v);
        }
    }
    omax[i] = m;
    omin[i] = mn;
}

// Octree level L >= 2: max and min over the (up to) 2^3 children.
__global__ void __launch_bounds__(256) oct_reduce2_kernel(const float* __restrict__ pmax, const float* __restrict__ pmin,
                                                          int px, int py, int pz, float* __restrict__ omax,
                                                          float* __restrict__ omin, int dx, int dy, int dz)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)dx * dy * dz) return;
    const int cx = (int)(i % dx), cy = (int)((i / dx) % dy), cz = (int)(i / ((long long)dx * dy));
    float m = 0.0f, mn = __int_as_float(0x7f800000);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int x = 2 * cx + (c & 1), y = 2 * cy + ((c >> 1) & 1), z = 2 * cz + (c >> 2);
        if (x < px && y < py && z < pz) {
            const size_t j = ((size_t)z * py + y) * (size_t)px + x;
            m = fmaxf(m, pmax[j]);
            mn = fminf(mn, pmin[j]);
        }
    }
    omax[i] = m;
    omin[i] = mn;
}

}  // namespace

cudaError_t launch_relayout(const float* src, const mcrt_scene* sc, cudaStream_t st)
{
    dim3 grid((sc->nb[0] + 3) / 4, sc->nb[1], sc->nb[2]);
    float* l1 = sc->d_pyr + sc->lev_off[1];
    float* l1min = sc->d_pyr + sc->pyr_capacity + sc->lev_off[1];
    if (sc->storage == MCRT_STORAGE_BF16)
        relayout_l1_kernel<true><<<grid, 256, 0, st>>>(src, sc->n[0], sc->n[1], sc->n[2], sc->nb[0], sc->nb[1],
                                                       sc->d_vox, l1, l1min);
    else
        relayout_l1_kernel<false><<<grid, 256, 0, st>>>(src, sc->n[0], sc->n[1], sc->n[2], sc->nb[0], sc->nb[1],
                                                        sc->d_vox, l1, l1min);
    return cudaGetLastError();
}

cudaError_t launch_reduce_level(const float* prev, const int* pd, float* out, const int* d, bool min_level,
                                cudaStream_t st)
{
    const long long cells = (long long)d[0] * d[1] * d[2];
    const int warps = 8;
    const long long blocks = (cells + warps - 1) / warps;
    if (min_level)
        reduce_level_kernel<true><<<(unsigned)blocks, 32 * warps, 0, st>>>(prev, pd[0], pd[1], pd[2], out, d[0], d[1],
                                                                            d[2]);
    else
        reduce_level_kernel<false><<<(unsigned)blocks, 32 * warps, 0, st>>>(prev, pd[0], pd[1], pd[2], out, d[0], d[1],
                                                                             d[2]);
    return cudaGetLastError();
}

cudaError_t launch_leafmap(const mcrt_scene* sc, float tau, int finest, int grid, cudaStream_t st)
{
    LevelTable T{};
    const bool oct = grid == MCRT_GRID_OCTREE;
    const int levels = oct ? sc->oct_levels : sc->levels;
    const int lb = oct ? 1 : 3;
    if (levels < 1 || levels > kMaxGridLevels) return cudaErrorInvalidValue;
    for (int L = 1; L <= levels; ++L) {
        if (oct) {
            T.p[L] = sc->d_oct + sc->oct_off[L];
            T.pmin[L] = sc->d_oct + sc->oct_capacity + sc->oct_off[L];
            for (int a = 0; a < 3; ++a) T.dims[L][a] = sc->oct_dims[3 * L + a];
        } else {
            T.p[L] = sc->d_pyr + sc->lev_off[L];
            T.pmin[L] = sc->d_pyr + sc->pyr_capacity + sc->lev_off[L];
            for (int a = 0; a < 3; ++a) T.dims[L][a] = sc->lev_dims[3 * L + a];
        }
        T.hz[L] = sc->h[2] * (float)(1 << (lb * L));
    }
    const int* n1 = oct ? &sc->oct_dims[3] : sc->nb;
    const long long cells = (long long)n1[0] * n1[1] * n1[2];
    leafmap_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(T, levels, finest, tau, lb, n1[0], n1[1], n1[2],
                                                                      oct ? sc->d_oleaf : sc->d_leaf);
    return cudaGetLastError();
}

cudaError_t launch_octree(const mcrt_scene* sc, const DevScene& S, cudaStream_t st)
{
    const int* d1 = &sc->oct_dims[3];
    const long long n1 = (long long)d1[0] * d1[1] * d1[2];
    float* mx = sc->d_oct;
    float* mn = sc->d_oct + sc->oct_capacity;
    if (sc->storage == MCRT_STORAGE_BF16)
        oct_level1_kernel<true><<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(S, d1[0], d1[1], d1[2], mx + sc->oct_off[1],
                                                                              mn + sc->oct_off[1]);
    else
        oct_level1_kernel<false><<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(S, d1[0], d1[1], d1[2],
                                                                               mx + sc->oct_off[1], mn + sc->oct_off[1]);
    for (int L = 2; L <= sc->oct_levels; ++L) {
        const int* pd = &sc->oct_dims[3 * (L - 1)];
        const int* d = &sc->oct_dims[3 * L];
        const long long n = (long long)d[0] * d[1] * d[2];
        oct_reduce2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            mx + sc->oct_off[L - 1], mn + sc->oct_off[L - 1], pd[0], pd[1], pd[2], mx + sc->oct_off[L],
            mn + sc->oct_off[L], d[0], d[1], d[2]);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Heightfield ground: max pyramid.  Level 0 holds each cell's maximum over
// its 4 corner heights (periodic); level L the maximum over 4 x 4 cells of
// level L - 1.  Also a scan for invalid heights (not finite, < 0 or above
// the top of the field).
// ---------------------------------------------------------------------------
namespace {

__global__ void hf_cellmax_kernel(const float* __restrict__ h, int nx, int ny, float* __restrict__ out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nx * ny) return;
    const int i = (int)(idx % nx), j = (int)(idx / nx);
    const int i1 = i + 1 == nx ? 0 : i + 1, j1 = j + 1 == ny ? 0 : j + 1;
    out[idx] = fmaxf(fmaxf(h[(size_t)j * nx + i], h[(size_t)j * nx + i1]),
                     fmaxf(h[(size_t)j1 * nx + i], h[(size_t)j1 * nx + i1]));
}

__global__ void hf_reduce4_kernel(const float* __restrict__ in, int nx, int ny, float* __restrict__ out)
{
    // out is (nx / 4) x (ny / 4)
    const int ox = nx >> 2, oy = ny >> 2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)ox * oy) return;
    const int i = (int)(idx % ox), j = (int)(idx / ox);
    float m = in[(size_t)(4 * j) * nx + 4 * i];
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) m = fmaxf(m, in[(size_t)(4 * j + b) * nx + 4 * i + a]);
    out[idx] = m;
}

__global__ void hf_check_kernel(const float* __restrict__ h, long long n, float top, int* __restrict__ bad)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const float v = h[idx];
    if (!(v >= 0.0f && v <= top)) atomicOr(bad, 1);
}

}  // namespace

cudaError_t launch_hf_pyramid(const float* h, int nx, int ny, float* pyr, const int* off, int levels, cudaStream_t st)
{
    const long long n0 = (long long)nx * ny;
    hf_cellmax_kernel<<<(unsigned)((n0 + 255) / 256), 256, 0, st>>>(h, nx, ny, pyr + off[0]);
    for (int L = 1; L < levels; ++L) {
        const int px = nx >> (2 * (L - 1)), py = ny >> (2 * (L - 1));
        const long long n = (long long)(px >> 2) * (py >> 2);
        hf_reduce4_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pyr + off[L - 1], px, py, pyr + off[L]);
    }
    return cudaGetLastError();
}

cudaError_t launch_hf_check(const float* h, long long n, float top, int* bad, cudaStream_t st)
{
    hf_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(h, n, top, bad);
    return cudaGetLastError();
}

}  // namespace mcrt
