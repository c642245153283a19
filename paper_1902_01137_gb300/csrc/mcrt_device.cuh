// mcrt_device.cuh -- device-side building blocks of the tracer (sm_103a).
//
//  * Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
//    per-(path, event, stream) draw sequence.
//  * The FP32 leaf traversal over a max grid -- the 8^L pyramid or the
//    paper's 2^L octree (Sec. 3.1.1): the ray steps from leaf to leaf, a leaf
//    being the coarsest grid cell whose majorant times its height is <= tau~
//    (Sec. 4.2), or a cell of the finest tracked level.  A leaf is an aligned
//    block of 2^s voxels per axis; the traversal only sees s.
//    Every operation is an explicitly rounded IEEE binary32 operation, so the
//    leaf sequence and distances are reproducible bit for bit.
//  * Henyey-Greenstein sampling/evaluation and direction frames (Sec. 4.1).
//
// No file here is shared with the CPU oracle; the oracle implements the same
// definitions independently.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcrt {

// Bounds-checked build (-DMCRT_CHECKED; the default build compiles every
// check away): MCRT_CHECK(cond, code) counts a violated index condition in
// a device word of this translation unit and keeps the first code; the
// caller then clamps the index, so nothing faults.  Codes: 1 voxel, 2
// leaf-map entry, 3 tally entry, 4 heightfield corner, 5 heightfield
// pyramid cell.
#ifdef MCRT_CHECKED
static __device__ unsigned int g_mcrt_bounds[2];   // violations, first code
__device__ __forceinline__ void mcrt_bounds_fail(unsigned code)
{
    atomicAdd(&g_mcrt_bounds[0], 1u);
    atomicCAS(&g_mcrt_bounds[1], 0u, code);
}
#define MCRT_CHECK(cond, code) do { if (!(cond)) mcrt_bounds_fail(code); } while (0)
#else
#define MCRT_CHECK(cond, code) do { } while (0)
#endif

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInv4Pi = 0.0795774715459476679f;

// --------------------------------------------------------------------------
// Philox4x32-10
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Random numbers are addressed: stream s of event e of path p evaluates
// Philox at counter (p lo, p hi, (e << 2) | s, block) and uses fixed words of
// the block -- block 0 word 0: first optical depth of a flight or a flux
// path's direct sun ray; block j >= 1: the j-th tentative collision (test or
// roulette draw, next optical depth); stream 1 block 0: the vertex ending the
// flight of event e (two direction draws, roulette) and, word 3, the first
// optical depth of its sun ray; stream 2 block 0: path start (and, word 2, a
// camera path's first optical depth); blocks kBlockVertex and kBlockVertex - 1
// of stream 0: a learned vertex (and a Rayleigh vertex's species).  Streams:
// 0 flight, 1 vertex and its sun ray, 2 path start, 3 direct sun ray of a
// flux path.
constexpr uint32_t kBlockVertex = 0xFFFFFFFFu;

__device__ __forceinline__ float u01(uint32_t w)
{
    return (float)((w >> 8) + 1u) * 5.9604644775390625e-8f;   // ((w >> 8) + 1) 2^-24
}

__device__ __forceinline__ uint4 draw_block(unsigned long long path, uint32_t c2, uint32_t block, uint2 key)
{
    return philox4x32_10(make_uint4((uint32_t)path, (uint32_t)(path >> 32), c2, block), key);
}

// --------------------------------------------------------------------------
// Scene as seen by the kernels
// --------------------------------------------------------------------------
constexpr int kMaxHfLevels = 12;
constexpr int kMaxGridLevels = 20;   // octree levels for fields up to 2^20 voxels per axis

struct DevScene {
    int n[3];            // voxels per axis
    float h[3];          // voxel size [km]
    float inv_h[3];      // 1 / h, round to nearest
    float Lper[2];       // n * h for the periodic axes
    int nb[3];           // bricks (8^3 voxels) per axis == level-1 cells
    const float* __restrict__ vox;       // brick-major FP32 field, or null
    const uint16_t* __restrict__ vox16;  // brick-major BF16 field, or null
    const uint2* __restrict__ leaf;      // per level-1 cell: {majorant bits, minorant | leaf shift}
    int lb;              // log2 of the grid's branching per axis: 3 (8^L pyramid) or 1 (2^L octree)
    int nl[3];           // level-1 cells per axis of the tracked grid (leaf-map dims)
    float k_clear, ssa_clear, ssa_cloud, g;
    float k_gas;         // extra uniform pure absorber
    float albedo;        // Lambertian ground
    float sun[3];        // unit vector toward the sun
    int rayleigh;        // clear air scatters with the Rayleigh phase function (else HG with g)
    // heightfield ground (hf null: flat ground at z = 0).  Heights sit at
    // the corners of a periodic grid of hn[0] x hn[1] cells; hpyr holds the
    // cell maxima (level 0: max of a cell's 4 corners) and hlev - 1 coarser
    // levels of 4 x 4 blocks, concatenated at hoff[level].
    const float* __restrict__ hf;
    const float* __restrict__ hpyr;
    int hn[2];
    float hc[2];         // cell size [km]
    float inv_hc[2];
    float hmax;          // largest height
    int hmask[2];        // hn - 1 when hn is a power of two (index wrap by mask), else -1
    int hlev;
    int hoff[kMaxHfLevels];
};

__device__ __forceinline__ size_t brick_index(const DevScene& S, int i, int j, int k)
{
    const size_t b = ((size_t)(k >> 3) * (size_t)S.nb[1] + (size_t)(j >> 3)) * (size_t)S.nb[0] + (size_t)(i >> 3);
    const uint32_t off = ((((uint32_t)k & 7u) << 3 | ((uint32_t)j & 7u)) << 3) | ((uint32_t)i & 7u);
    return b * 512u + off;
}

template <bool BF16>
__device__ __forceinline__ float kfetch(const DevScene& S, int i, int j, int k)
{
#ifdef MCRT_CHECKED
    MCRT_CHECK(i >= 0 && i < S.n[0] && j >= 0 && j < S.n[1] && k >= 0 && k < S.n[2], 1);
    i = min(max(i, 0), S.n[0] - 1);
    j = min(max(j, 0), S.n[1] - 1);
    k = min(max(k, 0), S.n[2] - 1);
#endif
    const size_t idx = brick_index(S, i, j, k);
    if (BF16) return __uint_as_float((uint32_t)__ldg(S.vox16 + idx) << 16);
    return __ldg(S.vox + idx);
}

// --------------------------------------------------------------------------
// Leaf traversal
// --------------------------------------------------------------------------
struct Ray {
    float o[3];      // segment origin
    float d[3];      // unit direction
    float inv_d[3];  // 1 / d (0 where d == 0)
    int v[3];        // voxel of the current point
    int lev;         // leaf size as a shift: the leaf spans 2^lev voxels per axis
    float M;         // leaf majorant (+ k_gas)
    float mn;        // leaf minorant (+ k_gas)
    float t;         // distance of the current point from o
    float texit;     // distance of the leaf exit from o
    int ax;          // exit axis
    uint32_t steps;  // leaves entered (guard)
};

// Voxel range [lo, hi] of the current leaf on axis a.
__device__ __forceinline__ int leaf_lo(const Ray& R, int a) { return (R.v[a] >> R.lev) << R.lev; }
__device__ __forceinline__ int leaf_hi(const DevScene& S, const Ray& R, int a)
{
    return min(leaf_lo(R, a) + (1 << R.lev), S.n[a]) - 1;
}

// Voxel of coordinate p on one axis: floor(p / h) by the rounded reciprocal,
// one lower when moving down onto an exact face, clamped to [lo, hi].
__device__ __forceinline__ int locate(float p, float d, float h, float inv_h, int lo, int hi)
{
    int i = __float2int_rd(__fmul_rn(p, inv_h));
    if (d < 0.0f && __fmul_rn(__int2float_rn(i), h) == p) i -= 1;
    return min(max(i, lo), hi);
}

// Leaf-map entry of the level-1 cell (of the tracked grid) holding voxel v.
__device__ __forceinline__ const uint2* leaf_entry(const DevScene& S, const int v[3])
{
    const int b = S.lb;
#ifdef MCRT_CHECKED
    int w[3];
    for (int a = 0; a < 3; ++a) {
        MCRT_CHECK(v[a] >= 0 && v[a] < S.n[a] && (v[a] >> b) < S.nl[a], 2);
        w[a] = min(max(v[a], 0), S.n[a] - 1);
    }
    return S.leaf + ((size_t)(w[2] >> b) * S.nl[1] + (w[1] >> b)) * S.nl[0] + (w[0] >> b);
#else
    return S.leaf + ((size_t)(v[2] >> b) * S.nl[1] + (v[1] >> b)) * S.nl[0] + (v[0] >> b);
#endif
}

// Finish entering the leaf holding R.v from its leaf-map entry: size,
// majorant and the exit distance / axis.
template <bool BF16>
__device__ __forceinline__ void finish_leaf(const DevScene& S, Ray& R, uint2 e)
{
    // entry: .x majorant bits, .y = minorant rounded down to bfloat16 | shift
    R.lev = (int)(e.y & 0xFFFFu);
    float M = __uint_as_float(e.x), mn = __uint_as_float(e.y & 0xFFFF0000u);
    if (R.lev == 0) M = mn = kfetch<BF16>(S, R.v[0], R.v[1], R.v[2]);
    R.M = __fadd_rn(M, S.k_gas);
    R.mn = __fadd_rn(mn, S.k_gas);
    const int s = R.lev;
    float ta[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lo = (R.v[a] >> s) << s;
        const int hi = min(lo + (1 << s), S.n[a]) - 1;
        const float d = R.d[a];
        if (d == 0.0f) {
            ta[a] = __int_as_float(0x7f800000);
        } else {
            const int B = d > 0.0f ? hi + 1 : lo;
            ta[a] = __fmul_rn(__fsub_rn(__fmul_rn(__int2float_rn(B), S.h[a]), R.o[a]), R.inv_d[a]);
        }
    }
    int ax = 0;
    float tm = ta[0];
    if (ta[1] < tm) { ax = 1; tm = ta[1]; }
    if (ta[2] < tm) { ax = 2; tm = ta[2]; }
    R.ax = ax;
    R.texit = fmaxf(tm, R.t);
}

// Start a ray at point p (inside the field, x/y in [0, L)) along unit d.
template <bool BF16>
__device__ __forceinline__ void ray_begin(const DevScene& S, Ray& R, const float p[3], const float d[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.o[a] = p[a];
        R.d[a] = d[a];
        R.inv_d[a] = (d[a] != 0.0f) ? __frcp_rn(d[a]) : 0.0f;
        R.v[a] = locate(p[a], d[a], S.h[a], S.inv_h[a], 0, S.n[a] - 1);
    }
    R.t = 0.0f;
    R.steps = 0;
    finish_leaf<BF16>(S, R, __ldg(leaf_entry(S, R.v)));
}

enum StepResult { kInside = 0, kTop = 1, kGround = 2 };

// Point at distance tn along the current segment and its voxel on each axis,
// clamped into the current leaf (so the extinction read there is bounded by
// the leaf majorant).  With `face`, tn is the leaf exit and the exit axis
// index instead steps across the face (hi + 1 or lo - 1).
__device__ __forceinline__ void advance(const DevScene& S, const Ray& R, float tn, bool face, float p[3], int nv[3])
{
    const int s = R.lev;
    int lo[3], hi[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        p[b] = __fmaf_rn(tn, R.d[b], R.o[b]);
        lo[b] = (R.v[b] >> s) << s;
        hi[b] = min(lo[b] + (1 << s), S.n[b]) - 1;
        nv[b] = locate(p[b], R.d[b], S.h[b], S.inv_h[b], lo[b], hi[b]);
    }
    // the exit axis steps across the face (its located value is discarded)
    if (face) {
        if (R.ax == 0) nv[0] = R.d[0] > 0.0f ? hi[0] + 1 : lo[0] - 1;
        else if (R.ax == 1) nv[1] = R.d[1] > 0.0f ? hi[1] + 1 : lo[1] - 1;
        else nv[2] = R.d[2] > 0.0f ? hi[2] + 1 : lo[2] - 1;
    }
}

// Complete a face crossing prepared by advance(face = true): the ground or
// the top, or the periodic wrap of x / y (the segment then restarts on the
// face: o on the face exactly, t = 0, *wrapped_dt = distance of the finished
// segment), then the new voxel.  The caller loads the leaf-map entry of R.v
// and calls finish_leaf when the result is kInside.
__device__ __forceinline__ int cross_face(const DevScene& S, Ray& R, const float p[3], int nv[3], float* wrapped_dt)
{
    const int ax = R.ax;
    const float te = R.texit;
    *wrapped_dt = 0.0f;
    R.t = te;
    if (ax == 2) {
        if (nv[2] < 0) return kGround;
        if (nv[2] >= S.n[2]) return kTop;
    } else {
        int wrapped = 0;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (b != ax) continue;
            if (nv[b] < 0) { nv[b] = S.n[b] - 1; wrapped = 1; }
            else if (nv[b] >= S.n[b]) { nv[b] = 0; wrapped = 2; }
        }
        if (wrapped) {
            *wrapped_dt = te;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                R.o[b] = p[b];
                if (b == ax) R.o[b] = (wrapped == 1) ? (b == 0 ? S.Lper[0] : S.Lper[1]) : 0.0f;
            }
            R.t = 0.0f;
        }
    }
    R.v[0] = nv[0]; R.v[1] = nv[1]; R.v[2] = nv[2];
    ++R.steps;
    return kInside;
}

// Cross the exit face of the current leaf (advance + cross_face); p receives
// the exit point before any wrap shift.
__device__ __forceinline__ int step_face(const DevScene& S, Ray& R, float p[3], float* wrapped_dt)
{
    int nv[3];
    advance(S, R, R.texit, true, p, nv);
    return cross_face(S, R, p, nv, wrapped_dt);
}

// --------------------------------------------------------------------------
// Scattering
// --------------------------------------------------------------------------
// HG phase function normalised over 4 pi sr.
__device__ __forceinline__ float hg_pdf(float g, float mu)
{
    const float den = fmaxf(1.0f + g * g - 2.0f * g * mu, 1e-12f);
    const float r = rsqrtf(den);
    return (1.0f - g * g) * kInv4Pi * r * r * r;
}

// Inverse-CDF HG cosine for xi in (0, 1].
__device__ __forceinline__ float hg_sample_mu(float g, float xi)
{
    if (fabsf(g) < 1e-4f) return 1.0f - 2.0f * xi;
    const float s = __fdividef(1.0f - g * g, 1.0f - g + 2.0f * g * xi);
    const float mu = __fdividef(1.0f + g * g - s * s, 2.0f * g);
    return fminf(fmaxf(mu, -1.0f), 1.0f);
}

// Direction with cosine mu to unit d and azimuth 2 pi xi, in the
// orthonormal frame of Duff et al. (JCGT 2017).
__device__ __forceinline__ void rotate_dir(const float d[3], float mu, float xi, float out[3])
{
    const float sign = copysignf(1.0f, d[2]);
    const float a = -__frcp_rn(sign + d[2]);
    const float b = d[0] * d[1] * a;
    const float b1x = 1.0f + sign * d[0] * d[0] * a, b1y = sign * b, b1z = -sign * d[0];
    const float b2x = b, b2y = sign + d[1] * d[1] * a, b2z = -d[1];
    const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    float sp, cp;
    sincospif(2.0f * xi, &sp, &cp);
    const float c = st * cp, s = st * sp;
    float rx = c * b1x + s * b2x + mu * d[0];
    float ry = c * b1y + s * b2y + mu * d[1];
    float rz = c * b1z + s * b2z + mu * d[2];
    const float inv = rsqrtf(rx * rx + ry * ry + rz * rz);
    out[0] = rx * inv; out[1] = ry * inv; out[2] = rz * inv;
}

// Rayleigh phase function normalised over 4 pi sr: 3 (1 + mu^2) / (16 pi).
__device__ __forceinline__ float rayleigh_pdf(float mu)
{
    return (3.0f / (16.0f * kPi)) * (1.0f + mu * mu);
}

// Inverse-CDF Rayleigh cosine for xi in (0, 1]: the real root of
// mu^3 + 3 mu + 4 - 8 xi = 0 (Cardano), A^(1/3) - A^(-1/3) with
// A = 4 xi - 2 + sqrt((4 xi - 2)^2 + 1).
__device__ __forceinline__ float rayleigh_sample_mu(float xi)
{
    const float b = 4.0f * xi - 2.0f;
    const float c = cbrtf(b + sqrtf(b * b + 1.0f));
    return fminf(fmaxf(c - __frcp_rn(c), -1.0f), 1.0f);
}

// Share of the scattering at total extinction k_tot due to the droplets.
__device__ __forceinline__ float cloud_scatter_share(const DevScene& S, float k_tot)
{
    const float k = k_tot - S.k_gas;
    const float kc = fmaxf(k - S.k_clear, 0.0f);
    const float sc = kc * S.ssa_cloud, sr = (k - kc) * S.ssa_clear;
    return sc + sr > 0.0f ? __fdividef(sc, sc + sr) : 1.0f;
}

// d/dg of ln p_HG(mu) = -2g / (1 - g^2) - 3 (g - mu) / (1 + g^2 - 2 g mu).
__device__ __forceinline__ float hg_dlog_dg(float g, float mu)
{
    return __fdividef(-2.0f * g, 1.0f - g * g) - __fdividef(3.0f * (g - mu), fmaxf(1.0f + g * g - 2.0f * g * mu, 1e-12f));
}

// Cosine-weighted direction about +z, cos(theta) = sqrt(xi1) > 0.
__device__ __forceinline__ void cosine_up(float xi1, float xi2, float out[3])
{
    const float st = sqrtf(fmaxf(0.0f, 1.0f - xi1));
    float sp, cp;
    sincospif(2.0f * xi2, &sp, &cp);
    out[0] = st * cp; out[1] = st * sp; out[2] = sqrtf(xi1);
}

// Cosine-weighted direction about the unit normal n (Duff et al. frame);
// the same draws as cosine_up, tilted.
__device__ __forceinline__ void cosine_about(const float n[3], float xi1, float xi2, float out[3])
{
    const float sign = copysignf(1.0f, n[2]);
    const float a = -__frcp_rn(sign + n[2]);
    const float b = n[0] * n[1] * a;
    const float st = sqrtf(fmaxf(0.0f, 1.0f - xi1)), ct = sqrtf(xi1);
    float sp, cp;
    sincospif(2.0f * xi2, &sp, &cp);
    const float c = st * cp, s = st * sp;
    out[0] = c * (1.0f + sign * n[0] * n[0] * a) + s * b + ct * n[0];
    out[1] = c * (sign * b) + s * (sign + n[1] * n[1] * a) + ct * n[1];
    out[2] = c * (-sign * n[0]) + s * (-n[1]) + ct * n[2];
}

// --------------------------------------------------------------------------
// Heightfield ground.  Cell (i, j) is cut along its diagonal from corner
// (i, j) to (i+1, j+1): with u, v the position in the cell scaled to [0, 1],
// triangle A (u >= v) has corners 00, 10, 11 and triangle B (u < v) corners
// 00, 11, 01; on a triangle the surface is z = c + a u + b v.
// --------------------------------------------------------------------------
constexpr float kTerrainOffset = 1e-5f;   // km: a path leaves the surface this far along its normal

__device__ __forceinline__ int wrap_mod(int i, int n)
{
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Periodic index on axis a at pyramid level L (n = hn >> 2L cells).
__device__ __forceinline__ int hf_wrap(const DevScene& S, int a, int i, int L)
{
    return S.hmask[a] >= 0 ? (i & (S.hmask[a] >> (2 * L))) : wrap_mod(i, S.hn[a] >> (2 * L));
}

// The 4 corner heights of cell (i, j): h[0] = (i, j), h[1] = (i+1, j),
// h[2] = (i, j+1), h[3] = (i+1, j+1).
__device__ __forceinline__ void hf_corners(const DevScene& S, int i, int j, float h[4])
{
    const int i0 = hf_wrap(S, 0, i, 0), i1 = hf_wrap(S, 0, i + 1, 0);
    const size_t r0 = (size_t)hf_wrap(S, 1, j, 0) * S.hn[0], r1 = (size_t)hf_wrap(S, 1, j + 1, 0) * S.hn[0];
    MCRT_CHECK(i0 >= 0 && i0 < S.hn[0] && i1 >= 0 && i1 < S.hn[0] && r0 < (size_t)S.hn[0] * S.hn[1] &&
                   r1 < (size_t)S.hn[0] * S.hn[1], 4);
    h[0] = __ldg(S.hf + r0 + i0);
    h[1] = __ldg(S.hf + r0 + i1);
    h[2] = __ldg(S.hf + r1 + i0);
    h[3] = __ldg(S.hf + r1 + i1);
}

__device__ __forceinline__ void hf_plane(const float h[4], bool triA, float* a, float* b, float* c)
{
    *c = h[0];
    if (triA) { *a = h[1] - h[0]; *b = h[3] - h[1]; }
    else      { *a = h[3] - h[2]; *b = h[2] - h[0]; }
}

// Surface height at (x, y) and the unit upward normal of its triangle.
__device__ __forceinline__ float hf_height(const DevScene& S, float x, float y, float n[3])
{
    const float fx = x * S.inv_hc[0], fy = y * S.inv_hc[1];
    const int i = __float2int_rd(fx), j = __float2int_rd(fy);
    const float u = fx - (float)i, v = fy - (float)j;
    float hc4[4];
    hf_corners(S, i, j, hc4);
    float a, b, c;
    hf_plane(hc4, u >= v, &a, &b, &c);
    const float gx = a * S.inv_hc[0], gy = b * S.inv_hc[1];
    const float inv = rsqrtf(gx * gx + gy * gy + 1.0f);
    n[0] = -gx * inv; n[1] = -gy * inv; n[2] = inv;
    return c + a * u + b * v;
}

// Ray-surface walk.  Only the part of the ray o + t d with z <= hmax can
// hit (it reaches z = 0, at or below every height, last).  The ray's
// horizontal projection walks the max pyramid over unwrapped cell indices:
// a cell whose maximum lies below the ray's lowest point over the cell is
// skipped whole, otherwise the walk descends into its 4 x 4 children; after
// a step that leaves the parent block it climbs one level.  A ray starting
// inside the relief layer starts at level 0 (it is near the surface), one
// entering from above at the top level.  In a level-0 cell the ray crosses
// at most two triangle pieces (split where u = v); on a piece the ray's
// height above the plane, f(t), is linear and the hit is where f first
// reaches 0 (the piece start if f <= 0 there).  A horizontal ray is walked
// for at most two domain lengths.  The walk is split into a start and
// single steps so the tracer can interleave it with other lanes' work.
struct TerrainWalk {
    int L, i, j;
    float t, t1;
};

// Sets up the walk; false when the ray cannot meet the surface.
__device__ __forceinline__ bool terrain_walk_begin(const DevScene& S, const float o[3], const float d[3],
                                                   TerrainWalk& W)
{
    float t0 = 0.0f;
    if (o[2] > S.hmax) {
        if (!(d[2] < 0.0f)) return false;
        t0 = __fdiv_rn(S.hmax - o[2], d[2]);
    }
    if (d[2] < 0.0f) W.t1 = __fdiv_rn(-o[2], d[2]);
    else if (d[2] > 0.0f) W.t1 = __fdiv_rn(S.hmax - o[2], d[2]);
    else W.t1 = 2.0f * fmaxf(S.Lper[0], S.Lper[1]);
    if (W.t1 < t0) return false;
    W.L = t0 > 0.0f ? S.hlev - 1 : 0;
    W.t = t0;
    const float cx = S.hc[0] * (float)(1 << (2 * W.L)), cy = S.hc[1] * (float)(1 << (2 * W.L));
    const float x = __fmaf_rn(t0, d[0], o[0]), y = __fmaf_rn(t0, d[1], o[1]);
    W.i = __float2int_rd(__fdiv_rn(x, cx));
    W.j = __float2int_rd(__fdiv_rn(y, cy));
    if (d[0] < 0.0f && (float)W.i * cx == x) W.i -= 1;
    if (d[1] < 0.0f && (float)W.j * cy == y) W.j -= 1;
    return true;
}

// One step of the walk (a descent, a cell test and step, or a climb).
// Returns true when the walk is over, with *t_hit the hit distance or +inf.
__device__ __forceinline__ bool terrain_walk_step(const DevScene& S, const float o[3], const float d[3],
                                                  const float inv_d[3], TerrainWalk& W, float* t_hit)
{
    const float kInf = __int_as_float(0x7f800000);
    const int sh = 2 * W.L;
    const float cx = S.hc[0] * (float)(1 << sh), cy = S.hc[1] * (float)(1 << sh);
    const float tx = d[0] > 0.0f ? ((float)(W.i + 1) * cx - o[0]) * inv_d[0]
                   : d[0] < 0.0f ? ((float)W.i * cx - o[0]) * inv_d[0] : kInf;
    const float ty = d[1] > 0.0f ? ((float)(W.j + 1) * cy - o[1]) * inv_d[1]
                   : d[1] < 0.0f ? ((float)W.j * cy - o[1]) * inv_d[1] : kInf;
    const float te = fmaxf(fminf(fminf(tx, ty), W.t1), W.t);
    const int nx = S.hn[0] >> sh;
    MCRT_CHECK(W.L >= 0 && W.L < S.hlev && hf_wrap(S, 0, W.i, W.L) < nx && hf_wrap(S, 1, W.j, W.L) < (S.hn[1] >> sh) &&
                   hf_wrap(S, 0, W.i, W.L) >= 0 && hf_wrap(S, 1, W.j, W.L) >= 0, 5);
    const float cmax = __ldg(S.hpyr + S.hoff[W.L] + (size_t)hf_wrap(S, 1, W.j, W.L) * nx + hf_wrap(S, 0, W.i, W.L));
    const float zlo = __fmaf_rn(d[2] < 0.0f ? te : W.t, d[2], o[2]);
    if (zlo <= cmax) {
        if (W.L > 0) {
            // descend into the child holding the point at t (1 / child size:
            // inv_hc scaled by 4^-(L-1), exact)
            const float hx = cx * 0.25f, hy = cy * 0.25f;
            const float x = __fmaf_rn(W.t, d[0], o[0]), y = __fmaf_rn(W.t, d[1], o[1]);
            const float sc = __int_as_float((127 - 2 * (W.L - 1)) << 23);
            int ci = __float2int_rd(x * (S.inv_hc[0] * sc)), cj = __float2int_rd(y * (S.inv_hc[1] * sc));
            if (d[0] < 0.0f && (float)ci * hx == x) ci -= 1;
            if (d[1] < 0.0f && (float)cj * hy == y) cj -= 1;
            W.i = min(max(ci, 4 * W.i), 4 * W.i + 3);
            W.j = min(max(cj, 4 * W.j), 4 * W.j + 3);
            --W.L;
            return false;
        }
        // level 0: the triangle pieces of [t, te]
        const float g0 = (o[0] * S.inv_hc[0] - (float)W.i) - (o[1] * S.inv_hc[1] - (float)W.j);
        const float g1 = d[0] * S.inv_hc[0] - d[1] * S.inv_hc[1];
        float cut1 = te;
        int np = 1;
        if (g1 != 0.0f) {
            const float tm = __fdividef(-g0, g1);
            if (tm > W.t && tm < te) { cut1 = tm; np = 2; }
        }
        float hc4[4];
        hf_corners(S, W.i, W.j, hc4);
        for (int q = 0; q < np; ++q) {
            const float a0 = q == 0 ? W.t : cut1, b0 = q == 0 ? cut1 : te;
            const bool triA = __fmaf_rn(g1, 0.5f * (a0 + b0), g0) >= 0.0f;
            float A, B, Cc;
            hf_plane(hc4, triA, &A, &B, &Cc);
            const float ua = __fmaf_rn(a0, d[0], o[0]) * S.inv_hc[0] - (float)W.i;
            const float va = __fmaf_rn(a0, d[1], o[1]) * S.inv_hc[1] - (float)W.j;
            const float ub = __fmaf_rn(b0, d[0], o[0]) * S.inv_hc[0] - (float)W.i;
            const float vb = __fmaf_rn(b0, d[1], o[1]) * S.inv_hc[1] - (float)W.j;
            const float fa = __fmaf_rn(a0, d[2], o[2]) - (Cc + A * ua + B * va);
            const float fb = __fmaf_rn(b0, d[2], o[2]) - (Cc + A * ub + B * vb);
            if (fa <= 0.0f) { *t_hit = a0; return true; }
            if (fb <= 0.0f) { *t_hit = a0 + fa * __fdividef(b0 - a0, fa - fb); return true; }
        }
    }
    // step to the next cell of this level; climb when leaving the parent block
    if (te >= W.t1) { *t_hit = kInf; return true; }
    const int pi = W.i >> 2, pj = W.j >> 2;
    if (tx <= ty) W.i += d[0] > 0.0f ? 1 : -1;
    else W.j += d[1] > 0.0f ? 1 : -1;
    W.t = te;
    if (W.L < S.hlev - 1 && ((W.i >> 2) != pi || (W.j >> 2) != pj)) {
        W.i >>= 2;
        W.j >>= 2;
        ++W.L;
    }
    return false;
}

// First distance t >= 0 at which the ray o + t d meets the surface, or
// +inf (the whole walk at once; at most 2^16 steps).
static __device__ __forceinline__ float terrain_hit(const DevScene& S, const float o[3], const float d[3])
{
    const float kInf = __int_as_float(0x7f800000);
    TerrainWalk W;
    if (!terrain_walk_begin(S, o, d, W)) return kInf;
    const float inv_d[3] = {d[0] != 0.0f ? __frcp_rn(d[0]) : 0.0f, d[1] != 0.0f ? __frcp_rn(d[1]) : 0.0f, 0.0f};
    float th = kInf;
    for (int it = 0; it < (1 << 16); ++it)
        if (terrain_walk_step(S, o, d, inv_d, W, &th)) return th;
    return kInf;
}

// Single-scattering albedo of the mixture at total extinction k_tot.
__device__ __forceinline__ float omega_at(const DevScene& S, float k_tot)
{
    const float k = k_tot - S.k_gas;
    const float kc = fmaxf(k - S.k_clear, 0.0f);
    const float kcl = k - kc;
    return k_tot > 0.0f ? __fdividef(kc * S.ssa_cloud + kcl * S.ssa_clear, k_tot) : 0.0f;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace mcrt
