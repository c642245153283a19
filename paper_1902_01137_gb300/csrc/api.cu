// api.cu -- the C ABI declared in include/mcrt.h: argument checks, device
// memory ownership, launch configuration and status reporting.  Every device
// step of the method runs in the kernels of majorant.cu and trace.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>
#include <utility>

#include "mcrt_internal.h"

using namespace mcrt;

namespace {

thread_local std::string g_err;   // errors of calls without a context

int fail(mcrt_ctx* ctx, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(mcrt_ctx* ctx, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_err = buf;
    return code;
}

#define CK(ctx, call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define LAUNCH(ctx, call)      \
    do {                       \
        (ctx)->launches++;     \
        CK((ctx), (call));     \
    } while (0)

template <class T>
cudaError_t dalloc(mcrt_ctx* ctx, T** p, size_t bytes)
{
    return cudaMallocAsync(reinterpret_cast<void**>(p), bytes == 0 ? 16 : bytes, ctx->stream);
}

void dfree(mcrt_ctx* ctx, void* p)
{
    if (p) cudaFreeAsync(p, ctx->stream);
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

}  // namespace

namespace mcrt {

DevScene make_dev_scene(const mcrt_scene* sc, float k_gas)
{
    DevScene S{};
    for (int a = 0; a < 3; ++a) {
        S.n[a] = sc->n[a];
        S.h[a] = sc->h[a];
        S.inv_h[a] = 1.0f / sc->h[a];
        S.nb[a] = sc->nb[a];
    }
    S.Lper[0] = (float)sc->n[0] * sc->h[0];
    S.Lper[1] = (float)sc->n[1] * sc->h[1];
    if (sc->storage == MCRT_STORAGE_BF16) S.vox16 = static_cast<const uint16_t*>(sc->d_vox);
    else S.vox = static_cast<const float*>(sc->d_vox);
    // the leaf map last built (ensure_leaf) decides the grid tracked
    if (sc->leaf_grid == MCRT_GRID_OCTREE && sc->oct_levels > 0) {
        S.leaf = sc->d_oleaf;
        S.lb = 1;
        for (int a = 0; a < 3; ++a) S.nl[a] = sc->oct_dims[3 + a];
    } else {
        S.leaf = sc->d_leaf;
        S.lb = 3;
        for (int a = 0; a < 3; ++a) S.nl[a] = sc->nb[a];
    }
    S.k_clear = sc->k_clear;
    S.ssa_clear = sc->ssa_clear;
    S.ssa_cloud = sc->ssa_cloud;
    S.g = sc->g;
    S.k_gas = k_gas;
    S.albedo = sc->albedo;
    S.rayleigh = sc->clear_phase == MCRT_PHASE_RAYLEIGH;
    for (int a = 0; a < 3; ++a) S.sun[a] = sc->sun[a];
    if (sc->d_hf) {
        S.hf = sc->d_hf;
        S.hpyr = sc->d_hpyr;
        for (int a = 0; a < 2; ++a) {
            S.hn[a] = sc->hn[a];
            S.hmask[a] = (sc->hn[a] & (sc->hn[a] - 1)) == 0 ? sc->hn[a] - 1 : -1;
            S.hc[a] = (float)((double)sc->n[a] * sc->h[a] / sc->hn[a]);
            S.inv_hc[a] = 1.0f / S.hc[a];
        }
        S.hmax = sc->hmax;
        S.hlev = sc->hlev;
        for (int L = 0; L < kMaxHfLevels; ++L) S.hoff[L] = sc->hoff[L];
    }
    return S;
}

}  // namespace mcrt

extern "C" {

int mcrt_version(int32_t* abi_version)
{
    if (abi_version) *abi_version = MCRT_ABI_VERSION;
    return MCRT_OK;
}

const char* mcrt_status_string(int s)
{
    switch (s) {
    case MCRT_OK: return "ok";
    case MCRT_ERR_ARG: return "invalid argument";
    case MCRT_ERR_OOM: return "out of memory";
    case MCRT_ERR_CUDA: return "CUDA error";
    case MCRT_ERR_TIMEOUT: return "deadline expired";
    case MCRT_ERR_CANCELLED: return "cancelled";
    case MCRT_ERR_STATE: return "call out of order";
    case MCRT_ERR_BOUNDS: return "buffer too small";
    case MCRT_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

int mcrt_create(mcrt_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(nullptr, MCRT_ERR_ARG, "mcrt_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, MCRT_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev)
        return fail(nullptr, MCRT_ERR_ARG, "mcrt_create: device %d out of range [0, %d)", device, ndev);
    mcrt_ctx* c = new (std::nothrow) mcrt_ctx();
    if (!c) return fail(nullptr, MCRT_ERR_OOM, "mcrt_create: host allocation failed");
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    int l2 = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, MCRT_ERR_CUDA, "mcrt_create: %s", cudaGetErrorString(e));
    }
    c->l2_bytes = (size_t)l2;
    *out = c;
    return MCRT_OK;
}

int mcrt_destroy(mcrt_ctx* ctx)
{
    if (!ctx) return fail(nullptr, MCRT_ERR_ARG, "mcrt_destroy: NULL context");
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
    return MCRT_OK;
}

const char* mcrt_last_error(const mcrt_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

int mcrt_launch_count(const mcrt_ctx* ctx, uint64_t* count)
{
    if (!ctx || !count) return fail(nullptr, MCRT_ERR_ARG, "mcrt_launch_count: NULL argument");
    *count = ctx->launches;
    return MCRT_OK;
}

// ---------------------------------------------------------------------------
// Scene
// ---------------------------------------------------------------------------
int mcrt_scene_create(mcrt_ctx* ctx, const mcrt_field_desc* d, mcrt_scene** out)
{
    NvtxRange nvtx_range("mcrt_scene_create");
    if (!ctx || !d || !out) return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: NULL argument");
    *out = nullptr;
    ctx->err.clear();
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx > (1 << 20) || d->ny > (1 << 20) || d->nz > (1 << 20))
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: bad size %d x %d x %d", d->nx, d->ny, d->nz);
    if (!finite_pos(d->dx) || !finite_pos(d->dy) || !finite_pos(d->dz))
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: voxel size must be finite and > 0");
    if (!d->ext) return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: ext is NULL");
    if (d->ext_mem != MCRT_MEM_HOST && d->ext_mem != MCRT_MEM_DEVICE)
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: ext_mem must be MCRT_MEM_HOST or MCRT_MEM_DEVICE");
    if (d->storage != MCRT_STORAGE_F32 && d->storage != MCRT_STORAGE_BF16)
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: bad storage %d", d->storage);
    if (!(std::isfinite(d->k_clear) && d->k_clear >= 0.0f))
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: k_clear must be finite and >= 0");
    if (!(d->ssa_clear >= 0.0f && d->ssa_clear <= 1.0f && d->ssa_cloud >= 0.0f && d->ssa_cloud <= 1.0f))
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: albedos must be in [0, 1]");
    if (!(std::fabs(d->hg_g) < 1.0f)) return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_create: |g| must be < 1");
    CK(ctx, cudaSetDevice(ctx->device));
    mcrt_scene* sc = new (std::nothrow) mcrt_scene();
    if (!sc) return fail(ctx, MCRT_ERR_OOM, "mcrt_scene_create: host allocation failed");
    sc->ctx = ctx;
    sc->n[0] = d->nx; sc->n[1] = d->ny; sc->n[2] = d->nz;
    sc->h[0] = d->dx; sc->h[1] = d->dy; sc->h[2] = d->dz;
    for (int a = 0; a < 3; ++a) sc->nb[a] = ceil_div(sc->n[a], 8);
    sc->k_clear = d->k_clear; sc->ssa_clear = d->ssa_clear; sc->ssa_cloud = d->ssa_cloud; sc->g = d->hg_g;
    sc->storage = d->storage;
    const size_t nbricks = (size_t)sc->nb[0] * sc->nb[1] * sc->nb[2];
    sc->vox_bytes = nbricks * 512 * (sc->storage == MCRT_STORAGE_BF16 ? 2 : 4);
    // pyramid capacity: up to 8 levels; level dims filled now
    sc->lev_off.assign(10, 0);
    sc->lev_dims.assign(30, 0);
    size_t tot = 0;
    for (int L = 1; L <= 8; ++L) {
        int f = 1 << (3 * L);
        int dd[3] = {ceil_div(sc->n[0], f), ceil_div(sc->n[1], f), ceil_div(sc->n[2], f)};
        for (int a = 0; a < 3; ++a) sc->lev_dims[3 * L + a] = dd[a];
        sc->lev_off[L] = tot;
        tot += (size_t)dd[0] * dd[1] * dd[2];
    }
    sc->pyr_capacity = tot;
    cudaError_t e = dalloc(ctx, &sc->d_vox, sc->vox_bytes);
    if (e == cudaSuccess) e = dalloc(ctx, &sc->d_pyr, 2 * tot * sizeof(float));   // max levels, then min levels
    if (e == cudaSuccess) e = dalloc(ctx, &sc->d_leaf, nbricks * sizeof(uint2));
    const float* src = d->ext;
    float* staging = nullptr;
    const size_t nvox = (size_t)d->nx * d->ny * d->nz;
    if (e == cudaSuccess && d->ext_mem == MCRT_MEM_HOST) {
        // page-locked host memory mapped into the device's address space is
        // read by the relayout kernel itself, over the host link, in the
        // same pass that writes the bricks; other host memory goes through
        // a device staging copy
        cudaPointerAttributes pa{};
        const float* mapped = nullptr;
        if (cudaPointerGetAttributes(&pa, d->ext) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            mapped = static_cast<const float*>(pa.devicePointer);
        else
            (void)cudaGetLastError();
        if (mapped) {
            src = mapped;
        } else {
            e = dalloc(ctx, &staging, nvox * sizeof(float));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(staging, d->ext, nvox * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
            src = staging;
        }
    }
    if (e == cudaSuccess) {
        ctx->launches++;
        e = launch_relayout(src, sc, ctx->stream);
    }
    if (staging) dfree(ctx, staging);
    if (e != cudaSuccess) {
        dfree(ctx, sc->d_vox); dfree(ctx, sc->d_pyr); dfree(ctx, sc->d_leaf);
        delete sc;
        return fail(ctx, e == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA, "mcrt_scene_create: %s",
                    cudaGetErrorString(e));
    }
    if (d->ext_mem == MCRT_MEM_HOST) {
        // the caller's host buffer is only borrowed for this call
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    *out = sc;
    return MCRT_OK;
}

int mcrt_scene_destroy(mcrt_scene* sc)
{
    if (!sc) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_destroy: NULL scene");
    mcrt_ctx* ctx = sc->ctx;
    dfree(ctx, sc->d_vox);
    dfree(ctx, sc->d_pyr);
    dfree(ctx, sc->d_leaf);
    dfree(ctx, sc->d_oct);
    dfree(ctx, sc->d_oleaf);
    dfree(ctx, sc->d_hf);
    dfree(ctx, sc->d_hpyr);
    cudaStreamSynchronize(ctx->stream);
    delete sc;
    return MCRT_OK;
}

int mcrt_scene_build_majorants(mcrt_scene* sc, int32_t levels)
{
    NvtxRange nvtx_range("mcrt_scene_build_majorants");
    if (!sc) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_build_majorants: NULL scene");
    mcrt_ctx* ctx = sc->ctx;
    if (levels < 0 || levels > 8)
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_build_majorants: levels %d not in [0, 8]", levels);
    if (levels == 0) {
        levels = 1;
        while (levels < 8 && !(sc->lev_dims[3 * levels] == 1 && sc->lev_dims[3 * levels + 1] == 1 &&
                               sc->lev_dims[3 * levels + 2] == 1))
            ++levels;
    }
    CK(ctx, cudaSetDevice(ctx->device));
    for (int L = 2; L <= levels; ++L) {
        LAUNCH(ctx, launch_reduce_level(sc->d_pyr + sc->lev_off[L - 1], &sc->lev_dims[3 * (L - 1)],
                                        sc->d_pyr + sc->lev_off[L], &sc->lev_dims[3 * L], false, ctx->stream));
        float* mn = sc->d_pyr + sc->pyr_capacity;
        LAUNCH(ctx, launch_reduce_level(mn + sc->lev_off[L - 1], &sc->lev_dims[3 * (L - 1)], mn + sc->lev_off[L],
                                        &sc->lev_dims[3 * L], true, ctx->stream));
    }
    sc->levels = levels;
    sc->leaf_valid = false;
    sc->gen++;
    return MCRT_OK;
}

int mcrt_scene_levels(const mcrt_scene* sc, int32_t* levels)
{
    if (!sc || !levels) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_levels: NULL argument");
    *levels = sc->levels;
    return MCRT_OK;
}

int mcrt_scene_majorant_dims(const mcrt_scene* sc, int32_t level, int32_t dims[3])
{
    if (!sc || !dims) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_majorant_dims: NULL argument");
    if (level < 1 || level > 8) return fail(sc->ctx, MCRT_ERR_ARG, "mcrt_scene_majorant_dims: bad level %d", level);
    for (int a = 0; a < 3; ++a) dims[a] = sc->lev_dims[3 * level + a];
    return MCRT_OK;
}

int mcrt_scene_read_majorants(const mcrt_scene* sc, int32_t level, float* host_out, size_t n)
{
    if (!sc || !host_out) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_read_majorants: NULL argument");
    mcrt_ctx* ctx = sc->ctx;
    if (sc->levels == 0) return fail(ctx, MCRT_ERR_STATE, "mcrt_scene_read_majorants: majorants not built");
    if (level < 1 || level > sc->levels)
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_read_majorants: level %d not in [1, %d]", level, sc->levels);
    const size_t cells = (size_t)sc->lev_dims[3 * level] * sc->lev_dims[3 * level + 1] * sc->lev_dims[3 * level + 2];
    if (n < cells) return fail(ctx, MCRT_ERR_BOUNDS, "mcrt_scene_read_majorants: need %zu values", cells);
    CK(ctx, cudaMemcpyAsync(host_out, sc->d_pyr + sc->lev_off[level], cells * sizeof(float), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

int mcrt_scene_read_minorants(const mcrt_scene* sc, int32_t level, float* host_out, size_t n)
{
    if (!sc || !host_out) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_read_minorants: NULL argument");
    mcrt_ctx* ctx = sc->ctx;
    if (sc->levels == 0) return fail(ctx, MCRT_ERR_STATE, "mcrt_scene_read_minorants: majorants not built");
    if (level < 1 || level > sc->levels)
        return fail(ctx, MCRT_ERR_ARG, "mcrt_scene_read_minorants: level %d not in [1, %d]", level, sc->levels);
    const size_t cells = (size_t)sc->lev_dims[3 * level] * sc->lev_dims[3 * level + 1] * sc->lev_dims[3 * level + 2];
    if (n < cells) return fail(ctx, MCRT_ERR_BOUNDS, "mcrt_scene_read_minorants: need %zu values", cells);
    CK(ctx, cudaMemcpyAsync(host_out, sc->d_pyr + sc->pyr_capacity + sc->lev_off[level], cells * sizeof(float),
                            cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

int mcrt_scene_build_octree(mcrt_scene* sc, int32_t levels)
{
    NvtxRange nvtx_range("mcrt_scene_build_octree");
    const char* who = "mcrt_scene_build_octree";
    if (!sc) return fail(nullptr, MCRT_ERR_ARG, "%s: NULL scene", who);
    mcrt_ctx* ctx = sc->ctx;
    if (levels < 0 || levels > kMaxGridLevels)
        return fail(ctx, MCRT_ERR_ARG, "%s: levels %d not in [0, %d]", who, levels, kMaxGridLevels);
    if (levels == 0) {
        const int nmax = std::max(sc->n[0], std::max(sc->n[1], sc->n[2]));
        levels = 1;
        while (levels < kMaxGridLevels && (1 << levels) < nmax) ++levels;
    }
    CK(ctx, cudaSetDevice(ctx->device));
    std::vector<size_t> off(kMaxGridLevels + 2, 0);
    std::vector<int> dims(3 * (kMaxGridLevels + 2), 0);
    size_t tot = 0;
    for (int L = 1; L <= levels; ++L) {
        for (int a = 0; a < 3; ++a) dims[3 * L + a] = ceil_div(sc->n[a], 1 << L);
        off[L] = tot;
        tot += (size_t)dims[3 * L] * dims[3 * L + 1] * dims[3 * L + 2];
    }
    const size_t n1 = (size_t)dims[3] * dims[4] * dims[5];
    // replace the previous octree (its leaf map goes with it)
    if (sc->leaf_grid == MCRT_GRID_OCTREE) sc->leaf_valid = false;
    sc->gen++;
    dfree(ctx, sc->d_oct);
    dfree(ctx, sc->d_oleaf);
    sc->d_oct = nullptr;
    sc->d_oleaf = nullptr;
    sc->oct_levels = 0;
    cudaError_t e = dalloc(ctx, &sc->d_oct, 2 * tot * sizeof(float));
    if (e == cudaSuccess) e = dalloc(ctx, &sc->d_oleaf, n1 * sizeof(uint2));
    if (e != cudaSuccess) {
        dfree(ctx, sc->d_oct);
        dfree(ctx, sc->d_oleaf);
        sc->d_oct = nullptr;
        sc->d_oleaf = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA, "%s: %s", who,
                    cudaGetErrorString(e));
    }
    sc->oct_off = off;
    sc->oct_dims = dims;
    sc->oct_capacity = tot;
    sc->oct_levels = levels;
    ctx->launches += (uint64_t)levels;
    e = launch_octree(sc, make_dev_scene(sc, 0.0f), ctx->stream);
    if (e != cudaSuccess) {
        sc->oct_levels = 0;
        return fail(ctx, MCRT_ERR_CUDA, "%s: %s", who, cudaGetErrorString(e));
    }
    return MCRT_OK;
}

int mcrt_scene_octree_levels(const mcrt_scene* sc, int32_t* levels)
{
    if (!sc || !levels) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_octree_levels: NULL argument");
    *levels = sc->oct_levels;
    return MCRT_OK;
}

int mcrt_scene_octree_dims(const mcrt_scene* sc, int32_t level, int32_t dims[3])
{
    if (!sc || !dims) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_octree_dims: NULL argument");
    if (sc->oct_levels == 0) return fail(sc->ctx, MCRT_ERR_STATE, "mcrt_scene_octree_dims: octree not built");
    if (level < 1 || level > sc->oct_levels)
        return fail(sc->ctx, MCRT_ERR_ARG, "mcrt_scene_octree_dims: level %d not in [1, %d]", level, sc->oct_levels);
    for (int a = 0; a < 3; ++a) dims[a] = sc->oct_dims[3 * level + a];
    return MCRT_OK;
}

int mcrt_scene_read_octree(const mcrt_scene* sc, int32_t level, float* max_out, float* min_out, size_t n)
{
    const char* who = "mcrt_scene_read_octree";
    if (!sc) return fail(nullptr, MCRT_ERR_ARG, "%s: NULL scene", who);
    mcrt_ctx* ctx = sc->ctx;
    if (sc->oct_levels == 0) return fail(ctx, MCRT_ERR_STATE, "%s: octree not built", who);
    if (level < 1 || level > sc->oct_levels)
        return fail(ctx, MCRT_ERR_ARG, "%s: level %d not in [1, %d]", who, level, sc->oct_levels);
    const size_t cells = (size_t)sc->oct_dims[3 * level] * sc->oct_dims[3 * level + 1] * sc->oct_dims[3 * level + 2];
    if (n < cells) return fail(ctx, MCRT_ERR_BOUNDS, "%s: need %zu values", who, cells);
    CK(ctx, cudaSetDevice(ctx->device));
    if (max_out)
        CK(ctx, cudaMemcpyAsync(max_out, sc->d_oct + sc->oct_off[level], cells * sizeof(float), cudaMemcpyDeviceToHost,
                                ctx->stream));
    if (min_out)
        CK(ctx, cudaMemcpyAsync(min_out, sc->d_oct + sc->oct_capacity + sc->oct_off[level], cells * sizeof(float),
                                cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

int mcrt_scene_set_clear_sky_phase(mcrt_scene* sc, int32_t phase)
{
    if (!sc) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_set_clear_sky_phase: NULL scene");
    if (phase != MCRT_PHASE_HG && phase != MCRT_PHASE_RAYLEIGH)
        return fail(sc->ctx, MCRT_ERR_ARG, "mcrt_scene_set_clear_sky_phase: bad phase %d", phase);
    sc->clear_phase = phase;
    sc->gen++;
    return MCRT_OK;
}

int mcrt_scene_set_ground_flat(mcrt_scene* sc, float albedo)
{
    if (!sc) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_set_ground_flat: NULL scene");
    if (!(albedo >= 0.0f && albedo <= 1.0f))
        return fail(sc->ctx, MCRT_ERR_ARG, "mcrt_scene_set_ground_flat: albedo must be in [0, 1]");
    sc->albedo = albedo;
    dfree(sc->ctx, sc->d_hf);
    dfree(sc->ctx, sc->d_hpyr);
    sc->d_hf = sc->d_hpyr = nullptr;
    sc->hlev = 0;
    sc->gen++;
    return MCRT_OK;
}

int mcrt_scene_set_ground_heightfield(mcrt_scene* sc, const float* heights, int32_t hnx, int32_t hny, int32_t mem,
                                      float albedo)
{
    NvtxRange nvtx_range("mcrt_scene_set_ground_heightfield");
    const char* who = "mcrt_scene_set_ground_heightfield";
    if (!sc || !heights) return fail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = sc->ctx;
    if (!(albedo >= 0.0f && albedo <= 1.0f)) return fail(ctx, MCRT_ERR_ARG, "%s: albedo must be in [0, 1]", who);
    if (hnx < 1 || hny < 1 || hnx > (1 << 16) || hny > (1 << 16))
        return fail(ctx, MCRT_ERR_ARG, "%s: bad size %d x %d", who, hnx, hny);
    if (mem != MCRT_MEM_HOST && mem != MCRT_MEM_DEVICE)
        return fail(ctx, MCRT_ERR_ARG, "%s: mem must be MCRT_MEM_HOST or MCRT_MEM_DEVICE", who);
    CK(ctx, cudaSetDevice(ctx->device));
    // levels: 4 x 4 blocks while both sizes divide
    int lev = 1;
    while (lev < kMaxHfLevels && hnx % (1 << (2 * lev)) == 0 && hny % (1 << (2 * lev)) == 0) ++lev;
    int off[kMaxHfLevels] = {};
    size_t total = 0;
    for (int L = 0; L < lev; ++L) {
        off[L] = (int)total;
        total += (size_t)(hnx >> (2 * L)) * (size_t)(hny >> (2 * L));
    }
    const size_t n = (size_t)hnx * hny;
    float *dh = nullptr, *dp = nullptr;
    int* bad = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dh), n * sizeof(float), ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&dp), total * sizeof(float), ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&bad), sizeof(int), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dh, heights, n * sizeof(float),
                            mem == MCRT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream);
    const float top = (float)sc->n[2] * sc->h[2];
    if (e == cudaSuccess) { ctx->launches++; e = launch_hf_check(dh, (long long)n, top, bad, ctx->stream); }
    if (e == cudaSuccess) { ctx->launches += lev; e = launch_hf_pyramid(dh, hnx, hny, dp, off, lev, ctx->stream); }
    const size_t ntop = (size_t)(hnx >> (2 * (lev - 1))) * (size_t)(hny >> (2 * (lev - 1)));
    std::vector<float> tops(ntop);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tops.data(), dp + off[lev - 1], ntop * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (bad) cudaFreeAsync(bad, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess || hbad) {
        dfree(ctx, dh);
        dfree(ctx, dp);
        if (e != cudaSuccess) return fail(ctx, MCRT_ERR_CUDA, "%s: %s", who, cudaGetErrorString(e));
        return fail(ctx, MCRT_ERR_ARG, "%s: heights must be finite and in [0, %g] km", who, (double)top);
    }
    dfree(ctx, sc->d_hf);
    dfree(ctx, sc->d_hpyr);
    sc->d_hf = dh;
    sc->d_hpyr = dp;
    sc->hn[0] = hnx;
    sc->hn[1] = hny;
    sc->hlev = lev;
    for (int L = 0; L < kMaxHfLevels; ++L) sc->hoff[L] = off[L];
    float hm = 0.0f;
    for (float v : tops) hm = std::fmax(hm, v);
    sc->hmax = hm;
    sc->albedo = albedo;
    sc->gen++;
    return MCRT_OK;
}

int mcrt_scene_set_sun(mcrt_scene* sc, float zenith_deg, float azimuth_deg)
{
    if (!sc) return fail(nullptr, MCRT_ERR_ARG, "mcrt_scene_set_sun: NULL scene");
    if (!(zenith_deg >= 0.0f && zenith_deg < 90.0f) || !std::isfinite(azimuth_deg))
        return fail(sc->ctx, MCRT_ERR_ARG, "mcrt_scene_set_sun: zenith must be in [0, 90) degrees");
    const double z = zenith_deg * M_PI / 180.0, a = azimuth_deg * M_PI / 180.0;
    sc->sun_zenith = zenith_deg;
    sc->sun_azimuth = azimuth_deg;
    sc->sun[0] = (float)(std::sin(z) * std::cos(a));
    sc->sun[1] = (float)(std::sin(z) * std::sin(a));
    sc->sun[2] = (float)std::cos(z);
    return MCRT_OK;
}

// ---------------------------------------------------------------------------
// Tracing
// ---------------------------------------------------------------------------
int mcrt_trace_opts_default(mcrt_trace_opts* o)
{
    if (!o) return fail(nullptr, MCRT_ERR_ARG, "mcrt_trace_opts_default: NULL");
    std::memset(o, 0, sizeof(*o));
    o->tau_merge = 1.0f;
    o->finest_level = 0;
    o->sun_mode = MCRT_SUN_RATIO;
    return MCRT_OK;
}

extern "C++" {
namespace mcrt {

// Shared by every trace entry point (the no-allocation call included).
int check_opts(mcrt_scene* sc, const mcrt_trace_opts* o, const char* who)
{
    mcrt_ctx* ctx = sc->ctx;
    if (sc->levels == 0) return fail(ctx, MCRT_ERR_STATE, "%s: majorants not built", who);
    if (!(o->tau_merge >= 0.0f)) return fail(ctx, MCRT_ERR_ARG, "%s: tau_merge must be >= 0", who);
    if (o->finest_level < 0 || o->finest_level > 1 || o->finest_level > sc->levels)
        return fail(ctx, MCRT_ERR_ARG, "%s: finest_level must be 0 or 1", who);
    if (o->max_order < 0) return fail(ctx, MCRT_ERR_ARG, "%s: max_order must be >= 0", who);
    if (o->sun_mode != MCRT_SUN_RATIO && o->sun_mode != MCRT_SUN_DELTA && o->sun_mode != MCRT_SUN_DECOMP)
        return fail(ctx, MCRT_ERR_ARG, "%s: bad sun_mode", who);
    if (o->block_size < 0 || o->block_size > 1024 || (o->block_size % 32) != 0)
        return fail(ctx, MCRT_ERR_ARG, "%s: block_size must be a multiple of 32 up to 1024", who);
    if (o->block_size > 128) return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: block_size above 128", who);
    if (o->grid_size < 0 || o->chunk < 0) return fail(ctx, MCRT_ERR_ARG, "%s: negative launch shape", who);
    if (o->rare_batch < 0 || o->rare_batch > 32) return fail(ctx, MCRT_ERR_ARG, "%s: rare_batch must be in [0, 32]", who);
    if (o->proposal) {
        if (o->proposal->ctx != ctx) return fail(ctx, MCRT_ERR_ARG, "%s: proposal belongs to another context", who);
        if (o->n_learned < 0 || o->n_learned > 64) return fail(ctx, MCRT_ERR_ARG, "%s: n_learned must be in [0, 64]", who);
        if (!(o->mis_alpha >= 0.0f && o->mis_alpha <= 1.0f)) return fail(ctx, MCRT_ERR_ARG, "%s: mis_alpha must be in [0, 1]", who);
        if (o->batch_paths < 0 || o->train_steps < 0 || !(o->learning_rate >= 0.0f))
            return fail(ctx, MCRT_ERR_ARG, "%s: bad learned-mode options", who);
        if (o->count_events) return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: counting with a proposal", who);
        if (sc->d_hf) return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: a proposal over a heightfield ground", who);
        if (o->sun_mode == MCRT_SUN_DECOMP)
            return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: decomposition tracking with a proposal", who);
        if (sc->clear_phase == MCRT_PHASE_RAYLEIGH)
            return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: a proposal with Rayleigh clear air", who);
    }
    if (!(o->deadline_ms >= 0.0)) return fail(ctx, MCRT_ERR_ARG, "%s: deadline_ms must be >= 0", who);
    if (o->grid != MCRT_GRID_PYRAMID && o->grid != MCRT_GRID_OCTREE) return fail(ctx, MCRT_ERR_ARG, "%s: bad grid", who);
    if (o->pixel_order != MCRT_ORDER_COST && o->pixel_order != MCRT_ORDER_RASTER)
        return fail(ctx, MCRT_ERR_ARG, "%s: bad pixel_order", who);
    if (o->grid == MCRT_GRID_OCTREE && sc->oct_levels == 0)
        return fail(ctx, MCRT_ERR_STATE, "%s: octree not built (mcrt_scene_build_octree)", who);
    if (o->shard_count < 0 || o->shard_index < 0 || o->shard_index >= (o->shard_count > 1 ? o->shard_count : 1))
        return fail(ctx, MCRT_ERR_ARG, "%s: shard_index %d of %d", who, o->shard_index, o->shard_count);
    if (o->shard_count > 1 && o->proposal)
        return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: sharding with a proposal", who);
    if (o->schedule != MCRT_SCHEDULE_PERSISTENT && o->schedule != MCRT_SCHEDULE_WAVEFRONT)
        return fail(ctx, MCRT_ERR_ARG, "%s: bad schedule", who);
    if (o->wavefront_slots < 0 || o->wavefront_slots > (1 << 26))
        return fail(ctx, MCRT_ERR_ARG, "%s: wavefront_slots must be in [0, 2^26]", who);
    if (o->schedule == MCRT_SCHEDULE_WAVEFRONT &&
        (o->proposal || o->shard_count > 1 || o->sun_mode == MCRT_SUN_DECOMP || sc->clear_phase == MCRT_PHASE_RAYLEIGH ||
         sc->d_hf || o->count_events || o->deadline_ms > 0.0 || o->cancel_flag))
        return fail(ctx, MCRT_ERR_UNSUPPORTED,
                    "%s: the wavefront schedule traces plain images only (no proposal, shards, decomposition "
                    "tracking, Rayleigh air, heightfield, event counts, deadline or cancel flag)", who);
    return MCRT_OK;
}

int ensure_leaf(mcrt_scene* sc, float tau, int finest, int grid)
{
    mcrt_ctx* ctx = sc->ctx;
    if (sc->leaf_valid && sc->leaf_tau == tau && sc->leaf_finest == finest && sc->leaf_grid == grid) return MCRT_OK;
    LAUNCH(ctx, launch_leafmap(sc, tau, finest, grid, ctx->stream));
    sc->gen++;
    sc->leaf_valid = true;
    sc->leaf_tau = tau;
    sc->leaf_finest = finest;
    sc->leaf_grid = grid;
    return MCRT_OK;
}

}  // namespace mcrt
}  // extern "C++"

namespace {

int get_tally(mcrt_ctx* ctx, int ncells, int nq, mcrt_tally** inout, const char* who)
{
    mcrt_tally* t = *inout;
    if (t && (t->ctx != ctx || t->ncells != ncells || t->nq != nq))
        return fail(ctx, MCRT_ERR_ARG, "%s: tally shape (%d, %d) does not match (%d, %d)", who, t ? t->ncells : 0,
                    t ? t->nq : 0, ncells, nq);
    if (!t) {
        t = new (std::nothrow) mcrt_tally();
        if (!t) return fail(ctx, MCRT_ERR_OOM, "%s: host allocation failed", who);
        t->ctx = ctx;
        t->ncells = ncells;
        t->nq = nq;
        const size_t m = (size_t)ncells * nq;
        cudaError_t e = dalloc(ctx, &t->d_s1, m * sizeof(double));
        if (e == cudaSuccess) e = dalloc(ctx, &t->d_s2, m * sizeof(double));
        if (e == cudaSuccess) e = dalloc(ctx, &t->d_counters, kNumCounters * sizeof(unsigned long long));
        if (e == cudaSuccess) e = dalloc(ctx, &t->d_work, sizeof(WorkState));
        if (e == cudaSuccess) e = dalloc(ctx, &t->d_out, 2 * m * sizeof(double));
        if (e != cudaSuccess) {
            dfree(ctx, t->d_s1); dfree(ctx, t->d_s2); dfree(ctx, t->d_counters); dfree(ctx, t->d_work);
            dfree(ctx, t->d_out);
            delete t;
            return fail(ctx, MCRT_ERR_OOM, "%s: %s", who, cudaGetErrorString(e));
        }
        *inout = t;
    }
    const size_t m = (size_t)ncells * nq;
    t->cell_n.clear();
    CK(ctx, cudaMemsetAsync(t->d_s1, 0, m * sizeof(double), ctx->stream));
    CK(ctx, cudaMemsetAsync(t->d_s2, 0, m * sizeof(double), ctx->stream));
    CK(ctx, cudaMemsetAsync(t->d_counters, 0, kNumCounters * sizeof(unsigned long long), ctx->stream));
    CK(ctx, cudaMemsetAsync(t->d_work, 0, sizeof(WorkState), ctx->stream));
    return MCRT_OK;
}

// Claim order of a camera trace (MCRT_ORDER_COST): per tile of pixels the
// majorant optical depth along its central view ray, tiles sorted by it
// (largest first, ties in raster order), expanded to one pixel per claim
// rank in *d_order (device, freed by the caller with dfree).
int make_claim_order(mcrt_scene* sc, const TraceParams& P, uint32_t** d_order, const char* who)
{
    mcrt_ctx* ctx = sc->ctx;
    int tx = 0;
    const int n = order_tiles(P.width, P.height, &tx);
    float* d_cost = nullptr;
    uint32_t* d_tiles = nullptr;
    CK(ctx, dalloc(ctx, &d_cost, (size_t)n * sizeof(float)));
    ctx->launches++;
    cudaError_t e = launch_view_cost(P, sc->storage == MCRT_STORAGE_BF16, d_cost, ctx->stream);
    std::vector<float> cost((size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cost.data(), d_cost, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost,
                                              ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, d_cost);
    if (e != cudaSuccess) return fail(ctx, MCRT_ERR_CUDA, "%s: claim order: %s", who, cudaGetErrorString(e));
    std::vector<uint32_t> tiles((size_t)2 * n);
    for (int i = 0; i < n; ++i) {
        tiles[i] = (uint32_t)i;
        if (!(cost[i] >= 0.0f)) cost[i] = 3.0e38f;     // NaN: treat as the most costly
    }
    std::stable_sort(tiles.begin(), tiles.begin() + n, [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
    uint32_t acc = 0;
    for (int b = 0; b < n; ++b) {
        const int x0 = (int)(tiles[b] % (uint32_t)tx) * 8, y0 = (int)(tiles[b] / (uint32_t)tx) * 8;
        tiles[n + b] = acc;
        acc += (uint32_t)(std::min(8, P.width - x0) * std::min(8, P.height - y0));
    }
    e = dalloc(ctx, &d_tiles, (size_t)2 * n * sizeof(uint32_t));
    if (e == cudaSuccess) e = dalloc(ctx, d_order, (size_t)P.width * P.height * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tiles, tiles.data(), (size_t)2 * n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess) {
        ctx->launches++;
        e = launch_expand_order(d_tiles, d_tiles + n, n, P.width, P.height, *d_order, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);    // the host vector is read by the copy
    dfree(ctx, d_tiles);
    if (e != cudaSuccess) {
        dfree(ctx, *d_order);
        *d_order = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA, "%s: claim order: %s", who,
                    cudaGetErrorString(e));
    }
    return MCRT_OK;
}

int run_trace(mcrt_scene* sc, TraceParams& P, int sensor, const mcrt_trace_opts* o, mcrt_tally* t, const char* who)
{
    mcrt_ctx* ctx = sc->ctx;
    const bool bf16 = sc->storage == MCRT_STORAGE_BF16;
    const bool count = o->count_events != 0;
    const int block = o->block_size ? o->block_size : 128;
    int grid = o->grid_size;
    if (!grid) grid = ctx->sm_count * trace_blocks_per_sm(sensor, bf16, count, P.S.hf != nullptr, P.sun_mode == MCRT_SUN_DECOMP || P.S.rayleigh, block);
    if (!o->chunk) P.chunk = auto_chunk(P.total, (unsigned long long)grid * block, sensor == kCamera ? P.spp : 0u);
    P.s1 = t->d_s1;
    P.s2 = t->d_s2;
    P.counters = t->d_counters;
    P.work = static_cast<WorkState*>(t->d_work);
    P.deadline_ns = o->deadline_ms > 0.0 ? (unsigned long long)(o->deadline_ms * 1e6) : 0ull;
    P.cancel = reinterpret_cast<const volatile int*>(o->cancel_flag);
    P.max_order = o->max_order;
    P.sun_mode = o->sun_mode;
    P.max_steps = 1u << 22;
    set_rare_batch(P, o->rare_batch);
    cudaEvent_t e0, e1;
    CK(ctx, cudaEventCreate(&e0));
    CK(ctx, cudaEventCreate(&e1));
    CK(ctx, cudaEventRecord(e0, ctx->stream));
    ctx->launches++;
    cudaError_t le = launch_trace(P, sensor, bf16, count, grid, block, ctx->stream);
    CK(ctx, cudaEventRecord(e1, ctx->stream));
    WorkState ws{};
    cudaError_t ce = cudaMemcpyAsync(&ws, t->d_work, sizeof(ws), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(ctx, le);
    CK(ctx, ce);
    CK(ctx, se);
    t->kernel_ms = ms;
    if (ws.status == 1) return fail(ctx, MCRT_ERR_TIMEOUT, "%s: deadline of %g ms expired", who, o->deadline_ms);
    if (ws.status == 2) return fail(ctx, MCRT_ERR_CANCELLED, "%s: cancelled", who);
    return MCRT_OK;
}

// The camera trace as a wavefront of stage kernels over SoA queues.
int run_wavefront(mcrt_scene* sc, TraceParams& P, const mcrt_trace_opts* o, mcrt_tally* t, const char* who)
{
    mcrt_ctx* ctx = sc->ctx;
    P.s1 = t->d_s1;
    P.s2 = t->d_s2;
    P.counters = t->d_counters;
    P.work = static_cast<WorkState*>(t->d_work);
    P.max_order = o->max_order;
    P.sun_mode = o->sun_mode;
    P.max_steps = 1u << 22;
    unsigned long long slots = o->wavefront_slots ? (unsigned long long)o->wavefront_slots : (1ull << 21);
    if (slots > P.total) slots = P.total ? P.total : 1ull;
    WavefrontStats ws{};
    const cudaError_t e = wavefront_camera(P, sc->storage == MCRT_STORAGE_BF16, (unsigned)slots, ctx->sm_count,
                                           ctx->stream, &ws);
    ctx->launches += ws.launches;
    if (e != cudaSuccess)
        return fail(ctx, e == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA, "%s: wavefront: %s", who,
                    cudaGetErrorString(e));
    if (ws.overflow) return fail(ctx, MCRT_ERR_CUDA, "%s: wavefront queue overflow (%u)", who, ws.overflow);
    t->kernel_ms = ws.ms;
    return MCRT_OK;
}

// Learned proposal: paths are traced in batches; within a batch, pass 0
// runs fresh paths up to their first volume vertex, the network evaluates the
// stopped paths' features, and each later pass resumes them (one-sample MIS
// direction) up to the next learned vertex; after n_learned passes the paths
// finish with HG sampling.  With learning on, every batch ends with Adam
// steps on the vertices its resumed paths recorded.
int run_learned(mcrt_scene* sc, const TraceParams& P0, int sensor, const mcrt_trace_opts* o, mcrt_tally* t,
                unsigned long long spp, const char* who)
{
    mcrt_ctx* ctx = sc->ctx;
    mcrt_proposal* prop = o->proposal;
    const bool bf16 = sc->storage == MCRT_STORAGE_BF16;
    const int NL = o->n_learned ? o->n_learned : 8;
    const float alpha = o->mis_alpha > 0.0f ? o->mis_alpha : 0.5f;
    const float lr = o->learning_rate > 0.0f ? o->learning_rate : 1e-3f;
    const int steps = o->train_steps ? o->train_steps : 1;
    // a frozen network takes large batches: each batch ends every pass with
    // its slowest paths, so fewer, larger batches waste less of the GPU
    unsigned long long B = o->batch_paths ? (unsigned long long)o->batch_paths : (o->learn ? (1ull << 21) : (1ull << 25));
    if (B < spp) B = spp;
    B = (B / spp) * spp;                                 // batches hold whole pixels
    const unsigned long long total = P0.total;
    RecordDump* dump = ctx->rec_dump;                   // records to the host, no training
    if (dump) B = total;
    if (B > total) B = total;
    const unsigned rec_cap = (o->learn || dump) ? (1u << 20) : 0u;
    const int block = o->block_size ? o->block_size : 128;
    const int grid = o->grid_size ? o->grid_size : ctx->sm_count * trace_learned_blocks_per_sm(sensor, bf16, block);
    // work buffers
    uint4 *qa = nullptr, *qb = nullptr, *fa = nullptr, *fb = nullptr, *rfeat = nullptr;
    float *mix = nullptr, *fin = nullptr, *rdir = nullptr, *rval = nullptr, *tgt = nullptr;
    unsigned* cnt = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(p), bytes ? bytes : 16, ctx->stream);
    };
    A(&qa, B * 64); A(&qb, B * 64); A(&fa, B * 32); A(&fb, B * 32); A(&mix, B * 192); A(&fin, B * 4);
    A(&cnt, 16);
    if (rec_cap) { A(&rfeat, (size_t)rec_cap * 32); A(&rdir, (size_t)rec_cap * 12); A(&rval, (size_t)rec_cap * 16); A(&tgt, (size_t)rec_cap * 4); }
    auto release = [&]() {
        for (void* p : {(void*)qa, (void*)qb, (void*)fa, (void*)fb, (void*)mix, (void*)fin, (void*)cnt, (void*)rfeat,
                        (void*)rdir, (void*)rval, (void*)tgt})
            if (p) cudaFreeAsync(p, ctx->stream);
    };
    if (e != cudaSuccess) { release(); return fail(ctx, MCRT_ERR_OOM, "%s: %s", who, cudaGetErrorString(e)); }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
    int status = 0;
    const int lev2 = sc->levels >= 2 ? 2 : sc->levels;
    for (unsigned long long b0 = 0; b0 < total && e == cudaSuccess && status == 0; b0 += B) {
        const unsigned long long nb = (total - b0 < B) ? total - b0 : B;
        const bool warm = o->learn && prop->step == 0 && !dump;   // untrained network: HG only, records collected
        TraceParams P = P0;
        P.learned = 1;
        P.n_learned = NL;
        P.mis_alpha = warm ? 1.0f : alpha;
        P.path_base = b0;
        P.final_score = fin;
        P.pyr1 = sc->d_pyr + sc->lev_off[1];
        P.pyr2 = sc->d_pyr + sc->lev_off[lev2];
        for (int a = 0; a < 3; ++a) { P.d1[a] = sc->lev_dims[3 + a]; P.d2[a] = sc->lev_dims[3 * lev2 + a]; }
        P.lev2 = lev2;
        P.rec_cap = rec_cap;
        P.rec_slots = rec_cap ? rec_cap / (unsigned)NL : 0u;
        P.rec_feat = rfeat; P.rec_dir = rdir; P.rec_val = rval;
        P.rec_count = rec_cap ? cnt + 1 : nullptr;
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 16, ctx->stream);
        uint4 *qin = qa, *qout = qb, *fin_feat = fa, *fout = fb;
        unsigned n_in = 0;
        for (int r = 0; r <= NL && e == cudaSuccess; ++r) {
            P.resume = r > 0;
            P.total = r == 0 ? nb : n_in;
            P.chunk = r > 0 ? 1u
                            : (o->chunk ? P0.chunk
                                        : auto_chunk(nb, (unsigned long long)grid * block,
                                                     sensor == kCamera ? (uint32_t)spp : 0u));
            P.qin = qin; P.qin_feat = fin_feat; P.qin_mix = mix;
            P.qout = qout; P.qout_feat = fout; P.qout_count = cnt; P.qout_cap = (unsigned)nb;
            if (P.total == 0) break;
            if (r > 0) {
                ctx->launches++;
                e = launch_mlp_infer(prop->d_wbf, prop->d_bias, fin_feat, (int)n_in, mix, nullptr, ctx->sm_count,
                                     ctx->stream, true);
            }
            if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4, ctx->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(t->d_work, 0, sizeof(WorkState), ctx->stream);
            if (e == cudaSuccess) { ctx->launches++; e = launch_trace_learned(P, sensor, bf16, grid, block, ctx->stream); }
            WorkState ws{};
            unsigned n_out = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&n_out, cnt, 4, cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&ws, t->d_work, sizeof(ws), cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (ws.status) { status = ws.status; break; }
            n_in = n_out;
            // the outgoing buffers of this pass are the incoming ones of the next
            qin = (r % 2 == 0) ? qb : qa;
            qout = (r % 2 == 0) ? qa : qb;
            fin_feat = (r % 2 == 0) ? fb : fa;
            fout = (r % 2 == 0) ? fa : fb;
        }
        if (e == cudaSuccess && status == 0 && rec_cap) {
            unsigned nrec = 0;
            e = cudaMemcpyAsync(&nrec, cnt + 1, 4, cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (nrec > rec_cap) nrec = rec_cap;
            if (e == cudaSuccess && nrec > 0) {
                ctx->launches++;
                e = launch_targets(rval, fin, nrec, tgt, ctx->stream);
                if (dump && e == cudaSuccess) {
                    const unsigned nc = nrec < (unsigned)dump->cap ? nrec : (unsigned)dump->cap;
                    std::vector<uint16_t> hf((size_t)nc * 16);
                    std::vector<float> hv((size_t)nc * 4), ht(nc);
                    e = cudaMemcpyAsync(hf.data(), rfeat, hf.size() * 2, cudaMemcpyDeviceToHost, ctx->stream);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(dump->dir, rdir, (size_t)nc * 12, cudaMemcpyDeviceToHost, ctx->stream);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(hv.data(), rval, hv.size() * 4, cudaMemcpyDeviceToHost, ctx->stream);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(ht.data(), tgt, ht.size() * 4, cudaMemcpyDeviceToHost, ctx->stream);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
                    for (unsigned i = 0; e == cudaSuccess && i < nc; ++i) {
                        for (int a = 0; a < 9; ++a) {
                            const uint32_t bits = (uint32_t)hf[(size_t)i * 16 + a] << 16;
                            std::memcpy(&dump->feat[(size_t)i * 9 + a], &bits, 4);
                        }
                        uint32_t pid;
                        std::memcpy(&pid, &hv[(size_t)i * 4 + 3], 4);
                        dump->path[i] = b0 + pid;
                        dump->val[(size_t)i * 4] = hv[(size_t)i * 4];
                        dump->val[(size_t)i * 4 + 1] = hv[(size_t)i * 4 + 1];
                        dump->val[(size_t)i * 4 + 2] = hv[(size_t)i * 4 + 2];
                        dump->val[(size_t)i * 4 + 3] = ht[i];
                    }
                }
                if (dump) dump->count = (int32_t)nrec;
                for (int k = 0; k < steps && e == cudaSuccess && !dump; ++k) {
                    e = cudaMemsetAsync(prop->d_grad, 0, kMlpParams * sizeof(float), ctx->stream);
                    if (e == cudaSuccess) {
                        ctx->launches += 3;
                        e = prop->train_mode == MCRT_TRAIN_FP32
                                ? launch_mlp_train(prop->d_params, rfeat, rdir, tgt, (int)nrec, 1.0f / (float)nrec,
                                                   prop->d_grad, prop->d_loss, ctx->sm_count, ctx->stream)
                                : launch_mlp_train_tc(prop->d_wbf, prop->d_bias, prop->d_params, rfeat, rdir, tgt,
                                                      (int)nrec, 1.0f / (float)nrec, prop->d_grad, prop->d_loss,
                                                      ctx->sm_count, ctx->stream);
                    }
                    if (e == cudaSuccess) {
                        prop->step++;
                        e = launch_adam(prop->d_params, prop->d_m, prop->d_v, prop->d_grad, kMlpParams, lr, 0.9f, 0.999f,
                                        1e-8f, prop->step, ctx->stream);
                    }
                    if (e == cudaSuccess) e = launch_pack(prop->d_params, prop->d_wbf, prop->d_bias, ctx->stream);
                }
            }
        }
    }
    cudaEventRecord(e1, ctx->stream);
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    CK(ctx, e);
    CK(ctx, se);
    t->kernel_ms = ms;
    int terr = 0;
    CK(ctx, tc5_take_error(&terr, ctx->stream));
    if (terr) return fail(ctx, MCRT_ERR_TIMEOUT, "%s: a tensor-core wait of the proposal network ran out", who);
    if (status == 1) return fail(ctx, MCRT_ERR_TIMEOUT, "%s: deadline of %g ms expired", who, o->deadline_ms);
    if (status == 2) return fail(ctx, MCRT_ERR_CANCELLED, "%s: cancelled", who);
    return MCRT_OK;
}

}  // namespace

int mcrt_trace_camera(mcrt_scene* sc, const mcrt_camera_desc* cam, uint32_t spp, uint64_t seed,
                      const mcrt_trace_opts* opts, mcrt_tally** tally)
{
    NvtxRange nvtx_range("mcrt_trace_camera");
    const char* who = "mcrt_trace_camera";
    if (!sc || !cam || !tally) return fail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = sc->ctx;
    ctx->err.clear();
    mcrt_trace_opts dflt;
    mcrt_trace_opts_default(&dflt);
    const mcrt_trace_opts* o = opts ? opts : &dflt;
    int rc = check_opts(sc, o, who);
    if (rc) return rc;
    if (cam->width < 1 || cam->height < 1 || (long long)cam->width * cam->height > (1ll << 31) - 1)
        return fail(ctx, MCRT_ERR_ARG, "%s: bad image size %d x %d", who, cam->width, cam->height);
    if (spp < 1) return fail(ctx, MCRT_ERR_ARG, "%s: spp must be >= 1", who);
    if (!(cam->fov_deg > 0.0f && cam->fov_deg < 180.0f)) return fail(ctx, MCRT_ERR_ARG, "%s: fov must be in (0, 180)", who);
    // camera frame (host, double, then float)
    double f[3], r[3], u[3];
    double n = 0;
    for (int a = 0; a < 3; ++a) { f[a] = (double)cam->target[a] - cam->pos[a]; n += f[a] * f[a]; }
    n = std::sqrt(n);
    if (!(n > 0)) return fail(ctx, MCRT_ERR_ARG, "%s: target equals position", who);
    for (int a = 0; a < 3; ++a) f[a] /= n;
    const double* up = nullptr;
    double upd[3] = {cam->up[0], cam->up[1], cam->up[2]};
    up = upd;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    n = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(n > 1e-12)) return fail(ctx, MCRT_ERR_ARG, "%s: up vector parallel to the view direction", who);
    for (int a = 0; a < 3; ++a) r[a] /= n;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    const int ncells = cam->width * cam->height;
    CK(ctx, cudaSetDevice(ctx->device));
    rc = ensure_leaf(sc, o->tau_merge, o->finest_level, o->grid);
    if (rc) return rc;
    rc = get_tally(ctx, ncells, 1, tally, who);
    if (rc) return rc;
    mcrt_tally* t = *tally;
    t->n_per_cell = spp;
    TraceParams P{};
    P.S = make_dev_scene(sc, 0.0f);
    P.total = (unsigned long long)ncells * spp;
    uint32_t chunk = o->chunk ? (uint32_t)o->chunk : 4u;
    if (chunk > spp) chunk = spp;
    while (spp % chunk) --chunk;   // a chunk never straddles two pixels
    P.chunk = chunk;
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    P.width = cam->width;
    P.height = cam->height;
    P.spp = spp;
    for (int a = 0; a < 3; ++a) {
        P.cam_pos[a] = cam->pos[a];
        P.cam_f[a] = (float)f[a];
        P.cam_r[a] = (float)r[a];
        P.cam_u[a] = (float)u[a];
    }
    P.tan_half = (float)std::tan(0.5 * cam->fov_deg * M_PI / 180.0);
    P.aspect = (float)cam->height / (float)cam->width;
    P.inv_width = 1.0f / (float)cam->width;
    P.inv_height = 1.0f / (float)cam->height;
    P.Lz = (float)sc->n[2] * sc->h[2];
    if (o->proposal) {
        P.deadline_ns = o->deadline_ms > 0.0 ? (unsigned long long)(o->deadline_ms * 1e6) : 0ull;
        P.cancel = reinterpret_cast<const volatile int*>(o->cancel_flag);
        P.max_order = o->max_order;
        P.sun_mode = o->sun_mode;
        P.max_steps = 1u << 22;
        set_rare_batch(P, o->rare_batch);
        P.s1 = t->d_s1; P.s2 = t->d_s2; P.counters = t->d_counters; P.work = static_cast<WorkState*>(t->d_work);
        return run_learned(sc, P, kCamera, o, t, spp, who);
    }
    uint32_t* d_order = nullptr;
    if (o->pixel_order == MCRT_ORDER_COST) {
        rc = make_claim_order(sc, P, &d_order, who);
        if (rc) return rc;
        P.pix_order = d_order;
    }
    if (o->schedule == MCRT_SCHEDULE_WAVEFRONT) {
        rc = run_wavefront(sc, P, o, t, who);
        dfree(ctx, d_order);
        return rc;
    }
    if (o->shard_count > 1) {
        // this shard's pixels: every shard_count-th position of the claim order
        const uint32_t nsh = (uint32_t)o->shard_count, idx = (uint32_t)o->shard_index, npix = (uint32_t)ncells;
        const uint32_t n_r = idx < npix ? (npix - idx + nsh - 1) / nsh : 0u;
        uint32_t* d_sh = nullptr;
        cudaError_t e = dalloc(ctx, &d_sh, (size_t)(n_r ? n_r : 1) * sizeof(uint32_t));
        if (e == cudaSuccess) {
            ctx->launches++;
            e = launch_shard_order(d_order, n_r, nsh, idx, d_sh, ctx->stream);
        }
        dfree(ctx, d_order);
        d_order = d_sh;
        if (e != cudaSuccess) {
            dfree(ctx, d_order);
            return fail(ctx, e == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA, "%s: shard order: %s", who,
                        cudaGetErrorString(e));
        }
        P.pix_order = d_order;
        P.total = (unsigned long long)n_r * spp;
    }
    rc = run_trace(sc, P, kCamera, o, t, who);
    dfree(ctx, d_order);
    return rc;
}

int mcrt_trace_flux(mcrt_scene* sc, uint64_t npaths, uint64_t seed, const mcrt_trace_opts* opts, mcrt_tally** tally)
{
    NvtxRange nvtx_range("mcrt_trace_flux");
    const char* who = "mcrt_trace_flux";
    if (!sc || !tally) return fail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = sc->ctx;
    ctx->err.clear();
    mcrt_trace_opts dflt;
    mcrt_trace_opts_default(&dflt);
    const mcrt_trace_opts* o = opts ? opts : &dflt;
    int rc = check_opts(sc, o, who);
    if (rc) return rc;
    if (o->schedule != MCRT_SCHEDULE_PERSISTENT)
        return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: the wavefront schedule traces camera images only", who);
    if (npaths < 1) return fail(ctx, MCRT_ERR_ARG, "%s: npaths must be >= 1", who);
    CK(ctx, cudaSetDevice(ctx->device));
    rc = ensure_leaf(sc, o->tau_merge, o->finest_level, o->grid);
    if (rc) return rc;
    rc = get_tally(ctx, 1, 3, tally, who);
    if (rc) return rc;
    mcrt_tally* t = *tally;
    t->n_per_cell = npaths;
    TraceParams P{};
    P.S = make_dev_scene(sc, 0.0f);
    P.total = npaths;
    P.chunk = o->chunk ? (uint32_t)o->chunk : 4u;
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    P.spp = 1;
    P.Lz = (float)sc->n[2] * sc->h[2];
    if (o->proposal) {
        P.deadline_ns = o->deadline_ms > 0.0 ? (unsigned long long)(o->deadline_ms * 1e6) : 0ull;
        P.cancel = reinterpret_cast<const volatile int*>(o->cancel_flag);
        P.max_order = o->max_order;
        P.sun_mode = o->sun_mode;
        P.max_steps = 1u << 22;
        set_rare_batch(P, o->rare_batch);
        P.s1 = t->d_s1; P.s2 = t->d_s2; P.counters = t->d_counters; P.work = static_cast<WorkState*>(t->d_work);
        return run_learned(sc, P, kFlux, o, t, 1ull, who);
    }
    if (o->shard_count > 1) {
        // this shard's path ids: [n i / c, n (i + 1) / c)
        const unsigned __int128 n = npaths;
        const unsigned long long b = (unsigned long long)(n * (unsigned)o->shard_index / (unsigned)o->shard_count);
        const unsigned long long e = (unsigned long long)(n * (unsigned)(o->shard_index + 1) / (unsigned)o->shard_count);
        P.path_base = b;
        P.total = e - b;
    }
    return run_trace(sc, P, kFlux, o, t, who);
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// Validates a batch and lays its items out for the kernel: chunk-aligned
// path-id ranges, one device scene per item (its field, its band's gas
// absorption, its sun) and its Philox key.
int prepare_batch(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n, const mcrt_trace_opts* o, const char* who,
                  std::vector<BatchItem>& h, unsigned long long& total, bool& bf16)
{
    if (n < 1 || n > (1 << 20)) return fail(ctx, MCRT_ERR_ARG, "%s: item count %d not in [1, 2^20]", who, n);
    if (o->proposal) return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: learned proposal in batches", who);
    if (o->shard_count > 1) return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: sharding in batches (items are the unit)", who);
    if (o->sun_mode == MCRT_SUN_DECOMP) return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: decomposition tracking in batches", who);
    if (o->schedule != MCRT_SCHEDULE_PERSISTENT)
        return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: the wavefront schedule traces camera images only", who);
    const uint32_t chunk = o->chunk ? (uint32_t)o->chunk : 4u;
    h.assign((size_t)n, BatchItem{});
    unsigned long long begin = 0;
    bf16 = false;
    CK(ctx, cudaSetDevice(ctx->device));
    for (int i = 0; i < n; ++i) {
        const mcrt_batch_item& it = items[i];
        if (!it.scene || it.scene->ctx != ctx) return fail(ctx, MCRT_ERR_ARG, "%s: item %d: bad scene", who, i);
        mcrt_scene* sc = const_cast<mcrt_scene*>(it.scene);
        int rc = check_opts(sc, o, who);
        if (rc) return rc;
        if (it.npaths < 1) return fail(ctx, MCRT_ERR_ARG, "%s: item %d: npaths must be >= 1", who, i);
        if (!(it.k_gas >= 0.0f) || !std::isfinite(it.k_gas))
            return fail(ctx, MCRT_ERR_ARG, "%s: item %d: k_gas must be finite and >= 0", who, i);
        if (!(it.sun_zenith_deg >= 0.0f && it.sun_zenith_deg < 90.0f) || !std::isfinite(it.sun_azimuth_deg))
            return fail(ctx, MCRT_ERR_ARG, "%s: item %d: sun zenith must be in [0, 90)", who, i);
        if (sc->d_hf) return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: item %d: heightfield ground in batches", who, i);
        if (sc->clear_phase == MCRT_PHASE_RAYLEIGH)
            return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: item %d: Rayleigh clear air in batches", who, i);
        if (i > 0 && (sc->storage == MCRT_STORAGE_BF16) != bf16)
            return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: items mix FP32 and BF16 storage", who);
        bf16 = sc->storage == MCRT_STORAGE_BF16;
        rc = ensure_leaf(sc, o->tau_merge, o->finest_level, o->grid);
        if (rc) return rc;
        h[i].S = make_dev_scene(sc, it.k_gas);
        const double z = it.sun_zenith_deg * M_PI / 180.0, a = it.sun_azimuth_deg * M_PI / 180.0;
        h[i].S.sun[0] = (float)(std::sin(z) * std::cos(a));
        h[i].S.sun[1] = (float)(std::sin(z) * std::sin(a));
        h[i].S.sun[2] = (float)std::cos(z);
        h[i].begin = begin;
        h[i].npaths = it.npaths;
        h[i].key = make_uint2((uint32_t)it.seed, (uint32_t)(it.seed >> 32));
        begin += (it.npaths + chunk - 1) / chunk * chunk;
    }
    total = begin;
    return MCRT_OK;
}

// Kernel parameters of a batch whose items and tally are on the device.
TraceParams batch_params(const std::vector<BatchItem>& h, const BatchItem* d_items, unsigned long long total,
                         const mcrt_trace_opts* o, mcrt_tally* t)
{
    TraceParams P{};
    P.S = h[0].S;
    P.items = d_items;
    P.n_items = (int)h.size();
    P.total = total;
    P.chunk = o->chunk ? (uint32_t)o->chunk : 4u;
    P.key = h[0].key;
    P.spp = 1;
    P.s1 = t->d_s1; P.s2 = t->d_s2; P.counters = t->d_counters; P.work = static_cast<WorkState*>(t->d_work);
    P.deadline_ns = o->deadline_ms > 0.0 ? (unsigned long long)(o->deadline_ms * 1e6) : 0ull;
    P.cancel = reinterpret_cast<const volatile int*>(o->cancel_flag);
    P.max_order = o->max_order;
    P.sun_mode = o->sun_mode;
    P.max_steps = 1u << 22;
    set_rare_batch(P, o->rare_batch);
    return P;
}

// A batch tally: n cells x 5 quantities with each cell's own path count.
int batch_tally(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n, mcrt_tally** tally, const char* who)
{
    int rc = get_tally(ctx, n, 5, tally, who);
    if (rc) return rc;
    mcrt_tally* t = *tally;
    t->n_per_cell = 0;
    t->cell_n.assign((size_t)n, 0);
    for (int i = 0; i < n; ++i) t->cell_n[i] = items[i].npaths;
    if (t->d_cell_n) dfree(ctx, t->d_cell_n);
    t->d_cell_n = nullptr;
    CK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&t->d_cell_n), sizeof(unsigned long long) * (size_t)n,
                            ctx->stream));
    CK(ctx, cudaMemcpyAsync(t->d_cell_n, t->cell_n.data(), sizeof(unsigned long long) * (size_t)n,
                            cudaMemcpyHostToDevice, ctx->stream));
    return MCRT_OK;
}

int batch_grid(mcrt_ctx* ctx, const mcrt_trace_opts* o, bool bf16, int* block)
{
    *block = o->block_size ? o->block_size : 128;
    return o->grid_size ? o->grid_size : ctx->sm_count * trace_batch_blocks_per_sm(bf16, o->count_events != 0, o->batch_dalpha != 0, *block);
}

}  // namespace

extern "C" {

int mcrt_trace_batch(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n, const mcrt_trace_opts* opts,
                     mcrt_tally** tally)
{
    NvtxRange nvtx_range("mcrt_trace_batch");
    const char* who = "mcrt_trace_batch";
    if (!ctx || !items || !tally) return fail(ctx, MCRT_ERR_ARG, "%s: NULL argument", who);
    ctx->err.clear();
    mcrt_trace_opts dflt;
    mcrt_trace_opts_default(&dflt);
    const mcrt_trace_opts* o = opts ? opts : &dflt;
    std::vector<BatchItem> h;
    unsigned long long total = 0;
    bool bf16 = false;
    int rc = prepare_batch(ctx, items, n, o, who, h, total, bf16);
    if (rc) return rc;
    rc = batch_tally(ctx, items, n, tally, who);
    if (rc) return rc;
    mcrt_tally* t = *tally;
    BatchItem* d_items = nullptr;
    CK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&d_items), sizeof(BatchItem) * (size_t)n, ctx->stream));
    cudaError_t e = cudaMemcpyAsync(d_items, h.data(), sizeof(BatchItem) * (size_t)n, cudaMemcpyHostToDevice,
                                    ctx->stream);
    const TraceParams P = batch_params(h, d_items, total, o, t);
    int block = 0;
    const int grid = batch_grid(ctx, o, bf16, &block);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    if (e == cudaSuccess) { ctx->launches++; e = launch_trace_batch(P, bf16, o->count_events != 0, o->batch_dalpha != 0, grid, block, ctx->stream); }
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    WorkState ws{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ws, t->d_work, sizeof(ws), cudaMemcpyDeviceToHost, ctx->stream);
    cudaFreeAsync(d_items, ctx->stream);
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(ctx, e);
    CK(ctx, se);
    t->kernel_ms = ms;
    if (ws.status == 1) return fail(ctx, MCRT_ERR_TIMEOUT, "%s: deadline of %g ms expired", who, o->deadline_ms);
    if (ws.status == 2) return fail(ctx, MCRT_ERR_CANCELLED, "%s: cancelled", who);
    return MCRT_OK;
}

int mcrt_autotune_batch(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n, double path_fraction,
                        mcrt_trace_opts* opts_inout, float* best_ms)
{
    NvtxRange nvtx_range("mcrt_autotune_batch");
    const char* who = "mcrt_autotune_batch";
    if (!ctx || !items || !opts_inout) return fail(ctx, MCRT_ERR_ARG, "%s: NULL argument", who);
    if (!(path_fraction > 0.0 && path_fraction <= 1.0)) return fail(ctx, MCRT_ERR_ARG, "%s: path_fraction in (0, 1]", who);
    if (n < 1) return fail(ctx, MCRT_ERR_ARG, "%s: no items", who);
    std::vector<mcrt_batch_item> sub(items, items + n);
    for (auto& it : sub) {
        it.npaths = (uint64_t)std::ceil((double)it.npaths * path_fraction);
        if (it.npaths < 1) it.npaths = 1;
    }
    // candidate launch shapes: paths per claim x lanes a rare phase waits for x block size
    const int chunks[] = {1, 2, 4, 8};
    const int rares[] = {4, 8, 12};
    const int blocks[] = {64, 128};
    mcrt_tally* t = nullptr;
    float best = 3.0e38f;
    mcrt_trace_opts bo = *opts_inout;
    for (int b : blocks)
        for (int c : chunks)
            for (int r : rares) {
                mcrt_trace_opts o = *opts_inout;
                o.chunk = c;
                o.rare_batch = r;
                o.block_size = b;
                o.grid_size = 0;
                for (int rep = 0; rep < 2; ++rep) {          // the better of two runs
                    int rc = mcrt_trace_batch(ctx, sub.data(), n, &o, &t);
                    if (rc) { if (t) mcrt_tally_destroy(t); return rc; }
                    if (t->kernel_ms < best) { best = t->kernel_ms; bo = o; }
                }
            }
    if (t) mcrt_tally_destroy(t);
    *opts_inout = bo;
    if (best_ms) *best_ms = best;
    return MCRT_OK;
}

// A batch captured once into a CUDA graph: tally reset, the persistent
// trace kernel, finalize and the copies of the results and the status to
// pinned host memory replay as one graph launch.
struct mcrt_batch_plan {
    mcrt_ctx* ctx = nullptr;
    mcrt_trace_opts opts{};
    std::vector<mcrt_batch_item> items;   // the caller's items (scenes borrowed)
    std::vector<uint64_t> gens;           // each item's scene state when its record was made
    unsigned long long total = 0;
    bool bf16 = false;
    std::vector<BatchItem> h;
    BatchItem* d_items = nullptr;
    mcrt_tally* t = nullptr;
    cudaStream_t st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* h_out = nullptr;       // pinned: (mean, se) per entry
    WorkState* h_ws = nullptr;     // pinned: the kernel's status
};

namespace {

void plan_free(mcrt_batch_plan* p)
{
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->e0) cudaEventDestroy(p->e0);
    if (p->e1) cudaEventDestroy(p->e1);
    if (p->h_out) cudaFreeHost(p->h_out);
    if (p->h_ws) cudaFreeHost(p->h_ws);
    if (p->t) mcrt_tally_destroy(p->t);
    if (p->d_items) cudaFree(p->d_items);
    if (p->st) cudaStreamDestroy(p->st);
    delete p;
}

}  // namespace

int mcrt_batch_plan_create(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n, const mcrt_trace_opts* opts,
                           mcrt_batch_plan** out)
{
    NvtxRange nvtx_range("mcrt_batch_plan_create");
    const char* who = "mcrt_batch_plan_create";
    if (!ctx || !items || !out) return fail(ctx, MCRT_ERR_ARG, "%s: NULL argument", who);
    *out = nullptr;
    ctx->err.clear();
    mcrt_trace_opts dflt;
    mcrt_trace_opts_default(&dflt);
    const mcrt_trace_opts* o = opts ? opts : &dflt;
    if (o->deadline_ms > 0.0 || o->cancel_flag)
        return fail(ctx, MCRT_ERR_UNSUPPORTED, "%s: deadline and cancel flag are for direct calls", who);
    mcrt_batch_plan* p = new (std::nothrow) mcrt_batch_plan();
    if (!p) return fail(ctx, MCRT_ERR_OOM, "%s: host allocation failed", who);
    p->ctx = ctx;
    p->opts = *o;
    unsigned long long total = 0;
    bool bf16 = false;
    int rc = prepare_batch(ctx, items, n, o, who, p->h, total, bf16);
    if (rc == MCRT_OK) rc = batch_tally(ctx, items, n, &p->t, who);
    if (rc) { plan_free(p); return rc; }
    p->items.assign(items, items + n);
    p->gens.resize((size_t)n);
    for (int i = 0; i < n; ++i) p->gens[i] = items[i].scene->gen;
    p->total = total;
    p->bf16 = bf16;
    const size_t m = (size_t)n * 5;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->d_items), sizeof(BatchItem) * (size_t)n);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_items, p->h.data(), sizeof(BatchItem) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&p->h_out), 2 * m * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&p->h_ws), sizeof(WorkState));
    if (e == cudaSuccess) e = cudaEventCreate(&p->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->e1);
    if (e != cudaSuccess) {
        plan_free(p);
        return fail(ctx, e == cudaErrorMemoryAllocation ? MCRT_ERR_OOM : MCRT_ERR_CUDA, "%s: %s", who,
                    cudaGetErrorString(e));
    }
    mcrt_tally* t = p->t;
    const TraceParams P = batch_params(p->h, p->d_items, total, o, t);
    int block = 0;
    const int grid = batch_grid(ctx, o, bf16, &block);
    e = cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t c = cudaMemsetAsync(t->d_s1, 0, m * sizeof(double), p->st);
        if (c == cudaSuccess) c = cudaMemsetAsync(t->d_s2, 0, m * sizeof(double), p->st);
        if (c == cudaSuccess) c = cudaMemsetAsync(t->d_counters, 0, kNumCounters * sizeof(unsigned long long), p->st);
        if (c == cudaSuccess) c = cudaMemsetAsync(t->d_work, 0, sizeof(WorkState), p->st);
        if (c == cudaSuccess) c = launch_trace_batch(P, bf16, o->count_events != 0, o->batch_dalpha != 0, grid, block, p->st);
        if (c == cudaSuccess) c = launch_finalize(t->d_s1, t->d_s2, 0.0, (int)m, t->d_cell_n, 5, t->d_out, p->st);
        if (c == cudaSuccess)
            c = cudaMemcpyAsync(p->h_out, t->d_out, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, p->st);
        if (c == cudaSuccess) c = cudaMemcpyAsync(p->h_ws, t->d_work, sizeof(WorkState), cudaMemcpyDeviceToHost, p->st);
        e = cudaStreamEndCapture(p->st, &p->graph);
        if (c != cudaSuccess) e = c;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        plan_free(p);
        return fail(ctx, MCRT_ERR_CUDA, "%s: graph capture: %s", who, cudaGetErrorString(e));
    }
    *out = p;
    return MCRT_OK;
}

int mcrt_batch_plan_set_seeds(mcrt_batch_plan* p, const uint64_t* seeds, int32_t n)
{
    if (!p || !seeds) return fail(p ? p->ctx : nullptr, MCRT_ERR_ARG, "mcrt_batch_plan_set_seeds: NULL argument");
    if (n != (int32_t)p->h.size())
        return fail(p->ctx, MCRT_ERR_ARG, "mcrt_batch_plan_set_seeds: %d seeds for %zu items", n, p->h.size());
    for (int i = 0; i < n; ++i) p->h[i].key = make_uint2((uint32_t)seeds[i], (uint32_t)(seeds[i] >> 32));
    CK(p->ctx, cudaSetDevice(p->ctx->device));
    CK(p->ctx, cudaStreamSynchronize(p->st));
    CK(p->ctx, cudaMemcpy(p->d_items, p->h.data(), sizeof(BatchItem) * p->h.size(), cudaMemcpyHostToDevice));
    return MCRT_OK;
}

int mcrt_batch_plan_run(mcrt_batch_plan* p, double* mean, double* se, size_t count, float* kernel_ms)
{
    NvtxRange nvtx_range("mcrt_batch_plan_run");
    const char* who = "mcrt_batch_plan_run";
    if (!p) return fail(nullptr, MCRT_ERR_ARG, "%s: NULL plan", who);
    mcrt_ctx* ctx = p->ctx;
    const size_t m = p->h.size() * 5;
    if ((mean || se) && count < m) return fail(ctx, MCRT_ERR_BOUNDS, "%s: need %zu entries", who, m);
    CK(ctx, cudaSetDevice(ctx->device));
    // the scenes may have changed since the records were made (another
    // tau~ or grid traced in between rebuilt a leaf map, the octree was
    // rebuilt elsewhere in memory, the ground changed): bring the leaf maps
    // back to the plan's options and, if any scene changed, remake and
    // upload the item records before the graph reads them
    bool stale = false;
    for (size_t i = 0; i < p->items.size(); ++i) {
        mcrt_scene* sc = const_cast<mcrt_scene*>(p->items[i].scene);
        int rc = ensure_leaf(sc, p->opts.tau_merge, p->opts.finest_level, p->opts.grid);
        if (rc) return rc;
        if (sc->gen != p->gens[i]) stale = true;
    }
    if (stale) {
        std::vector<BatchItem> hh;
        unsigned long long total = 0;
        bool bf16 = false;
        int rc = prepare_batch(ctx, p->items.data(), (int32_t)p->items.size(), &p->opts, who, hh, total, bf16);
        if (rc) return rc;
        if (total != p->total || bf16 != p->bf16) return fail(ctx, MCRT_ERR_STATE, "%s: the items changed shape", who);
        for (size_t i = 0; i < hh.size(); ++i) hh[i].key = p->h[i].key;     // seeds set on the plan
        CK(ctx, cudaStreamSynchronize(p->st));
        p->h.swap(hh);
        CK(ctx, cudaMemcpy(p->d_items, p->h.data(), sizeof(BatchItem) * p->h.size(), cudaMemcpyHostToDevice));
        for (size_t i = 0; i < p->items.size(); ++i) p->gens[i] = p->items[i].scene->gen;
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));      // work queued before the call (e.g. field uploads)
    ctx->launches += 2;                               // trace + finalize
    CK(ctx, cudaEventRecord(p->e0, p->st));
    CK(ctx, cudaGraphLaunch(p->exec, p->st));
    CK(ctx, cudaEventRecord(p->e1, p->st));
    CK(ctx, cudaStreamSynchronize(p->st));
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p->e0, p->e1) != cudaSuccess) ms = 0.0f;
    p->t->kernel_ms = ms;
    if (kernel_ms) *kernel_ms = ms;
    if (p->h_ws->status != 0) return fail(ctx, MCRT_ERR_CUDA, "mcrt_batch_plan_run: kernel status %d", p->h_ws->status);
    for (size_t i = 0; i < m; ++i) {
        if (mean) mean[i] = p->h_out[2 * i];
        if (se) se[i] = p->h_out[2 * i + 1];
    }
    return MCRT_OK;
}

int mcrt_batch_plan_tally(const mcrt_batch_plan* p, const mcrt_tally** tally)
{
    if (!p || !tally) return fail(p ? p->ctx : nullptr, MCRT_ERR_ARG, "mcrt_batch_plan_tally: NULL argument");
    *tally = p->t;
    return MCRT_OK;
}

int mcrt_batch_plan_destroy(mcrt_batch_plan* p)
{
    if (!p) return fail(nullptr, MCRT_ERR_ARG, "mcrt_batch_plan_destroy: NULL plan");
    cudaSetDevice(p->ctx->device);
    plan_free(p);
    return MCRT_OK;
}

// ---------------------------------------------------------------------------
// Tallies
// ---------------------------------------------------------------------------
int mcrt_tally_shape(const mcrt_tally* t, int32_t* ncells, int32_t* nquant)
{
    if (!t) return fail(nullptr, MCRT_ERR_ARG, "mcrt_tally_shape: NULL tally");
    if (ncells) *ncells = t->ncells;
    if (nquant) *nquant = t->nq;
    return MCRT_OK;
}

int mcrt_tally_read(const mcrt_tally* t, double* mean, double* se, uint64_t* n, size_t count)
{
    if (!t) return fail(nullptr, MCRT_ERR_ARG, "mcrt_tally_read: NULL tally");
    mcrt_ctx* ctx = t->ctx;
    const size_t m = (size_t)t->ncells * t->nq;
    if (count < m) return fail(ctx, MCRT_ERR_BOUNDS, "mcrt_tally_read: need %zu entries", m);
    CK(ctx, cudaSetDevice(ctx->device));
    if (mean || se) {
        LAUNCH(ctx, launch_finalize(t->d_s1, t->d_s2, (double)t->n_per_cell, (int)m,
                                    t->cell_n.empty() ? nullptr : t->d_cell_n, t->nq, t->d_out, ctx->stream));
        double* h = new (std::nothrow) double[2 * m];
        if (!h) return fail(ctx, MCRT_ERR_OOM, "mcrt_tally_read: host allocation failed");
        cudaError_t e = cudaMemcpyAsync(h, t->d_out, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            delete[] h;
            return fail(ctx, MCRT_ERR_CUDA, "mcrt_tally_read: %s", cudaGetErrorString(e));
        }
        for (size_t i = 0; i < m; ++i) {
            if (mean) mean[i] = h[2 * i];
            if (se) se[i] = h[2 * i + 1];
        }
        delete[] h;
    }
    if (n)
        for (size_t i = 0; i < m; ++i) n[i] = t->cell_n.empty() ? t->n_per_cell : t->cell_n[i / t->nq];
    return MCRT_OK;
}

int mcrt_tally_read_sums(const mcrt_tally* t, double* s1, double* s2, size_t count)
{
    if (!t) return fail(nullptr, MCRT_ERR_ARG, "mcrt_tally_read_sums: NULL tally");
    mcrt_ctx* ctx = t->ctx;
    const size_t m = (size_t)t->ncells * t->nq;
    if (count < m) return fail(ctx, MCRT_ERR_BOUNDS, "mcrt_tally_read_sums: need %zu entries", m);
    if (s1) CK(ctx, cudaMemcpyAsync(s1, t->d_s1, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (s2) CK(ctx, cudaMemcpyAsync(s2, t->d_s2, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

int mcrt_tally_counters(const mcrt_tally* t, uint64_t* c, size_t n)
{
    if (!t || !c) return fail(nullptr, MCRT_ERR_ARG, "mcrt_tally_counters: NULL argument");
    mcrt_ctx* ctx = t->ctx;
    if (n < 10) return fail(ctx, MCRT_ERR_BOUNDS, "mcrt_tally_counters: need at least 10 entries");
    unsigned long long h[kNumCounters];
    CK(ctx, cudaMemcpyAsync(h, t->d_counters, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < n && i < (size_t)kNumCounters; ++i) c[i] = h[i];
    return MCRT_OK;
}

int mcrt_tally_kernel_ms(const mcrt_tally* t, float* ms)
{
    if (!t || !ms) return fail(nullptr, MCRT_ERR_ARG, "mcrt_tally_kernel_ms: NULL argument");
    *ms = t->kernel_ms;
    return MCRT_OK;
}

int mcrt_tally_destroy(mcrt_tally* t)
{
    if (!t) return fail(nullptr, MCRT_ERR_ARG, "mcrt_tally_destroy: NULL tally");
    mcrt_ctx* ctx = t->ctx;
    dfree(ctx, t->d_s1);
    dfree(ctx, t->d_s2);
    dfree(ctx, t->d_counters);
    dfree(ctx, t->d_work);
    dfree(ctx, t->d_out);
    dfree(ctx, t->d_cell_n);
    cudaStreamSynchronize(ctx->stream);
    delete t;
    return MCRT_OK;
}

// ---------------------------------------------------------------------------
// Checks
// ---------------------------------------------------------------------------
int mcrt_debug_bounds_violations(mcrt_ctx* ctx, int32_t* checked_build, uint64_t* count, int32_t* first_code)
{
    if (!ctx || !checked_build || !count || !first_code)
        return fail(ctx, MCRT_ERR_ARG, "mcrt_debug_bounds_violations: NULL argument");
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    unsigned n = 0, code = 0;
    CK(ctx, read_bounds_violations(&n, &code));
    *checked_build = bounds_checked_build() ? 1 : 0;
    *count = n;
    *first_code = (int32_t)code;
    return MCRT_OK;
}

int mcrt_debug_learned_records(mcrt_scene* sc, const mcrt_camera_desc* cam, uint64_t n, uint64_t seed,
                               const mcrt_trace_opts* opts, int32_t cap, float* feat, float* dir, float* val,
                               uint64_t* path, int32_t* count)
{
    const char* who = "mcrt_debug_learned_records";
    if (!sc || !opts || !count || cap < 0 || (cap > 0 && (!feat || !dir || !val || !path)))
        return fail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = sc->ctx;
    if (!opts->proposal) return fail(ctx, MCRT_ERR_ARG, "%s: opts->proposal is NULL", who);
    const unsigned long long paths = cam ? n * (unsigned long long)(cam->width > 0 ? cam->width : 0) *
                                               (unsigned long long)(cam->height > 0 ? cam->height : 0)
                                         : n;
    if (paths > (1ull << 24)) return fail(ctx, MCRT_ERR_BOUNDS, "%s: at most 2^24 paths", who);
    if (cam && n > 0xFFFFFFFFull) return fail(ctx, MCRT_ERR_ARG, "%s: spp too large", who);
    RecordDump d;
    d.cap = cap; d.feat = feat; d.dir = dir; d.val = val; d.path = path;
    mcrt_trace_opts o = *opts;
    o.learn = 0;
    mcrt_tally* t = nullptr;
    ctx->rec_dump = &d;
    int rc = cam ? mcrt_trace_camera(sc, cam, (uint32_t)n, seed, &o, &t) : mcrt_trace_flux(sc, n, seed, &o, &t);
    ctx->rec_dump = nullptr;
    if (t) mcrt_tally_destroy(t);
    *count = d.count;
    return rc;
}

int mcrt_debug_pool_usage(mcrt_ctx* ctx, int32_t reset_high, uint64_t* used_current, uint64_t* used_high)
{
    if (!ctx || !used_current || !used_high) return fail(ctx, MCRT_ERR_ARG, "mcrt_debug_pool_usage: NULL argument");
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    cudaMemPool_t pool;
    CK(ctx, cudaDeviceGetMemPool(&pool, ctx->device));
    unsigned long long cur = 0, high = 0;
    CK(ctx, cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &cur));
    CK(ctx, cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
    if (reset_high) {
        unsigned long long zero = 0;
        CK(ctx, cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    *used_current = (uint64_t)cur;
    *used_high = (uint64_t)high;
    return MCRT_OK;
}

int mcrt_debug_dda(const mcrt_scene* sc_c, const float o[3], const float d[3], float tau, int32_t finest,
                   int32_t* cells, float* tio, int32_t cap, int32_t* count, int32_t* status)
{
    return mcrt_debug_dda_grid(sc_c, o, d, tau, finest, MCRT_GRID_PYRAMID, cells, tio, cap, count, status);
}

int mcrt_debug_dda_grid(const mcrt_scene* sc_c, const float o[3], const float d[3], float tau, int32_t finest,
                        int32_t grid, int32_t* cells, float* tio, int32_t cap, int32_t* count, int32_t* status)
{
    mcrt_scene* sc = const_cast<mcrt_scene*>(sc_c);
    if (!sc || !o || !d || !cells || !tio || !count || !status)
        return fail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "mcrt_debug_dda: NULL argument");
    mcrt_ctx* ctx = sc->ctx;
    if (cap < 1) return fail(ctx, MCRT_ERR_ARG, "mcrt_debug_dda: cap must be >= 1");
    mcrt_trace_opts op;
    mcrt_trace_opts_default(&op);
    op.tau_merge = tau;
    op.finest_level = finest;
    op.grid = grid;
    int rc = check_opts(sc, &op, "mcrt_debug_dda");
    if (rc) return rc;
    const float n2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(n2 > 0.0f) || !std::isfinite(n2)) return fail(ctx, MCRT_ERR_ARG, "mcrt_debug_dda: bad direction");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(o[a])) return fail(ctx, MCRT_ERR_ARG, "mcrt_debug_dda: bad origin");
    CK(ctx, cudaSetDevice(ctx->device));
    rc = ensure_leaf(sc, tau, finest, grid);
    if (rc) return rc;
    int* dcells = nullptr;
    float* dtio = nullptr;
    int* dcs = nullptr;
    CK(ctx, dalloc(ctx, &dcells, (size_t)cap * 4 * sizeof(int)));
    CK(ctx, dalloc(ctx, &dtio, (size_t)cap * 2 * sizeof(float)));
    CK(ctx, dalloc(ctx, &dcs, 2 * sizeof(int)));
    ctx->launches++;
    cudaError_t e = launch_debug_dda(make_dev_scene(sc, 0.0f), o, d, cap, dcells, dtio, dcs,
                                     sc->storage == MCRT_STORAGE_BF16, ctx->stream);
    int cs[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(cs, dcs, sizeof(cs), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && cs[0] > 0) {
        e = cudaMemcpyAsync(cells, dcells, (size_t)cs[0] * 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tio, dtio, (size_t)cs[0] * 2 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    dfree(ctx, dcells);
    dfree(ctx, dtio);
    dfree(ctx, dcs);
    CK(ctx, e);
    *count = cs[0];
    *status = cs[1];
    return MCRT_OK;
}

int mcrt_debug_terrain(const mcrt_scene* sc, int32_t n, const float* o, const float* d, float* t_out)
{
    const char* who = "mcrt_debug_terrain";
    if (!sc || (n > 0 && (!o || !d || !t_out))) return fail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = sc->ctx;
    if (!sc->d_hf) return fail(ctx, MCRT_ERR_STATE, "%s: the scene has a flat ground", who);
    if (n < 0 || n > (1 << 24)) return fail(ctx, MCRT_ERR_ARG, "%s: bad ray count %d", who, n);
    if (n == 0) return MCRT_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    float* buf = nullptr;
    CK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&buf), (size_t)n * 7 * sizeof(float), ctx->stream));
    cudaError_t e = cudaMemcpyAsync(buf, o, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf + 3 * (size_t)n, d, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        ctx->launches++;
        e = launch_debug_terrain(make_dev_scene(sc, 0.0f), buf, buf + 3 * (size_t)n, n, buf + 6 * (size_t)n, ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t_out, buf + 6 * (size_t)n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    cudaFreeAsync(buf, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    CK(ctx, e);
    return MCRT_OK;
}

int mcrt_debug_terrain_height(const mcrt_scene* sc, int32_t n, const float* xy, float* zn_out)
{
    const char* who = "mcrt_debug_terrain_height";
    if (!sc || (n > 0 && (!xy || !zn_out))) return fail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = sc->ctx;
    if (!sc->d_hf) return fail(ctx, MCRT_ERR_STATE, "%s: the scene has a flat ground", who);
    if (n < 0 || n > (1 << 24)) return fail(ctx, MCRT_ERR_ARG, "%s: bad point count %d", who, n);
    if (n == 0) return MCRT_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    float* buf = nullptr;
    CK(ctx, cudaMallocAsync(reinterpret_cast<void**>(&buf), (size_t)n * 6 * sizeof(float), ctx->stream));
    cudaError_t e = cudaMemcpyAsync(buf, xy, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        ctx->launches++;
        e = launch_debug_terrain_height(make_dev_scene(sc, 0.0f), buf, n, buf + 2 * (size_t)n, ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(zn_out, buf + 2 * (size_t)n, (size_t)n * 4 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    cudaFreeAsync(buf, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    CK(ctx, e);
    return MCRT_OK;
}

int mcrt_debug_philox(mcrt_ctx* ctx, const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n)
{
    if (!ctx || !ctr || !key || !out) return fail(ctx, MCRT_ERR_ARG, "mcrt_debug_philox: NULL argument");
    if (n == 0) return MCRT_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    CK(ctx, dalloc(ctx, &dc, n * 16));
    CK(ctx, dalloc(ctx, &dk, n * 8));
    CK(ctx, dalloc(ctx, &dout, n * 16));
    cudaError_t e = cudaMemcpyAsync(dc, ctr, n * 16, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dk, key, n * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        ctx->launches++;
        e = launch_debug_philox(dc, dk, dout, n, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, n * 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, dc);
    dfree(ctx, dk);
    dfree(ctx, dout);
    CK(ctx, e);
    return MCRT_OK;
}

}  // extern "C"
