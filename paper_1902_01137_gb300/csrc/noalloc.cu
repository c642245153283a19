// noalloc.cu -- a camera trace that performs no device allocation.
//
// Some callers cannot allocate GPU memory while they trace: code that runs
// inside another framework's memory budget, real-time loops that must not
// touch the allocator, or hosts whose allocator is owned by someone else.
// mcrt_trace_camera allocates its tally on first use; this entry point
// instead keeps the tracer's working memory (the work counter, the status
// word and the FP64 per-pixel sums) in one statically sized device array
// that lives as long as the library is loaded, and writes the per-pixel mean
// and standard error into buffers the caller already owns.
//
// Limits and rules:
//  * Images up to kNoAllocMaxPixels pixels (256 x 256); larger images are
//    rejected with MCRT_ERR_BOUNDS before any GPU work.
//  * Every GPU that loads the library holds the array (about 1 MiB) until
//    the process exits.
//  * All calls share the one array.  Each call clears the parts it uses
//    before tracing, but two calls whose GPU work overlaps (different
//    streams, or different host threads on one device) race on it: issue
//    these calls one after another on one stream.
//  * The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress); make that first call before capturing any
//    stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "mcrt_internal.h"

using namespace mcrt;

namespace {

constexpr int kNoAllocMaxPixels = 256 * 256;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    WorkState work;
    unsigned long long counters[kNumCounters];
    double s1[kNoAllocMaxPixels];
    double s2[kNoAllocMaxPixels];
};

// The working memory of every no-allocation call on this device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device (the host-side symbol is
// only a stand-in and must never be handed to a kernel).
std::mutex g_mu;
NoAllocScratch* g_addr[kMaxDevices] = {};

int nfail(mcrt_ctx* ctx, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

// Mean and standard error straight from the static sums into the caller's
// device buffers; NaN in both when the trace stopped early (deadline or
// cancel flag), whose partial sums estimate nothing.
__global__ void noalloc_finalize_kernel(double n, int count, double* __restrict__ mean, double* __restrict__ se)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (g_noalloc_scratch.work.status != 0) {
        mean[i] = __longlong_as_double(0x7ff8000000000000ll);
        se[i] = mean[i];
        return;
    }
    const double m = g_noalloc_scratch.s1[i] / n;
    double var = g_noalloc_scratch.s2[i] / n - m * m;
    if (var < 0.0) var = 0.0;
    mean[i] = m;
    se[i] = n > 1.0 ? sqrt(var / (n - 1.0)) : 0.0;
}

}  // namespace

extern "C" int mcrt_trace_camera_noalloc(mcrt_scene* sc, const mcrt_camera_desc* cam, uint32_t spp, uint64_t seed,
                                         const mcrt_trace_opts* opts, double* d_mean, double* d_stderr)
{
    NvtxRange nvtx_range("mcrt_trace_camera_noalloc");
    const char* who = "mcrt_trace_camera_noalloc";
    if (!sc || !cam || !d_mean || !d_stderr) return nfail(sc ? sc->ctx : nullptr, MCRT_ERR_ARG, "%s: NULL argument", who);
    mcrt_ctx* ctx = sc->ctx;
    ctx->err.clear();
    mcrt_trace_opts dflt;
    mcrt_trace_opts_default(&dflt);
    const mcrt_trace_opts* o = opts ? opts : &dflt;
    int rc = check_opts(sc, o, who);
    if (rc != MCRT_OK) return rc;
    if (o->schedule != MCRT_SCHEDULE_PERSISTENT)
        return nfail(ctx, MCRT_ERR_UNSUPPORTED, "%s: the wavefront schedule allocates its queues", who);
    if (cam->width < 1 || cam->height < 1)
        return nfail(ctx, MCRT_ERR_ARG, "%s: bad image size %d x %d", who, cam->width, cam->height);
    if ((long long)cam->width * cam->height > kNoAllocMaxPixels)
        return nfail(ctx, MCRT_ERR_BOUNDS, "%s: %d x %d pixels exceed the %d-pixel static working area", who,
                     cam->width, cam->height, kNoAllocMaxPixels);
    if (spp < 1) return nfail(ctx, MCRT_ERR_ARG, "%s: spp must be >= 1", who);
    if (!(cam->fov_deg > 0.0f && cam->fov_deg < 180.0f)) return nfail(ctx, MCRT_ERR_ARG, "%s: fov must be in (0, 180)", who);
    if (o->proposal) return nfail(ctx, MCRT_ERR_UNSUPPORTED, "%s: the learned proposal needs work buffers", who);
    if (o->shard_count > 1) return nfail(ctx, MCRT_ERR_UNSUPPORTED, "%s: a shard needs its own claim order", who);
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return nfail(ctx, MCRT_ERR_ARG, "%s: device index too large", who);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return nfail(ctx, MCRT_ERR_CUDA, "%s: cudaSetDevice: %s", who, cudaGetErrorString(e));

    // one-time lookup of the array's device address on this device
    NoAllocScratch* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[ctx->device]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return nfail(ctx, MCRT_ERR_CUDA, "%s: cudaGetSymbolAddress: %s", who, cudaGetErrorString(e));
            g_addr[ctx->device] = static_cast<NoAllocScratch*>(p);
        }
        scratch = g_addr[ctx->device];
    }

    // camera frame
    double f[3], r[3], u[3], n = 0;
    for (int a = 0; a < 3; ++a) { f[a] = (double)cam->target[a] - cam->pos[a]; n += f[a] * f[a]; }
    n = std::sqrt(n);
    if (!(n > 0)) return nfail(ctx, MCRT_ERR_ARG, "%s: target equals position", who);
    for (int a = 0; a < 3; ++a) f[a] /= n;
    r[0] = f[1] * cam->up[2] - f[2] * cam->up[1];
    r[1] = f[2] * cam->up[0] - f[0] * cam->up[2];
    r[2] = f[0] * cam->up[1] - f[1] * cam->up[0];
    n = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(n > 1e-12)) return nfail(ctx, MCRT_ERR_ARG, "%s: up vector parallel to the view direction", who);
    for (int a = 0; a < 3; ++a) r[a] /= n;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];

    // the leaf map of this (tau~, finest level, grid); rebuilt in place, no allocation
    rc = ensure_leaf(sc, o->tau_merge, o->finest_level, o->grid);
    if (rc != MCRT_OK) return rc;

    // clear what must start at zero: the work state, counters and the sums
    const int npix = cam->width * cam->height;
    e = cudaMemsetAsync(&scratch->work, 0, sizeof(WorkState) + sizeof(scratch->counters), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch->s1, 0, (size_t)npix * sizeof(double), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch->s2, 0, (size_t)npix * sizeof(double), ctx->stream);
    if (e != cudaSuccess) return nfail(ctx, MCRT_ERR_CUDA, "%s: clearing the working area: %s", who, cudaGetErrorString(e));

    TraceParams P{};
    P.S = make_dev_scene(sc, 0.0f);
    P.total = (unsigned long long)npix * spp;
    uint32_t chunk = o->chunk ? (uint32_t)o->chunk : 4u;
    if (chunk > spp) chunk = spp;
    while (spp % chunk) --chunk;
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
    P.s1 = scratch->s1;
    P.s2 = scratch->s2;
    P.counters = scratch->counters;
    P.work = &scratch->work;
    P.deadline_ns = o->deadline_ms > 0.0 ? (unsigned long long)(o->deadline_ms * 1e6) : 0ull;
    P.cancel = reinterpret_cast<const volatile int*>(o->cancel_flag);
    P.max_order = o->max_order;
    P.sun_mode = o->sun_mode;
    P.max_steps = 1u << 22;
    set_rare_batch(P, o->rare_batch);
    const bool bf16 = sc->storage == MCRT_STORAGE_BF16;
    const bool count = o->count_events != 0;
    const int block = o->block_size ? o->block_size : 128;
    const int grid = o->grid_size ? o->grid_size : ctx->sm_count * trace_blocks_per_sm(kCamera, bf16, count, P.S.hf != nullptr, P.sun_mode == MCRT_SUN_DECOMP || P.S.rayleigh, block);
    if (!o->chunk) P.chunk = auto_chunk(P.total, (unsigned long long)grid * block, spp);
    ctx->launches++;
    e = launch_trace(P, kCamera, bf16, count, grid, block, ctx->stream);
    if (e != cudaSuccess) return nfail(ctx, MCRT_ERR_CUDA, "%s: trace launch: %s", who, cudaGetErrorString(e));
    ctx->launches++;
    noalloc_finalize_kernel<<<(npix + 255) / 256, 256, 0, ctx->stream>>>((double)spp, npix, d_mean, d_stderr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(ctx, MCRT_ERR_CUDA, "%s: finalize launch: %s", who, cudaGetErrorString(e));
    WorkState ws{};
    e = cudaMemcpyAsync(&ws, &scratch->work, sizeof(ws), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return nfail(ctx, MCRT_ERR_CUDA, "%s: %s", who, cudaGetErrorString(e));
    if (ws.status == 1) return nfail(ctx, MCRT_ERR_TIMEOUT, "%s: deadline of %g ms expired", who, o->deadline_ms);
    if (ws.status == 2) return nfail(ctx, MCRT_ERR_CANCELLED, "%s: cancelled", who);
    return MCRT_OK;
}
