// trace.cu -- persistent path-tracing kernel (sm_103a).
//
// One GPU thread carries one path at a time; its state (traversal, weights,
// the two Philox draw sequences) lives in registers.  Every loop iteration
// advances each live lane by exactly one traversal step -- either one leaf
// crossed or one tentative collision handled -- whatever ray it is on (the
// path's free flight or a sun ray), so all lanes of a warp run the same code
// and divergence is limited to the short event-handling branches.  Lanes
// whose chunk of paths is done are refilled at the top of the loop: the warp
// ballots its idle lanes and claims new path ids for all of them with one
// atomic (work stays balanced to the last paths).
//
// Physics (Villefranque et al. 2019):
//   free flight: null-collision sampling over leaves of uniform majorant M
//     (Sec. 2.3 steps 4a-4g, Eq. 2; Sec. 2.4 piecewise-uniform majorant):
//     optical depth -ln u is spent leaf by leaf; at a tentative collision the
//     true k is read and the collision is real with probability k / M.
//   local estimate (Sec. 4.1): at each real collision or ground hit the path
//     scores w * phase-or-BRDF toward the sun * T_sun, T_sun by ratio tracking
//     (t *= 1 - k/M, Russian roulette below 0.1) or delta tracking.
//   events: HG scattering with weight omega, Lambertian ground with weight
//     albedo, Russian roulette below w = 0.01; escape at the top.
// Random numbers: path id p, event e: stream (e, 0) for the flight (block 0
// word 0 its first optical depth -- the camera's first flight takes word 2
// of the path-start block instead -- and block j its j-th tentative
// collision); (e, 1) for the vertex ending that flight and its sun ray
// (block 0: two direction draws, roulette and, in word 3, the sun ray's
// first optical depth; block j the sun ray's j-th tentative collision);
// (0, 2) for the camera jitter / ground point; (0, 3) for the direct sun ray
// of a flux path.  A learned vertex draws from blocks kBlockVertex and
// kBlockVertex - 1 of stream (e, 0) (word 1 of the latter: its sun ray's
// first optical depth), a Rayleigh vertex its species from word 0 of block
// kBlockVertex.
//
// Loop structure (one iteration): flush finished chunks and claim new ones
// (convergent); one Philox block per lane; one phase of work per lane (path
// start, traversal step, vertex, ray start -- a camera path start or a
// vertex, learned or not, goes on into the ray start it sets up, whose first
// optical depth is a word of the block already drawn); one 8-byte load (the
// voxel of a tentative collision or the leaf-map entry of the leaf entered);
// the leaf set-up; the end of a ray or path.
#include <cuda_bf16.h>

#include "mcrt_internal.h"

#ifndef MCRT_TRACE_MIN_BLOCKS
#define MCRT_TRACE_MIN_BLOCKS 7   // resident blocks of 128 threads the register budget must allow (72 registers)
#endif

namespace mcrt {

namespace {

constexpr unsigned kFull = 0xffffffffu;

enum Kind { kMain = 0, kSunLocal = 1, kSunDirect = 2 };
enum Event { EV_NONE = 0, EV_REAL, EV_GROUND, EV_ESCAPE, EV_SUN_END, EV_ABORT };

// Counter slots (see mcrt_tally_counters).
enum {
    C_PATHS = 0, C_TENT = 1, C_REAL = 2, C_GROUND = 3, C_LEAF = 4,
    C_SUN_TENT = 5, C_SUN_LEAF = 6, C_SUN_RAYS = 7, C_ABORT = 8, C_FLIGHTS = 9
};
constexpr int kCounters = 10;
// Extra slots filled with atomicMax in counting mode: [10] most loop
// iterations spent on one path, [11] longest time (ns) a warp ran before the
// work queue ran dry, [12] longest time (ns) a warp ran in total.
enum { C_MAX_ITERS = 10, C_T_DRY = 11, C_T_END = 12 };
// Counting mode also records, per warp, the SM clock cycles spent in each
// section of the loop body (slots 13..21): loop top, Philox, path start,
// ray start, step, vertex, load, after-load, ray/path end.
constexpr int C_SEC = 13;
constexpr int kSections = 9;
// ... and, per warp iteration, lane occupancy (slots 22..29): iterations,
// lanes holding a path, stepping, at a tentative collision, running a rare
// phase, waiting for one, iterations that ran rare phases, lanes without a path.
constexpr int C_OCC = 22;
constexpr int kOcc = 8;

// Each lane is in one phase per iteration: it starts a path, starts a ray
// (flight or sun ray), takes one traversal step, or handles the vertex that
// ended a flight.  Every lane evaluates one Philox block per iteration at
// one site, whose counter depends on the phase (a camera path start or a
// vertex that continues into its ray start takes that ray's first optical
// depth from a word of it); the voxel / leaf-entry load and the leaf set-up
// also run at one site each.
enum Phase { PH_IDLE = 0, PH_START, PH_BEGIN, PH_STEP, PH_VERTEX, PH_RESUME, PH_TERRAIN };

// EXTRA: the variants that also handle decomposition tracking of sun rays
// and Rayleigh clear air (chosen at run time); the others carry neither, so
// the paper's estimator keeps its registers.  In batches, EXTRA instead
// adds the dT/dalpha estimate.
template <int SENSOR, bool BF16, bool COUNT, bool LEARNED, bool BATCH = false, bool TERRAIN = false,
          bool EXTRA = false>
__global__ void __launch_bounds__(128, MCRT_TRACE_MIN_BLOCKS) trace_kernel(const __grid_constant__ TraceParams P)
{
    // quantities per path: camera radiance; flux T_dir, T_dif, T_tot (+ dT/dg, dT/dalpha in batches)
    constexpr int NQ = (SENSOR == kCamera) ? 1 : (BATCH ? 5 : 3);
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    // ---- per-lane state ------------------------------------------------------
    unsigned long long pid = 0, pend = 0;   // current path, end of the lane's chunk
    bool chunk = false;                     // the lane holds a chunk
    bool exhausted = false;                 // warp-uniform: nothing left to claim
    int phase = PH_IDLE;
    unsigned cell = 0;                      // tally cell of the chunk
    int px = 0, py = 0;                     // camera pixel of the chunk
    // chunk sums of x and x^2 in FP32 (a chunk is at most 8 paths: relative
    // error below 7 * 2^-24 of the sum of |x| before the FP64 atomic add)
    float acc[2 * NQ];
#pragma unroll
    for (int q = 0; q < 2 * NQ; ++q) acc[q] = 0.0f;
    Ray R;
    int kind = kMain;
    uint32_t c2 = 0, blk = 1, ev = 0;
    float tau = 0.0f, Ts = 1.0f, w = 1.0f, score = 0.0f, cf = 0.0f, tdir = 0.0f;
    bool term_after = false, vground = false;
    float vk = 0.0f;                        // extinction at the vertex
    uint32_t lv = 0;                        // volume vertices so far (learned mode)
    uint32_t cur_rec = 0xFFFFFFFFu;         // training record awaiting its own estimate
    bool suspend = false;                   // stop this path until the network has run
    float tg = __int_as_float(0x7f800000);  // heightfield: distance of the flight's ground hit from R.o
    float tpend = __int_as_float(0x7f800000);   // heightfield: where the flight enters the relief layer (walk pending)
    float fz = 1.0f;                        // heightfield flux: n_z of the surface at the path start
    float vx[3] = {0.0f, 0.0f, 0.0f}, nd[3] = {0.0f, 0.0f, 1.0f};
    unsigned long long cnt[kCounters];
#pragma unroll
    for (int q = 0; q < kCounters; ++q) cnt[q] = 0;
    uint32_t path_iters = 0, max_iters = 0;
    unsigned long long sec[kSections];
#pragma unroll
    for (int q = 0; q < kSections; ++q) sec[q] = 0;
    unsigned long long occ[kOcc];
#pragma unroll
    for (int q = 0; q < kOcc; ++q) occ[q] = 0;
    long long tclk = COUNT ? clock64() : 0;
    auto mark = [&](int q) {
        if (COUNT) {
            __syncwarp();
            const long long now = clock64();
            sec[q] += (unsigned long long)(now - tclk);
            tclk = now;
        }
    };
    int item = 0;                           // batch item of the lane's chunk
    uint2 rkey = P.key;                     // Philox key of that item
    float sg = 0.0f, sv_pending = 0.0f, cfs = 0.0f, dscore = 0.0f;   // d/dg (batches)
    float sa = 0.0f, dal = 0.0f;            // d/dalpha, the droplets' absorptivity (batches)
    uint64_t t_start = 0, t_dry = 0;
    if (P.deadline_ns || COUNT) t_start = globaltimer_ns();
    uint32_t iter = 0;

    for (;;) {
        // ---- flush finished chunks: lanes sharing a cell are summed first --
        bool pending = chunk && phase == PH_IDLE;
        if (pending) chunk = false;
        unsigned fmask = __ballot_sync(kFull, pending);
        while (fmask) {
            const int src = __ffs(fmask) - 1;
            const unsigned c = __shfl_sync(kFull, cell, src);
            MCRT_CHECK(c < (SENSOR == kCamera ? (unsigned)(P.width * P.height) : (BATCH ? (unsigned)P.n_items : 1u)), 3);
            const bool mine = pending && cell == c;
#pragma unroll
            for (int q = 0; q < 2 * NQ; ++q) {
                double a = mine ? (double)acc[q] : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
                if (lane == src) atomicAdd(((q & 1) ? P.s2 : P.s1) + (size_t)c * NQ + (q >> 1), a);
            }
            if (mine) {
                pending = false;
#pragma unroll
                for (int q = 0; q < 2 * NQ; ++q) acc[q] = 0.0f;
            }
            fmask = __ballot_sync(kFull, pending);
        }
        // ---- claim chunks for idle lanes (one atomic per warp) -------------
        const unsigned idle = __ballot_sync(kFull, !chunk);
        if (idle && !exhausted) {
            const int nidle = __popc(idle);
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&P.work->next, (unsigned long long)nidle * P.chunk);
            base = __shfl_sync(kFull, base, leader);
            if (base + (unsigned long long)nidle * P.chunk >= P.total) {
                exhausted = true;
                if (COUNT) t_dry = globaltimer_ns();
            }
            if (!chunk) {
                pid = base + (unsigned long long)__popc(idle & lt_mask) * P.chunk;
                if (pid < P.total) {
                    pend = min(pid + (unsigned long long)P.chunk, P.total);
                    chunk = true;
                    phase = (LEARNED && P.resume) ? PH_RESUME : PH_START;
                    // the batch (learned mode) or shard (flux) this launch traces
                    if (!BATCH && !(LEARNED && P.resume)) { pid += P.path_base; pend += P.path_base; }
                    if constexpr (BATCH) {
                        // items own chunk-aligned id ranges: find the item, use its local ids
                        int lo = 0, hi = P.n_items - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (P.items[mid].begin <= pid) lo = mid;
                            else hi = mid - 1;
                        }
                        item = lo;
                        const unsigned long long b = P.items[lo].begin, np = P.items[lo].npaths;
                        pid -= b;
                        pend = min(pend - b, np);
                        rkey = P.items[lo].key;
                        if (pid >= np) { chunk = false; phase = PH_IDLE; }
                    }
                    if constexpr (SENSOR == kCamera) {
                        unsigned long long pix = pid / P.spp;
                        if (!LEARNED && P.pix_order) {
                            // claims walk the pixels in the given order (costly
                            // ones first); a path keeps its id, so its draws and
                            // its result do not depend on the order
                            const unsigned long long off = pid - pix * P.spp;
                            pix = __ldg(P.pix_order + pix);
                            pid = pix * P.spp + off;
                            pend = pid + P.chunk;          // a chunk never straddles two pixels
                        }
                        cell = (unsigned)pix;
                        px = (int)(pix % (unsigned long long)P.width);
                        py = (int)(pix / (unsigned long long)P.width);
                    } else {
                        cell = BATCH ? (unsigned)item : 0u;
                    }
                }
            }
        }
        if (!__any_sync(kFull, chunk)) break;
        // ---- deadline / cancel, every 1024 iterations ------------------------
        if ((++iter & 1023u) == 0 && (P.deadline_ns || P.cancel)) {
            int stop = 0;
            if (lane == 0) {
                if (P.cancel && *P.cancel) stop = 2;
                else if (P.deadline_ns && globaltimer_ns() - t_start > P.deadline_ns) stop = 1;
                const int others = *reinterpret_cast<volatile int*>(&P.work->status);
                if (others) stop = others;
            }
            stop = __shfl_sync(kFull, stop, 0);
            if (stop) {
                if (lane == 0) atomicMax(&P.work->status, stop);
                break;
            }
        }
        if (COUNT && phase != PH_IDLE) ++path_iters;
        if (COUNT) { __syncwarp(); tclk = clock64(); }

        // ---- rare phases (path start, ray start, vertex) run in batches: a
        //      lane waits until enough lanes of its warp need one, or until
        //      few lanes are stepping ------------------------------------------
        // (heightfield: a flight whose current leaf reaches down into the relief
        //  layer first finds its ground hit, a rare phase of its own)
        if (TERRAIN && phase == PH_STEP && R.texit >= tpend) phase = PH_TERRAIN;
        const bool rare = phase == PH_START || phase == PH_BEGIN || phase == PH_VERTEX || phase == PH_RESUME ||
                          (TERRAIN && phase == PH_TERRAIN);
        const unsigned rare_mask = __ballot_sync(kFull, rare);
        const unsigned step_mask = __ballot_sync(kFull, phase == PH_STEP);
        const bool run_rare = __popc(rare_mask) >= P.rare_batch || __popc(step_mask) < P.min_steppers;
        // every rare kind runs in the same iteration: path starts and
        // vertices (learned ones resumed too) go on into their ray start, and
        // ground walks start there as well, so the ray-start and walk
        // branches execute once with all their lanes
        const int ph = (phase == PH_STEP || (rare && run_rare)) ? phase : PH_IDLE;

        // ---- the scene of the lane's chunk (one per batch item) ---------------
        const DevScene& S = BATCH ? P.items[item].S : P.S;

        // ---- the one Philox block of this iteration ---------------------------
        const float seg = (TERRAIN ? fminf(R.texit, tg) : R.texit) - R.t;
        // tracking majorant: the leaf's M, or M - m for a sun ray in
        // decomposition tracking (the minorant m is applied exactly)
        const bool decomp = EXTRA && kind != kMain && P.sun_mode == MCRT_SUN_DECOMP;
        const float Mt = decomp ? R.M - R.mn : R.M;
        const float Mseg = Mt * seg;
        const bool tent = ph == PH_STEP && Mt > 0.0f && tau < Mseg;
        if (COUNT) {
            const unsigned busy = __ballot_sync(kFull, chunk), tm = __ballot_sync(kFull, tent);
            const unsigned rr = __ballot_sync(kFull, rare && ph != PH_IDLE);
            occ[0] += 1; occ[1] += __popc(busy); occ[2] += __popc(step_mask); occ[3] += __popc(tm);
            occ[4] += __popc(rr); occ[5] += __popc(rare_mask) - __popc(rr); occ[6] += rr ? 1 : 0;
            occ[7] += 32 - __popc(busy);
        }
        uint32_t xc2 = c2, xblk = 0u;
        if (ph == PH_START) xc2 = 2u;
        else if (ph == PH_STEP) xblk = blk;
        else if (ph == PH_VERTEX) { xc2 = (ev << 2) | 1u; xblk = 0u; }   // the sun ray's block 0
        mark(0);
        const uint4 x = draw_block(pid, xc2, xblk, rkey);
        mark(1);

        // ---- phase work before the load ---------------------------------------
        int evc = EV_NONE;
        float p[3];
        int nv[3] = {0, 0, 0};
        const uint2* ptr = nullptr;
        uint32_t sub = 0;
        int st = kInside;
        bool setup = false;          // enter a leaf after the load
        bool walk = false;           // heightfield: find this ray's ground hit now
        bool merge = false;          // a path start or vertex whose ray starts in this iteration too
        uint32_t mword = 0u;         // ... the word giving that ray's first optical depth
        if (ph == PH_START) {
            w = 1.0f; score = 0.0f; ev = 0; tdir = 0.0f; term_after = false;
            if (BATCH) { sg = 0.0f; sv_pending = 0.0f; cfs = 0.0f; dscore = 0.0f; sa = 0.0f; dal = 0.0f; }
            if (COUNT) path_iters = 0;
            if constexpr (SENSOR == kCamera) {
                const float jx = 1.0f - u01(x.x), jy = 1.0f - u01(x.y);
                const float sx = (2.0f * ((float)px + jx) * P.inv_width - 1.0f) * P.tan_half;
                const float sy = (2.0f * ((float)py + jy) * P.inv_height - 1.0f) * P.tan_half * P.aspect;
                float d[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) d[a] = P.cam_f[a] + sx * P.cam_r[a] + sy * P.cam_u[a];
                const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                float q[3] = {P.cam_pos[0], P.cam_pos[1], P.cam_pos[2]};
#pragma unroll
                for (int a = 0; a < 3; ++a) d[a] *= inv;
                bool enters = true;
                if (q[2] > P.Lz) {
                    if (d[2] < 0.0f) {
                        const float t = __fdividef(P.Lz - q[2], d[2]);
                        q[0] += t * d[0];
                        q[1] += t * d[1];
                        q[2] = P.Lz;
                    } else {
                        enters = false;
                    }
                } else if (q[2] < 0.0f) {
                    enters = false;
                }
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    q[a] -= floorf(__fdividef(q[a], S.Lper[a])) * S.Lper[a];
                    if (!(q[a] < S.Lper[a]) || q[a] < 0.0f) q[a] = 0.0f;
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) { vx[a] = q[a]; nd[a] = d[a]; }
                kind = kMain;
                c2 = 0u;
                if (enters) { phase = PH_BEGIN; merge = true; mword = x.z; }
                else evc = EV_ESCAPE;          // a path that misses the field scores 0
            } else {
                vx[0] = (1.0f - u01(x.x)) * S.Lper[0];
                vx[1] = (1.0f - u01(x.y)) * S.Lper[1];
                vx[2] = 0.0f;
                if (!(vx[0] < S.Lper[0])) vx[0] = 0.0f;
                if (!(vx[1] < S.Lper[1])) vx[1] = 0.0f;
                kind = kSunDirect;
                c2 = 3u;
                Ts = 1.0f;
                phase = PH_BEGIN;      // (its four words used up: the ray starts next time)
                if constexpr (TERRAIN) {
                    // the surface point above (x, y), lifted along its normal;
                    // directions cosine-weighted about the normal; the direct
                    // irradiance of the tilted element per horizontal area is
                    // max(n.s, 0) / (n_z mu0) T_sun, kept in tdir until T_sun
                    float n[3];
                    vx[2] = hf_height(S, vx[0], vx[1], n);
#pragma unroll
                    for (int a = 0; a < 3; ++a) vx[a] += kTerrainOffset * n[a];
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        if (vx[a] < 0.0f) vx[a] += S.Lper[a];
                        if (!(vx[a] < S.Lper[a])) vx[a] -= S.Lper[a];
                        if (!(vx[a] >= 0.0f && vx[a] < S.Lper[a])) vx[a] = 0.0f;
                    }
                    cosine_about(n, u01(x.z), u01(x.w), nd);
                    fz = n[2];
                    const float ns = n[0] * S.sun[0] + n[1] * S.sun[1] + n[2] * S.sun[2];
                    tdir = __fdividef(fmaxf(ns, 0.0f), n[2] * S.sun[2]);
                    if (!(ns > 0.0f)) { kind = kMain; c2 = 0u; }     // self-shadowed: no direct sun ray
                } else {
                    cosine_up(u01(x.z), u01(x.w), nd);
                }
            }
        }
        mark(2);
        if (ph == PH_VERTEX) {
            // weight, estimate factor toward the sun, new direction, roulette
            const float xi1 = u01(x.x), xi2 = u01(x.y), xr = u01(x.z);
            const int order = (int)ev + 1;
            const bool score_it = (P.max_order == 0) || (order <= P.max_order);
            if (!vground) {
                const float om = omega_at(S, vk);
                const float mu = R.d[0] * S.sun[0] + R.d[1] * S.sun[1] + R.d[2] * S.sun[2];
                float ph = hg_pdf(S.g, mu);
                float mu_new;
                if (EXTRA && S.rayleigh) {
                    // Rayleigh clear air: the mixture phase function in the estimate;
                    // the species sampled with word 0 of the flight's vertex block
                    const float pc = cloud_scatter_share(S, vk);
                    ph = pc * ph + (1.0f - pc) * rayleigh_pdf(mu);
                    const uint4 xs = draw_block(pid, ev << 2, kBlockVertex, rkey);
                    mu_new = u01(xs.x) > pc ? rayleigh_sample_mu(xi1) : hg_sample_mu(S.g, xi1);
                } else {
                    mu_new = hg_sample_mu(S.g, xi1);
                }
                cf = score_it ? w * om * ph : 0.0f;
                w *= om;
                rotate_dir(R.d, mu_new, xi2, nd);
                if (BATCH) {
                    cfs = hg_dlog_dg(S.g, mu);
                    sv_pending = hg_dlog_dg(S.g, mu_new);
                    // d ln omega / d alpha = -k_cloud / (k omega) at this vertex
                    if (EXTRA && om > 0.0f) sa -= __fdividef(fmaxf(vk - S.k_gas - S.k_clear, 0.0f), vk * om);
                }
                if (COUNT) cnt[C_REAL]++;
            } else if constexpr (TERRAIN) {
                // tilted ground: leave the surface along its normal, estimate
                // with n.s, scatter cosine-weighted about n
                float n[3];
                hf_height(S, vx[0], vx[1], n);
#pragma unroll
                for (int a = 0; a < 3; ++a) vx[a] += kTerrainOffset * n[a];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    if (vx[a] < 0.0f) vx[a] += S.Lper[a];
                    if (!(vx[a] < S.Lper[a])) vx[a] -= S.Lper[a];
                    if (!(vx[a] >= 0.0f && vx[a] < S.Lper[a])) vx[a] = 0.0f;
                }
                const float ns = n[0] * S.sun[0] + n[1] * S.sun[1] + n[2] * S.sun[2];
                cf = (score_it && ns > 0.0f) ? w * (S.albedo * (1.0f / kPi)) * ns : 0.0f;
                w *= S.albedo;
                cosine_about(n, xi1, xi2, nd);
                if (COUNT) cnt[C_GROUND]++;
            } else {
                cf = score_it ? w * (S.albedo * (1.0f / kPi)) * fmaxf(S.sun[2], 0.0f) : 0.0f;
                w *= S.albedo;
                cosine_up(xi1, xi2, nd);
                if (BATCH) { cfs = 0.0f; sv_pending = 0.0f; }
                if (COUNT) cnt[C_GROUND]++;
            }
            term_after = (P.max_order > 0) && (order >= P.max_order);
            if (!term_after && w < 0.01f) {
                if (xr * 0.01f <= w) w = 0.01f;
                else term_after = true;
            }
            // (a ground facet turned away from the sun sends no sun ray)
            if (score_it && (!TERRAIN || !vground || cf > 0.0f)) {
                kind = kSunLocal;
                c2 = (ev << 2) | 1u;
                Ts = 1.0f;
                phase = PH_BEGIN;
                merge = true;
                mword = x.w;     // word 3 of the vertex block
            } else {
                Ts = 0.0f;
                evc = EV_SUN_END;
            }
        }

        if (LEARNED && ph == PH_RESUME) {
            // resume a path stopped at a learned vertex: state, network output,
            // one-sample MIS direction, weight p_HG / q
            const uint32_t slot = (uint32_t)pid;
            const uint4 q0 = P.qin[4 * (size_t)slot], q1 = P.qin[4 * (size_t)slot + 1];
            const uint4 q2 = P.qin[4 * (size_t)slot + 2], q3 = P.qin[4 * (size_t)slot + 3];
            pid = (unsigned long long)q0.x | ((unsigned long long)q0.y << 32);
            pend = pid + 1;
            ev = q0.z;
            lv = q0.w;
            vx[0] = __uint_as_float(q1.x); vx[1] = __uint_as_float(q1.y); vx[2] = __uint_as_float(q1.z);
            vk = __uint_as_float(q1.w);
            R.d[0] = __uint_as_float(q2.x); R.d[1] = __uint_as_float(q2.y); R.d[2] = __uint_as_float(q2.z);
            w = __uint_as_float(q2.w);
            score = __uint_as_float(q3.x);
            tdir = __uint_as_float(q3.y);
            term_after = false;
            if constexpr (SENSOR == kCamera) cell = (unsigned)(pid / P.spp);
            kind = kMain;
            c2 = ev << 2;
            const uint4 xv = draw_block(pid, ev << 2, kBlockVertex, P.key);
            const uint4 xl = draw_block(pid, ev << 2, kBlockVertex - 1u, P.key);
            const float xi1 = u01(xv.x), xi2 = u01(xv.y), xr = u01(xv.z), xc = u01(xv.w), xlobe = u01(xl.x);
            const int order = (int)ev + 1;
            const bool score_it = (P.max_order == 0) || (order <= P.max_order);
            const float om = omega_at(S, vk);
            const float mu_s = R.d[0] * S.sun[0] + R.d[1] * S.sun[1] + R.d[2] * S.sun[2];
            cf = score_it ? w * om * hg_pdf(S.g, mu_s) : 0.0f;
            const float* mix = P.qin_mix + 48 * (size_t)slot;
            if (xc <= P.mis_alpha) {
                rotate_dir(R.d, hg_sample_mu(S.g, xi1), xi2, nd);
            } else {
                int j = 7;
#pragma unroll
                for (int i = 0; i < 7; ++i)
                    if (j == 7 && xlobe <= __ldg(mix + 6 * i + 4)) j = i;
                const float mu_l[3] = {__ldg(mix + 6 * j), __ldg(mix + 6 * j + 1), __ldg(mix + 6 * j + 2)};
                const float kap = __ldg(mix + 6 * j + 3);
                float cw = 1.0f + __logf(xi1 + (1.0f - xi1) * __expf(-2.0f * kap)) / kap;
                cw = fminf(fmaxf(cw, -1.0f), 1.0f);
                rotate_dir(mu_l, cw, xi2, nd);
            }
            const float phg = hg_pdf(S.g, R.d[0] * nd[0] + R.d[1] * nd[1] + R.d[2] * nd[2]);
            // mixture density: sum of pi_j C(kappa_j) exp(kappa_j (mu_j . w - 1))
            float qv = 0.0f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float c = __ldg(mix + 6 * i) * nd[0] + __ldg(mix + 6 * i + 1) * nd[1] + __ldg(mix + 6 * i + 2) * nd[2];
                qv += __ldg(mix + 6 * i + 5) * __expf(__ldg(mix + 6 * i + 3) * (c - 1.0f));
            }
            const float qmix = P.mis_alpha * phg + (1.0f - P.mis_alpha) * qv;
            // training record: features, direction, score so far, w * omega
            if (P.rec_count && slot < P.rec_slots) {
                const unsigned idx = atomicAdd(P.rec_count, 1u);
                if (idx < P.rec_cap) {
                    P.rec_feat[2 * (size_t)idx] = P.qin_feat[2 * (size_t)slot];
                    P.rec_feat[2 * (size_t)idx + 1] = P.qin_feat[2 * (size_t)slot + 1];
                    P.rec_dir[3 * (size_t)idx] = nd[0];
                    P.rec_dir[3 * (size_t)idx + 1] = nd[1];
                    P.rec_dir[3 * (size_t)idx + 2] = nd[2];
                    P.rec_val[4 * (size_t)idx] = score;
                    P.rec_val[4 * (size_t)idx + 1] = w * om;
                    P.rec_val[4 * (size_t)idx + 2] = 0.0f;
                    P.rec_val[4 * (size_t)idx + 3] = __uint_as_float((uint32_t)(pid - P.path_base));
                    cur_rec = idx;
                }
            }
            w *= om * __fdividef(phg, fmaxf(qmix, 1e-30f));
            ++lv;
            if (COUNT) cnt[C_REAL]++;
            term_after = (P.max_order > 0) && (order >= P.max_order);
            if (!term_after && w < 0.01f) {
                if (xr * 0.01f <= w) w = 0.01f;
                else term_after = true;
            }
            if (score_it) {
                kind = kSunLocal;
                c2 = (ev << 2) | 1u;
                Ts = 1.0f;
                phase = PH_BEGIN;
                merge = true;
                mword = xl.y;    // word 1 of the lobe block
            } else {
                Ts = 0.0f;
                evc = EV_SUN_END;
            }
        }
        mark(5);
        // a lane whose camera path start, vertex or resumed vertex set up a
        // ray starts it now, so it skips one rare iteration and its wait;
        // the ray's first optical depth comes from a word of the block that
        // set it up (a flux path start uses all four words of its block, so
        // its direct sun ray starts in a later iteration, from its own block)
        const uint32_t tw = merge ? mword : x.x;
        if (ph == PH_BEGIN || merge) {
            // start a ray: the flight from vx along nd, or the sun ray from vx
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float d = (kind == kMain) ? nd[a] : S.sun[a];
                R.o[a] = vx[a];
                R.d[a] = d;
                R.inv_d[a] = (d != 0.0f) ? __frcp_rn(d) : 0.0f;
                R.v[a] = locate(vx[a], d, S.h[a], S.inv_h[a], 0, S.n[a] - 1);
            }
            R.t = 0.0f;
            R.steps = 0;
            ptr = leaf_entry(S, R.v);
            setup = true;
            tau = -__logf(u01(tw));
            blk = 1;
            if constexpr (TERRAIN) {
                // a sun ray that meets the surface is shadowed (found now: sun rays
                // only start inside the relief layer at the ground or below hmax);
                // a flight ends at the surface, found now when it starts inside the
                // relief layer, else once its traversal reaches z = hmax
                tg = __int_as_float(0x7f800000);
                tpend = __int_as_float(0x7f800000);
                if (kind == kMain && R.o[2] > S.hmax) {
                    if (R.d[2] < 0.0f) tpend = __fdiv_rn(S.hmax - R.o[2], R.d[2]);
                } else {
                    walk = true;
                }
            }
            if (COUNT) {
                if (kind == kMain) cnt[C_FLIGHTS]++;
                else cnt[C_SUN_RAYS]++;
            }
        }
        if (TERRAIN && ph == PH_TERRAIN) {
            walk = true;
            tpend = __int_as_float(0x7f800000);
            phase = PH_STEP;
        }
        if (TERRAIN && walk) {
            const float th = terrain_hit(S, R.o, R.d);
            if (kind == kMain) {
                tg = th;
            } else if (th < __int_as_float(0x7f800000)) {
                Ts = 0.0f;
                evc = EV_SUN_END;
                ptr = nullptr;
                setup = false;
            }
        }
        mark(3);
        if (ph == PH_STEP) {
            // one step: to the tentative collision inside the leaf, or across
            // the leaf's exit face; both share the point and voxel arithmetic
            const bool at_ground = TERRAIN && !tent && tg <= R.texit;   // the surface cuts this leaf
            const float tn = tent ? fminf(R.t + __fdividef(tau, Mt), TERRAIN ? fminf(R.texit, tg) : R.texit)
                                  : (at_ground ? tg : R.texit);
            if (decomp) Ts *= __expf(-R.mn * (tn - R.t));   // the control over this piece of the leaf
            advance(S, R, tn, !tent && !at_ground, p, nv);
            if (at_ground) {
                // ground vertex at the surface hit (x, y wrapped into the domain)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    if (p[a] < 0.0f) p[a] += S.Lper[a];
                    if (!(p[a] < S.Lper[a])) p[a] -= S.Lper[a];
                    if (!(p[a] >= 0.0f && p[a] < S.Lper[a])) p[a] = 0.0f;
                }
                vx[0] = p[0]; vx[1] = p[1]; vx[2] = fmaxf(p[2], 0.0f);
                vground = true;
                phase = PH_VERTEX;
            } else if (tent) {
                R.t = tn;
                // a voxel leaf's majorant is the voxel itself: its tentative
                // collision needs no load (k = M, so it is real; a sun ray's
                // ratio 1 - k/M is 0)
                if (R.lev != 0) {
                    const size_t idx = brick_index(S, nv[0], nv[1], nv[2]);
                    if (BF16) { ptr = reinterpret_cast<const uint2*>(S.vox16) + (idx >> 2); sub = (uint32_t)idx & 3u; }
                    else { ptr = reinterpret_cast<const uint2*>(S.vox) + (idx >> 1); sub = (uint32_t)idx & 1u; }
                }
            } else {
                tau -= Mseg;
                float wdt;
                st = cross_face(S, R, p, nv, &wdt);
                if (TERRAIN) { tg -= wdt; tpend -= wdt; }   // a periodic wrap restarts the segment
                if (st == kInside && decomp && Ts < 0.1f) {
                    // roulette at a leaf crossing: word 3 of the next block, which it uses up
                    if (u01(x.w) * 0.1f <= Ts) Ts = 0.1f;
                    else { Ts = 0.0f; evc = EV_SUN_END; }
                    ++blk;
                }
                if (st == kInside && evc == EV_NONE) {
                    ptr = leaf_entry(S, R.v);
                    setup = true;
                    if (COUNT) {
                        if (kind == kMain) cnt[C_LEAF]++;
                        else cnt[C_SUN_LEAF]++;
                    }
                } else if (st == kTop) {
                    evc = (kind == kMain) ? EV_ESCAPE : EV_SUN_END;
                } else {
                    if (kind == kMain) {
                        // ground hit: the vertex is handled in a later iteration
                        p[2] = 0.0f;
                        p[0] = fminf(fmaxf(p[0], 0.0f), S.Lper[0]);
                        p[1] = fminf(fmaxf(p[1], 0.0f), S.Lper[1]);
                        if (!(p[0] < S.Lper[0])) p[0] = 0.0f;
                        if (!(p[1] < S.Lper[1])) p[1] = 0.0f;
                        vx[0] = p[0]; vx[1] = p[1]; vx[2] = p[2];
                        vground = true;
                        phase = PH_VERTEX;
                    } else {
                        Ts = 0.0f;
                        evc = EV_SUN_END;
                    }
                }
            }
        }
        mark(4);
        // ---- the one load: voxel word or leaf-map entry ---------------------
        uint2 val = make_uint2(0u, 0u);
        if (ptr) val = __ldg(ptr);
        if (COUNT) asm volatile("" ::"r"(val.x), "r"(val.y));   // charge the load latency here
        mark(6);

        // ---- after the load ----------------------------------------------------
        if (setup) {
            finish_leaf<BF16>(S, R, val);
            if (ph == PH_BEGIN || merge) phase = PH_STEP;
            else if (R.steps > P.max_steps) evc = EV_ABORT;
        } else if (tent) {
            float kv;
            if (BF16) {
                const uint32_t wd = (sub & 2u) ? val.y : val.x;
                kv = __uint_as_float(((wd >> ((sub & 1u) * 16u)) & 0xFFFFu) << 16);
            } else {
                kv = __uint_as_float(sub ? val.y : val.x);
            }
            const float k = R.lev == 0 ? R.M : __fadd_rn(kv, S.k_gas);
            ++blk;
            const float u0 = u01(x.x);
            const float nt = -__logf(u01(x.y));
            if (kind == kMain) {
                if (COUNT) cnt[C_TENT]++;
                if (u0 * R.M <= k) {
                    vx[0] = p[0]; vx[1] = p[1]; vx[2] = p[2];
                    vk = k;
                    vground = false;
                    phase = PH_VERTEX;
                    if (LEARNED && lv < (uint32_t)P.n_learned) suspend = true;
                } else {
                    tau = nt;
                }
            } else {
                if (COUNT) cnt[C_SUN_TENT]++;
                bool ended = false;
                if (P.sun_mode == MCRT_SUN_DELTA) {
                    if (u0 * R.M <= k) { Ts = 0.0f; ended = true; }
                } else {
                    if (EXTRA && P.sun_mode == MCRT_SUN_DECOMP) Ts *= 1.0f - __fdividef(k - R.mn, R.M - R.mn);
                    else Ts *= 1.0f - __fdividef(k, R.M);
                    if (!(Ts > 0.0f)) { Ts = 0.0f; ended = true; }
                    else if (Ts < 0.1f) {
                        if (u0 * 0.1f <= Ts) Ts = 0.1f;
                        else { Ts = 0.0f; ended = true; }
                    }
                }
                if (ended) evc = EV_SUN_END;
                else tau = nt;
            }
        }

        mark(7);
        // ---- end of a ray or of the path -------------------------------------
        if (evc != EV_NONE) {
            bool path_done = false;
            if (evc == EV_ABORT) {
                if (COUNT) cnt[C_ABORT]++;
                if (kind == kMain) path_done = true;
                else { Ts = 0.0f; evc = EV_SUN_END; }
            }
            if (evc == EV_SUN_END) {
                if (kind == kSunDirect) {
                    tdir = TERRAIN ? tdir * Ts : Ts;
                    ev = 0;
                    kind = kMain;
                    c2 = 0u;
                    phase = PH_BEGIN;
                } else {
                    score += cf * Ts;
                    if (BATCH) {
                        dscore += cf * Ts * (sg + cfs);
                        if (EXTRA) dal += cf * Ts * sa;
                        sg += sv_pending;
                    }
                    if (LEARNED && cur_rec != 0xFFFFFFFFu) {
                        P.rec_val[4 * (size_t)cur_rec + 2] = cf * Ts;
                        cur_rec = 0xFFFFFFFFu;
                    }
                    if (term_after) {
                        path_done = true;
                    } else {
                        ++ev;
                        kind = kMain;
                        c2 = ev << 2;
                        phase = PH_BEGIN;
                    }
                }
            }
            if (evc == EV_ESCAPE) path_done = true;
            if (path_done) {
                if constexpr (SENSOR == kCamera) {
                    acc[0] += score;
                    acc[1] += score * score;
                } else {
                    const float pi_over_mu0 = __fdividef(kPi, TERRAIN ? fz * S.sun[2] : S.sun[2]);
                    const float tf = pi_over_mu0 * score;
                    const float tt = tdir + tf;
                    acc[0] += tdir; acc[1] += tdir * tdir;
                    acc[2] += tf; acc[3] += tf * tf;
                    acc[4] += tt; acc[5] += tt * tt;
                    if constexpr (BATCH) {
                        const float dt = pi_over_mu0 * dscore;
                        acc[6] += dt; acc[7] += dt * dt;
                        if (EXTRA) {
                            const float da = pi_over_mu0 * dal;
                            acc[8] += da; acc[9] += da * da;
                        }
                    }
                }
                if (COUNT) {
                    cnt[C_PATHS]++;
                    max_iters = max(max_iters, path_iters);
                }
                if (LEARNED && P.final_score) P.final_score[pid - P.path_base] = score;
                ++pid;
                phase = (pid < pend) ? PH_START : PH_IDLE;
            }
        }
        // ---- stop paths at a learned vertex: state and features to the queue
        if (LEARNED) {
            const unsigned smask = __ballot_sync(kFull, suspend);
            if (smask) {
                const int leader = __ffs(smask) - 1;
                unsigned base = 0;
                if (lane == leader) base = atomicAdd(P.qout_count, (unsigned)__popc(smask));
                base = __shfl_sync(kFull, base, leader);
                if (suspend) {
                    const unsigned slot = base + (unsigned)__popc(smask & lt_mask);
                    if (slot < P.qout_cap) {
                        // features: position in [-1, 1], incoming direction, ln(k), ln(M1), ln(M2)
                        const float Lz = (float)S.n[2] * S.h[2];
                        float f[9];
                        f[0] = 2.0f * vx[0] / S.Lper[0] - 1.0f;
                        f[1] = 2.0f * vx[1] / S.Lper[1] - 1.0f;
                        f[2] = 2.0f * vx[2] / Lz - 1.0f;
                        f[3] = R.d[0]; f[4] = R.d[1]; f[5] = R.d[2];
                        f[6] = logf(vk + 1e-6f);
                        const float M1 = __ldg(P.pyr1 + ((size_t)(nv[2] >> 3) * P.d1[1] + (nv[1] >> 3)) * P.d1[0] +
                                               (nv[0] >> 3));
                        const int s2 = 3 * P.lev2;
                        const float M2 = __ldg(P.pyr2 + ((size_t)(nv[2] >> s2) * P.d2[1] + (nv[1] >> s2)) * P.d2[0] +
                                               (nv[0] >> s2));
                        f[7] = logf(M1 + S.k_gas + 1e-6f);
                        f[8] = logf(M2 + S.k_gas + 1e-6f);
                        uint32_t pk[8];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const __nv_bfloat162 v = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
                            pk[i] = *reinterpret_cast<const uint32_t*>(&v);
                        }
                        pk[4] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f[8]));
                        pk[5] = pk[6] = pk[7] = 0u;
                        P.qout_feat[2 * (size_t)slot] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        P.qout_feat[2 * (size_t)slot + 1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        P.qout[4 * (size_t)slot] = make_uint4((uint32_t)pid, (uint32_t)(pid >> 32), ev, lv);
                        P.qout[4 * (size_t)slot + 1] = make_uint4(__float_as_uint(vx[0]), __float_as_uint(vx[1]),
                                                                  __float_as_uint(vx[2]), __float_as_uint(vk));
                        P.qout[4 * (size_t)slot + 2] = make_uint4(__float_as_uint(R.d[0]), __float_as_uint(R.d[1]),
                                                                  __float_as_uint(R.d[2]), __float_as_uint(w));
                        P.qout[4 * (size_t)slot + 3] = make_uint4(__float_as_uint(score), __float_as_uint(tdir), 0u, 0u);
                    }
                    suspend = false;
                    ++pid;
                    phase = (pid < pend) ? PH_START : PH_IDLE;
                }
            }
        }
        mark(8);
    }

    // ---- partial sums left by a deadline / cancel exit ------------------------
    if (chunk) {
#pragma unroll
        for (int q = 0; q < 2 * NQ; ++q)
            if (acc[q] != 0.0f) atomicAdd(((q & 1) ? P.s2 : P.s1) + (size_t)cell * NQ + (q >> 1), (double)acc[q]);
    }
    if (COUNT) {
#pragma unroll
        for (int q = 0; q < kCounters; ++q) {
            unsigned long long a = cnt[q];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
            if (lane == 0 && a) atomicAdd(P.counters + q, a);
        }
        unsigned mi = max_iters;
        for (int o = 16; o > 0; o >>= 1) mi = max(mi, __shfl_xor_sync(kFull, mi, o));
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < kSections; ++q) atomicAdd(P.counters + C_SEC + q, sec[q]);
#pragma unroll
            for (int q = 0; q < kOcc; ++q) atomicAdd(P.counters + C_OCC + q, occ[q]);
            const uint64_t t_end = globaltimer_ns();
            atomicMax(P.counters + C_MAX_ITERS, (unsigned long long)mi);
            if (t_dry) atomicMax(P.counters + C_T_DRY, (unsigned long long)(t_dry - t_start));
            atomicMax(P.counters + C_T_END, (unsigned long long)(t_end - t_start));
        }
    }
}

// Mean and standard error of each tally entry from its FP64 sums; a batch
// passes each cell's own path count (cell_n, nq entries per cell).
__global__ void finalize_kernel(const double* __restrict__ s1, const double* __restrict__ s2, double n_all, int count,
                                const unsigned long long* __restrict__ cell_n, int nq, double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double n = cell_n ? (double)cell_n[i / nq] : n_all;
    const double m = s1[i] / n;
    double var = s2[i] / n - m * m;
    if (var < 0.0) var = 0.0;
    out[2 * i] = m;
    out[2 * i + 1] = n > 1.0 ? sqrt(var / (n - 1.0)) : 0.0;
}

// One thread walks one ray and records its leaves (traversal check), with
// the same device functions as the tracer.
template <bool BF16>
__global__ void debug_dda_kernel(DevScene S, float ox, float oy, float oz, float dx, float dy, float dz, int cap,
                                 int* cells, float* tio, int* count_status)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    Ray R;
    const float p0[3] = {ox, oy, oz}, d[3] = {dx, dy, dz};
    ray_begin<BF16>(S, R, p0, d);
    float tbase = 0.0f;
    int n = 0, status = 0;
    for (;;) {
        if (n >= cap) { status = 3; break; }
        cells[4 * n + 0] = R.lev / S.lb;      // level of the tracked grid
        cells[4 * n + 1] = R.v[0] >> R.lev;
        cells[4 * n + 2] = R.v[1] >> R.lev;
        cells[4 * n + 3] = R.v[2] >> R.lev;
        tio[2 * n + 0] = __fadd_rn(tbase, R.t);
        tio[2 * n + 1] = __fadd_rn(tbase, R.texit);
        ++n;
        float wdt, p[3];
        const int st = step_face(S, R, p, &wdt);
        if (wdt != 0.0f) tbase = __fadd_rn(tbase, wdt);
        if (st == kTop) { status = 1; break; }
        if (st == kGround) { status = 2; break; }
        finish_leaf<BF16>(S, R, __ldg(leaf_entry(S, R.v)));
        if (R.steps > (1u << 22)) { status = 4; break; }
    }
    count_status[0] = n;
    count_status[1] = status;
}

// Claim order of a camera trace: the cost of each tile of kOrderTile^2
// pixels is estimated by the majorant optical depth along the view ray
// through the tile's centre (the sum of M times the length over the leaves
// it crosses, capped): paths that enter thick cloud scatter many times and
// run longest.  Tracing the costly tiles first leaves cheap paths for the
// end of the launch, where a long path would otherwise run alone.
constexpr int kOrderTile = 8;

template <bool BF16>
__global__ void view_cost_kernel(TraceParams P, int tiles_x, int tiles_y, float* __restrict__ cost)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tiles_x * tiles_y) return;
    const DevScene& S = P.S;
    const float cx = fminf((float)((i % tiles_x) * kOrderTile) + 0.5f * kOrderTile, (float)P.width - 0.5f);
    const float cy = fminf((float)((i / tiles_x) * kOrderTile) + 0.5f * kOrderTile, (float)P.height - 0.5f);
    const float sx = (2.0f * cx * P.inv_width - 1.0f) * P.tan_half;
    const float sy = (2.0f * cy * P.inv_height - 1.0f) * P.tan_half * P.aspect;
    float d[3], q[3] = {P.cam_pos[0], P.cam_pos[1], P.cam_pos[2]};
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = P.cam_f[a] + sx * P.cam_r[a] + sy * P.cam_u[a];
    const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] *= inv;
    float c = 0.0f;
    bool enters = true;
    if (q[2] > P.Lz) {
        if (d[2] < 0.0f) {
            const float t = (P.Lz - q[2]) / d[2];
            q[0] += t * d[0];
            q[1] += t * d[1];
            q[2] = P.Lz;
        } else {
            enters = false;
        }
    } else if (q[2] < 0.0f) {
        enters = false;
    }
    if (enters) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            q[a] -= floorf(q[a] / S.Lper[a]) * S.Lper[a];
            if (!(q[a] < S.Lper[a]) || q[a] < 0.0f) q[a] = 0.0f;
        }
        Ray R;
        ray_begin<BF16>(S, R, q, d);
        for (int n = 0; n < 4096 && c < 1e4f; ++n) {
            c += R.M * (R.texit - R.t);
            float wdt, p[3];
            const int st = step_face(S, R, p, &wdt);
            if (st != kInside) break;
            finish_leaf<BF16>(S, R, __ldg(leaf_entry(S, R.v)));
        }
    }
    cost[i] = c;
}

// order[prefix[b] + j] = the j-th pixel (row-major inside the tile) of the
// b-th tile in claim order.
// One shard of a claim order: out[i] = order[i * stride + offset] (the
// identity order when order is NULL).
__global__ void shard_order_kernel(const uint32_t* __restrict__ order, uint32_t n_out, uint32_t stride,
                                   uint32_t offset, uint32_t* __restrict__ out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    const uint32_t j = i * stride + offset;
    out[i] = order ? order[j] : j;
}

__global__ void expand_order_kernel(const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ prefix, int n,
                                    int tiles_x, int width, int height, uint32_t* __restrict__ order)
{
    const int b = blockIdx.x;
    if (b >= n) return;
    const uint32_t tile = tiles[b];
    const int x0 = (int)(tile % (uint32_t)tiles_x) * kOrderTile, y0 = (int)(tile / (uint32_t)tiles_x) * kOrderTile;
    const int tw = min(kOrderTile, width - x0), th = min(kOrderTile, height - y0);
    const int t = threadIdx.x;
    if (t >= tw * th) return;
    const int tx = t % tw, ty = t / tw;
    order[prefix[b] + t] = (uint32_t)((y0 + ty) * width + x0 + tx);
}

// One thread per ray: the heightfield hit distance (terrain check).
__global__ void debug_terrain_kernel(DevScene S, const float* __restrict__ o, const float* __restrict__ d, int n,
                                     float* __restrict__ t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float oo[3] = {o[3 * i], o[3 * i + 1], o[3 * i + 2]};
    const float dd[3] = {d[3 * i], d[3 * i + 1], d[3 * i + 2]};
    t[i] = terrain_hit(S, oo, dd);
}

// One thread per point: surface height and normal (z, nx, ny, nz).
__global__ void debug_terrain_height_kernel(DevScene S, const float* __restrict__ xy, int n, float* __restrict__ zn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float nn[3];
    zn[4 * i] = hf_height(S, xy[2 * i], xy[2 * i + 1], nn);
    zn[4 * i + 1] = nn[0]; zn[4 * i + 2] = nn[1]; zn[4 * i + 3] = nn[2];
}

__global__ void debug_philox_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                                    uint32_t* __restrict__ out, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 r = philox4x32_10(c, make_uint2(key[2 * i], key[2 * i + 1]));
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

template <int SENSOR, bool BF16, bool COUNT, bool LEARNED, bool TERRAIN = false, bool EXTRA = false>
const void* kernel_ptr()
{
    return reinterpret_cast<const void*>(&trace_kernel<SENSOR, BF16, COUNT, LEARNED, false, TERRAIN, EXTRA>);
}

template <bool TERRAIN, bool DECOMP>
const void* pick_t(int sensor, bool bf16, bool count)
{
    if (sensor == kCamera) {
        if (bf16) return count ? kernel_ptr<kCamera, true, true, false, TERRAIN, DECOMP>()
                               : kernel_ptr<kCamera, true, false, false, TERRAIN, DECOMP>();
        return count ? kernel_ptr<kCamera, false, true, false, TERRAIN, DECOMP>()
                     : kernel_ptr<kCamera, false, false, false, TERRAIN, DECOMP>();
    }
    if (bf16) return count ? kernel_ptr<kFlux, true, true, false, TERRAIN, DECOMP>()
                           : kernel_ptr<kFlux, true, false, false, TERRAIN, DECOMP>();
    return count ? kernel_ptr<kFlux, false, true, false, TERRAIN, DECOMP>()
                 : kernel_ptr<kFlux, false, false, false, TERRAIN, DECOMP>();
}

// Kernel of a plain trace: sensor, storage, counting, heightfield ground and
// whether decomposition tracking or Rayleigh clear air is in use (those have
// variants of their own, so the others keep their registers).
const void* pick(int sensor, bool bf16, bool count, bool terrain, bool extra)
{
    if (extra) return terrain ? pick_t<true, true>(sensor, bf16, count) : pick_t<false, true>(sensor, bf16, count);
    return terrain ? pick_t<true, false>(sensor, bf16, count) : pick_t<false, false>(sensor, bf16, count);
}

template <bool DALPHA>
const void* pick_batch_t(bool bf16, bool count)
{
    if (count)
        return bf16 ? reinterpret_cast<const void*>(&trace_kernel<kFlux, true, true, false, true, false, DALPHA>)
                    : reinterpret_cast<const void*>(&trace_kernel<kFlux, false, true, false, true, false, DALPHA>);
    return bf16 ? reinterpret_cast<const void*>(&trace_kernel<kFlux, true, false, false, true, false, DALPHA>)
                : reinterpret_cast<const void*>(&trace_kernel<kFlux, false, false, false, true, false, DALPHA>);
}

const void* pick_batch(bool bf16, bool count, bool dalpha)
{
    return dalpha ? pick_batch_t<true>(bf16, count) : pick_batch_t<false>(bf16, count);
}

const void* pick_learned(int sensor, bool bf16)
{
    if (sensor == kCamera) return bf16 ? kernel_ptr<kCamera, true, false, true>() : kernel_ptr<kCamera, false, false, true>();
    return bf16 ? kernel_ptr<kFlux, true, false, true>() : kernel_ptr<kFlux, false, false, true>();
}

// Target weight of each training record: the radiance its sampled direction
// brought back, (final score - score before the vertex - the vertex's own
// local estimate) / (w * omega).
__global__ void targets_kernel(const float* __restrict__ rec_val, const float* __restrict__ final_score, unsigned n,
                               float* __restrict__ tgt)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = reinterpret_cast<const float4*>(rec_val)[i];
    const float fin = final_score[__float_as_uint(v.w)];
    const float t = v.y > 0.0f ? (fin - v.x - v.z) / v.y : 0.0f;
    tgt[i] = fmaxf(t, 0.0f);
}

}  // namespace

cudaError_t launch_trace(const TraceParams& P, int sensor, bool bf16, bool count, int grid, int block,
                         cudaStream_t st)
{
    void* args[] = {const_cast<TraceParams*>(&P)};
    const bool extra = P.sun_mode == MCRT_SUN_DECOMP || P.S.rayleigh;
    return cudaLaunchKernel(pick(sensor, bf16, count, P.S.hf != nullptr, extra), dim3(grid), dim3(block), args, 0, st);
}

cudaError_t launch_trace_learned(const TraceParams& P, int sensor, bool bf16, int grid, int block, cudaStream_t st)
{
    void* args[] = {const_cast<TraceParams*>(&P)};
    return cudaLaunchKernel(pick_learned(sensor, bf16), dim3(grid), dim3(block), args, 0, st);
}

int trace_learned_blocks_per_sm(int sensor, bool bf16, int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick_learned(sensor, bf16), block, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_trace_batch(const TraceParams& P, bool bf16, bool count, bool dalpha, int grid, int block,
                               cudaStream_t st)
{
    void* args[] = {const_cast<TraceParams*>(&P)};
    return cudaLaunchKernel(pick_batch(bf16, count, dalpha), dim3(grid), dim3(block), args, 0, st);
}

int trace_batch_blocks_per_sm(bool bf16, bool count, bool dalpha, int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick_batch(bf16, count, dalpha), block, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_targets(const float* rec_val, const float* final_score, unsigned n, float* tgt, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    targets_kernel<<<(n + 255) / 256, 256, 0, st>>>(rec_val, final_score, n, tgt);
    return cudaGetLastError();
}

int trace_blocks_per_sm(int sensor, bool bf16, bool count, bool terrain, bool extra, int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick(sensor, bf16, count, terrain, extra), block, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_finalize(const double* s1, const double* s2, double n, int count, const unsigned long long* cell_n,
                            int nq, double* out, cudaStream_t st)
{
    finalize_kernel<<<(count + 255) / 256, 256, 0, st>>>(s1, s2, n, count, cell_n, nq, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_dda(const DevScene& S, const float* o, const float* d, int cap, int* cells, float* tio,
                             int* count_status, bool bf16, cudaStream_t st)
{
    if (bf16)
        debug_dda_kernel<true><<<1, 32, 0, st>>>(S, o[0], o[1], o[2], d[0], d[1], d[2], cap, cells, tio,
                                                  count_status);
    else
        debug_dda_kernel<false><<<1, 32, 0, st>>>(S, o[0], o[1], o[2], d[0], d[1], d[2], cap, cells, tio,
                                                   count_status);
    return cudaGetLastError();
}

// Bounds-checked build: read (and clear) this unit's violation word.
bool bounds_checked_build()
{
#ifdef MCRT_CHECKED
    return true;
#else
    return false;
#endif
}

cudaError_t read_bounds_violations(unsigned* count, unsigned* first_code)
{
    *count = 0;
    *first_code = 0;
#ifdef MCRT_CHECKED
    unsigned h[2] = {0, 0};
    cudaError_t e = cudaMemcpyFromSymbol(h, g_mcrt_bounds, sizeof(h));
    if (e != cudaSuccess) return e;
    const unsigned zero[2] = {0, 0};
    e = cudaMemcpyToSymbol(g_mcrt_bounds, zero, sizeof(zero));
    *count = h[0];
    *first_code = h[1];
    return e;
#else
    return cudaSuccess;
#endif
}

int order_tiles(int width, int height, int* tiles_x)
{
    *tiles_x = (width + kOrderTile - 1) / kOrderTile;
    return *tiles_x * ((height + kOrderTile - 1) / kOrderTile);
}

cudaError_t launch_view_cost(const TraceParams& P, bool bf16, float* cost, cudaStream_t st)
{
    int tx = 0;
    const int n = order_tiles(P.width, P.height, &tx);
    const int ty = n / tx;
    if (bf16) view_cost_kernel<true><<<(n + 127) / 128, 128, 0, st>>>(P, tx, ty, cost);
    else view_cost_kernel<false><<<(n + 127) / 128, 128, 0, st>>>(P, tx, ty, cost);
    return cudaGetLastError();
}

cudaError_t launch_shard_order(const uint32_t* order, uint32_t n_out, uint32_t stride, uint32_t offset,
                               uint32_t* out, cudaStream_t st)
{
    if (n_out == 0) return cudaSuccess;
    shard_order_kernel<<<(n_out + 255) / 256, 256, 0, st>>>(order, n_out, stride, offset, out);
    return cudaGetLastError();
}

cudaError_t launch_expand_order(const uint32_t* tiles, const uint32_t* prefix, int n, int width, int height,
                                uint32_t* order, cudaStream_t st)
{
    int tx = 0;
    order_tiles(width, height, &tx);
    expand_order_kernel<<<n, kOrderTile * kOrderTile, 0, st>>>(tiles, prefix, n, tx, width, height, order);
    return cudaGetLastError();
}

cudaError_t launch_debug_terrain(const DevScene& S, const float* o, const float* d, int n, float* t, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    debug_terrain_kernel<<<(n + 127) / 128, 128, 0, st>>>(S, o, d, n, t);
    return cudaGetLastError();
}

cudaError_t launch_debug_terrain_height(const DevScene& S, const float* xy, int n, float* zn, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    debug_terrain_height_kernel<<<(n + 127) / 128, 128, 0, st>>>(S, xy, n, zn);
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    debug_philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, key, out, n);
    return cudaGetLastError();
}

}  // namespace mcrt
