// wavefront.cu -- the plain camera estimator (Sec. 4.1's backward paths with
// local estimates) scheduled as a wavefront over structure-of-arrays queues,
// the alternative to the single persistent loop of trace.cu.
//
// A fixed pool of queue slots holds the paths in flight.  Each round runs
// three stage kernels:
//   flight  every queued flight (origin, direction, first optical depth) is
//           tracked to its end by null collisions through the max grid
//           (Sec. 2.2, 3.1): a real collision or a ground hit joins the
//           vertex queue, an escape or an aborted walk ends the path;
//   vertex  every queued vertex scatters (HG or the cosine law, the albedo
//           weight, Russian roulette below w = 0.01) and tracks its sun ray
//           by ratio (or delta) tracking for the local estimate; the path
//           then ends or queues its next flight for the next round;
//   start   new camera paths fill the flight queue's free slots;
// and a one-thread kernel closes the round (queue counts, slots to fill,
// the end of the trace).  Stage threads are persistent: a lane tracks one
// queue entry up to its push, then takes the next; pushes take one atomic
// per warp.  Every random number comes from the Philox counter the
// persistent kernel uses for it, and every step calls the same device
// functions in the same order, so each path scores the same value bit for
// bit; only the order of the FP64 tally additions differs.  The traversal
// is the shared device code of mcrt_device.cuh; the camera path start and
// the vertex are restated here from trace.cu's phases, statement for
// statement, and tests/test_gpu_wavefront.py holds the two schedules to
// the same images.
//
// A trace takes as many rounds as its longest path has events, and every
// stage kernel ends with its longest entry, so with the long random walks
// of optically thick clouds this schedule is slower than the persistent
// loop, where a lane on a long walk holds up no other lane.
#include <algorithm>

#include "mcrt_internal.h"

namespace mcrt {
namespace {

constexpr int kWfBlock = 128;
constexpr unsigned kFull = 0xffffffffu;

// One queue: per entry the path id, its tally cell, the index of its
// current event, the weight and score so far, a point, a direction, and
// one more float (a flight's first optical depth, a vertex's extinction).
struct WfQueue {
    unsigned long long* pid;
    uint32_t* cell;
    uint32_t* ev;
    uint32_t* ground;     // vertex entries: 1 at a ground hit
    float* w;
    float* score;
    float* x[3];
    float* d[3];
    float* aux;
    // flight entries: 0 for a flight not started yet, else the Philox block
    // of its next tentative collision, with the ray's current voxel, distance
    // along it and leaves entered (x: its current origin) -- a flight that
    // reached its step budget for the round goes on from there
    uint32_t* blk;
    uint32_t* vox[3];
    float* t;
    uint32_t* steps;
};

struct WfState {
    unsigned nf[2];               // flights queued in F[0], F[1]
    unsigned nv;                  // vertices queued
    unsigned fhead, vhead;        // next entry the flight / vertex stage takes
    unsigned need;                // free flight slots the start stage fills
    unsigned long long claimed;   // paths claimed so far
    unsigned done;                // nothing queued and nothing left to claim
    unsigned overflow;            // a push found its queue full (never expected)
};

struct WfParams {
    TraceParams P;
    WfQueue F[2];
    WfQueue V;
    WfState* st;
    unsigned cap;                 // entries per queue
};

// Entries the calling warp pushes: one atomic for the warp, the lanes'
// slots in lane order.  All 32 lanes must call it.
__device__ __forceinline__ unsigned wf_reserve(unsigned* count, bool want)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(kFull, want);
    unsigned base = 0;
    if (m) {
        const int leader = __ffs(m) - 1;
        if ((int)lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
        base = __shfl_sync(kFull, base, leader);
    }
    return base + (unsigned)__popc(m & ((1u << lane) - 1u));
}

__device__ __forceinline__ void wf_put(const WfQueue& Q, unsigned i, unsigned long long pid, uint32_t cell,
                                       uint32_t ev, uint32_t ground, float w, float score, const float x[3],
                                       const float d[3], float aux)
{
    Q.pid[i] = pid;
    Q.cell[i] = cell;
    Q.ev[i] = ev;
    Q.ground[i] = ground;
    Q.w[i] = w;
    Q.score[i] = score;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Q.x[a][i] = x[a];
        Q.d[a][i] = d[a];
    }
    Q.aux[i] = aux;
}

// The path's FP64 sums: x and x^2 (the square rounded in FP32, as the
// persistent kernel's one-path chunk sums hold it).
__device__ __forceinline__ void wf_tally(const TraceParams& P, uint32_t cell, float score)
{
    atomicAdd(P.s1 + cell, (double)score);
    atomicAdd(P.s2 + cell, (double)(score * score));
}

// A ray from o along unit d: its voxel, leaf and exit distance.
template <bool BF16>
__device__ __forceinline__ void wf_ray_start(const DevScene& S, Ray& R, const float o[3], const float d[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.o[a] = o[a];
        R.d[a] = d[a];
        R.inv_d[a] = (d[a] != 0.0f) ? __frcp_rn(d[a]) : 0.0f;
        R.v[a] = locate(o[a], d[a], S.h[a], S.inv_h[a], 0, S.n[a] - 1);
    }
    R.t = 0.0f;
    R.steps = 0;
    finish_leaf<BF16>(S, R, __ldg(leaf_entry(S, R.v)));
}

// A stage kernel's threads are persistent: a lane that finishes its entry
// takes the next one from the queue, so a warp does not wait for its
// slowest entry.  Idle lanes refill together, once kRefillLanes of them are
// idle (or all are), with one atomic per warp on the queue's read head.
constexpr int kRefillLanes = 8;

// Steps a flight takes in one round before it waits for the next round, so
// that no round waits long for one flight (one close to horizontal can wrap
// around the periodic domain for thousands of leaves).
constexpr uint32_t kStepsPerRound = 128;

// Queue entries for the idle lanes of the calling warp (all 32 lanes call
// it): true in a lane that got entry *i; *exhausted once the queue's n
// entries are all taken.
__device__ __forceinline__ bool wf_refill(unsigned* head, unsigned n, bool have, bool* exhausted, unsigned* i)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned idle = __ballot_sync(kFull, !have);
    if (*exhausted || idle == 0u || (__popc(idle) < kRefillLanes && idle != kFull)) return false;
    const int leader = __ffs(idle) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(head, (unsigned)__popc(idle));
    base = __shfl_sync(kFull, base, leader);
    if ((unsigned long long)base + (unsigned)__popc(idle) >= n) *exhausted = true;
    if (have) return false;
    *i = base + (unsigned)__popc(idle & ((1u << lane) - 1u));
    return *i < n;
}

// One step of a ray through its current leaf: to the tentative collision
// inside it (true, the voxel's extinction in *k) or across its exit face
// (false, the face's outcome in *st: kInside with the next leaf entered,
// kTop, or kGround).  p: the point reached.
template <bool BF16>
__device__ __forceinline__ bool wf_step(const DevScene& S, Ray& R, float& tau, float p[3], float* k, int* st)
{
    const float seg = R.texit - R.t;
    const float Mseg = R.M * seg;
    const bool tent = R.M > 0.0f && tau < Mseg;
    const float tn = tent ? fminf(R.t + __fdividef(tau, R.M), R.texit) : R.texit;
    int nv[3];
    advance(S, R, tn, !tent, p, nv);
    if (tent) {
        R.t = tn;
        *k = R.lev == 0 ? R.M : __fadd_rn(kfetch<BF16>(S, nv[0], nv[1], nv[2]), S.k_gas);
        return true;
    }
    tau -= Mseg;
    float wdt;
    *st = cross_face(S, R, p, nv, &wdt);
    if (*st == kInside) finish_leaf<BF16>(S, R, __ldg(leaf_entry(S, R.v)));
    return false;
}

// Flight stage: track each queued flight to its end.
template <bool BF16>
__global__ void __launch_bounds__(kWfBlock) wf_flight_kernel(const __grid_constant__ WfParams W, int in)
{
    const TraceParams& P = W.P;
    const DevScene& S = P.S;
    const WfQueue& F = W.F[in];
    const WfQueue& G = W.F[in ^ 1];       // flights of the next round
    const unsigned n = min(W.st->nf[in], W.cap);
    bool have = false, exhausted = false;
    unsigned long long pid = 0;
    uint32_t cell = 0, ev = 0, blk = 1, budget = 0;
    float w = 0.0f, score = 0.0f, tau = 0.0f;
    Ray R;
    for (;;) {
        unsigned i = 0;
        if (wf_refill(&W.st->fhead, n, have, &exhausted, &i)) {
            pid = F.pid[i];
            cell = F.cell[i];
            ev = F.ev[i];
            w = F.w[i];
            score = F.score[i];
            float o[3], d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = F.x[a][i];
                d[a] = F.d[a][i];
            }
            tau = F.aux[i];
            blk = F.blk[i];
            if (blk == 0u) {
                wf_ray_start<BF16>(S, R, o, d);
                blk = 1;
            } else {
                // a flight suspended at its step budget: re-entering its
                // leaf from the same voxel at the same distance gives the
                // same leaf, majorant and exit as before
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    R.o[a] = o[a];
                    R.d[a] = d[a];
                    R.inv_d[a] = (d[a] != 0.0f) ? __frcp_rn(d[a]) : 0.0f;
                    R.v[a] = (int)F.vox[a][i];
                }
                R.t = F.t[i];
                R.steps = F.steps[i];
                finish_leaf<BF16>(S, R, __ldg(leaf_entry(S, R.v)));
            }
            budget = kStepsPerRound;
            have = true;
        }
        if (!__any_sync(kFull, have)) break;
        int outcome = 0;                  // 1: vertex, 2: the path ends
        uint32_t ground = 0;
        float vx[3] = {0.0f, 0.0f, 0.0f}, vk = 0.0f;
        if (have) {
            float p[3], k = 0.0f;
            int st = kInside;
            if (wf_step<BF16>(S, R, tau, p, &k, &st)) {
                // tentative collision: real with probability k / M
                const uint4 x = draw_block(pid, ev << 2, blk, P.key);
                ++blk;
                const float u0 = u01(x.x);
                const float nt = -__logf(u01(x.y));
                if (u0 * R.M <= k) {
                    vx[0] = p[0]; vx[1] = p[1]; vx[2] = p[2];
                    vk = k;
                    outcome = 1;
                } else {
                    tau = nt;
                }
            } else if (st == kInside) {
                if (R.steps > P.max_steps) outcome = 2;     // aborted walk: the path ends
            } else if (st == kTop) {
                outcome = 2;
            } else {
                // ground hit (x, y kept inside the domain)
                p[2] = 0.0f;
                p[0] = fminf(fmaxf(p[0], 0.0f), S.Lper[0]);
                p[1] = fminf(fmaxf(p[1], 0.0f), S.Lper[1]);
                if (!(p[0] < S.Lper[0])) p[0] = 0.0f;
                if (!(p[1] < S.Lper[1])) p[1] = 0.0f;
                vx[0] = p[0]; vx[1] = p[1]; vx[2] = p[2];
                ground = 1;
                outcome = 1;
            }
        }
        // a flight that used up its steps for this round goes on in the next
        if (have && outcome == 0 && --budget == 0u) outcome = 3;
        const unsigned slot = wf_reserve(&W.st->nv, outcome == 1);
        if (outcome == 1) {
            if (slot < W.cap) wf_put(W.V, slot, pid, cell, ev, ground, w, score, vx, R.d, vk);
            else atomicOr(&W.st->overflow, 1u);
        } else if (outcome == 2) {
            wf_tally(P, cell, score);
        }
        const unsigned gslot = wf_reserve(&W.st->nf[in ^ 1], outcome == 3);
        if (outcome == 3) {
            if (gslot < W.cap) {
                wf_put(G, gslot, pid, cell, ev, 0u, w, score, R.o, R.d, tau);
                G.blk[gslot] = blk;
#pragma unroll
                for (int a = 0; a < 3; ++a) G.vox[a][gslot] = (uint32_t)R.v[a];
                G.t[gslot] = R.t;
                G.steps[gslot] = R.steps;
            } else {
                atomicOr(&W.st->overflow, 1u);
            }
        }
        if (outcome) have = false;
    }
}

// Vertex stage: scatter, track the sun ray, then end the path or queue its
// next flight in F[out].
template <bool BF16>
__global__ void __launch_bounds__(kWfBlock) wf_vertex_kernel(const __grid_constant__ WfParams W, int out)
{
    const TraceParams& P = W.P;
    const DevScene& S = P.S;
    const WfQueue& V = W.V;
    const unsigned n = min(W.st->nv, W.cap);
    bool have = false, exhausted = false, term_after = false;
    unsigned long long pid = 0;
    uint32_t cell = 0, ev = 0, blk = 1;
    float w = 0.0f, score = 0.0f, cf = 0.0f, Ts = 0.0f, tau = 0.0f;
    float vx[3] = {0.0f, 0.0f, 0.0f}, nd[3] = {0.0f, 0.0f, 1.0f};
    bool trk = false;                     // the sun ray is being tracked
    Ray R;
    for (;;) {
        unsigned i = 0;
        if (wf_refill(&W.st->vhead, n, have, &exhausted, &i)) {
            pid = V.pid[i];
            cell = V.cell[i];
            ev = V.ev[i];
            const bool ground = V.ground[i] != 0u;
            w = V.w[i];
            score = V.score[i];
            float d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                vx[a] = V.x[a][i];
                d[a] = V.d[a][i];
            }
            const float vk = V.aux[i];
            // the vertex block: two direction draws, the roulette, and (word 3)
            // the sun ray's first optical depth
            const uint4 x = draw_block(pid, (ev << 2) | 1u, 0u, P.key);
            const float xi1 = u01(x.x), xi2 = u01(x.y), xr = u01(x.z);
            const int order = (int)ev + 1;
            const bool score_it = (P.max_order == 0) || (order <= P.max_order);
            if (!ground) {
                const float om = omega_at(S, vk);
                const float mu = d[0] * S.sun[0] + d[1] * S.sun[1] + d[2] * S.sun[2];
                const float ph = hg_pdf(S.g, mu);
                const float mu_new = hg_sample_mu(S.g, xi1);
                cf = score_it ? w * om * ph : 0.0f;
                w *= om;
                rotate_dir(d, mu_new, xi2, nd);
            } else {
                cf = score_it ? w * (S.albedo * (1.0f / kPi)) * fmaxf(S.sun[2], 0.0f) : 0.0f;
                w *= S.albedo;
                cosine_up(xi1, xi2, nd);
            }
            term_after = (P.max_order > 0) && (order >= P.max_order);
            if (!term_after && w < 0.01f) {
                if (xr * 0.01f <= w) w = 0.01f;
                else term_after = true;
            }
            Ts = 0.0f;
            trk = score_it;
            if (trk) {
                // the sun ray: T_sun by ratio (or delta) tracking
                Ts = 1.0f;
                wf_ray_start<BF16>(S, R, vx, S.sun);
                tau = -__logf(u01(x.w));
                blk = 1;
            }
            have = true;
        }
        if (!__any_sync(kFull, have)) break;
        bool ended = false;
        if (have) {
            if (!trk) {
                ended = true;
            } else {
                float p[3], k = 0.0f;
                int st = kInside;
                if (wf_step<BF16>(S, R, tau, p, &k, &st)) {
                    const uint4 xb = draw_block(pid, (ev << 2) | 1u, blk, P.key);
                    ++blk;
                    const float u0 = u01(xb.x);
                    const float nt = -__logf(u01(xb.y));
                    if (P.sun_mode == MCRT_SUN_DELTA) {
                        if (u0 * R.M <= k) { Ts = 0.0f; ended = true; }
                    } else {
                        Ts *= 1.0f - __fdividef(k, R.M);
                        if (!(Ts > 0.0f)) {
                            Ts = 0.0f;
                            ended = true;
                        } else if (Ts < 0.1f) {
                            if (u0 * 0.1f <= Ts) Ts = 0.1f;
                            else { Ts = 0.0f; ended = true; }
                        }
                    }
                    if (!ended) tau = nt;
                } else if (st == kInside) {
                    if (R.steps > P.max_steps) { Ts = 0.0f; ended = true; }
                } else if (st == kTop) {
                    ended = true;
                } else {
                    Ts = 0.0f;
                    ended = true;
                }
            }
        }
        int outcome = 0;                  // 1: next flight, 2: the path ends
        float tau_next = 0.0f;
        if (ended) {
            score += cf * Ts;
            if (term_after) {
                outcome = 2;
            } else {
                ++ev;
                const uint4 xf = draw_block(pid, ev << 2, 0u, P.key);
                tau_next = -__logf(u01(xf.x));
                outcome = 1;
            }
        }
        const unsigned slot = wf_reserve(&W.st->nf[out], outcome == 1);
        if (outcome == 1) {
            if (slot < W.cap) {
                wf_put(W.F[out], slot, pid, cell, ev, 0u, w, score, vx, nd, tau_next);
                W.F[out].blk[slot] = 0u;
            } else {
                atomicOr(&W.st->overflow, 1u);
            }
        } else if (outcome == 2) {
            wf_tally(P, cell, score);
        }
        if (ended) have = false;
    }
}

// Start stage: claim new paths for the free slots of F[out]; path c of the
// claim order is sample c % spp of pixel pix_order[c / spp] (raster order
// without a claim order), id pixel * spp + sample.
__global__ void __launch_bounds__(kWfBlock) wf_start_kernel(const __grid_constant__ WfParams W, int out)
{
    const TraceParams& P = W.P;
    const DevScene& S = P.S;
    const unsigned n = min(W.st->need, W.cap);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned b = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
        const bool mine = b + lane < n;
        const unsigned m = __ballot_sync(kFull, mine);
        unsigned long long base = 0;
        if (m) {
            const int leader = __ffs(m) - 1;
            if ((int)lane == leader) base = atomicAdd(&W.st->claimed, (unsigned long long)__popc(m));
            base = __shfl_sync(kFull, base, leader);
        }
        const unsigned long long c = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
        bool enters = false;
        unsigned long long pid = 0;
        uint32_t cell = 0;
        float q[3] = {0.0f, 0.0f, 0.0f}, d[3] = {0.0f, 0.0f, 1.0f};
        float tau = 0.0f;
        if (mine && c < P.total) {
            unsigned long long pix = c / P.spp;
            const unsigned long long off = c - pix * P.spp;
            if (P.pix_order) pix = __ldg(P.pix_order + pix);
            pid = pix * P.spp + off;
            cell = (uint32_t)pix;
            const int px = (int)(pix % (unsigned long long)P.width);
            const int py = (int)(pix / (unsigned long long)P.width);
            // the pinhole ray through a jittered point of the pixel, moved
            // to the top of the field
            const uint4 x = draw_block(pid, 2u, 0u, P.key);
            const float jx = 1.0f - u01(x.x), jy = 1.0f - u01(x.y);
            const float sx = (2.0f * ((float)px + jx) * P.inv_width - 1.0f) * P.tan_half;
            const float sy = (2.0f * ((float)py + jy) * P.inv_height - 1.0f) * P.tan_half * P.aspect;
#pragma unroll
            for (int a = 0; a < 3; ++a) d[a] = P.cam_f[a] + sx * P.cam_r[a] + sy * P.cam_u[a];
            const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            q[0] = P.cam_pos[0]; q[1] = P.cam_pos[1]; q[2] = P.cam_pos[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) d[a] *= inv;
            enters = true;
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
            tau = -__logf(u01(x.z));
            // a path that misses the field scores 0: nothing to add
        }
        const unsigned slot = wf_reserve(&W.st->nf[out], enters);
        if (enters) {
            if (slot < W.cap) {
                wf_put(W.F[out], slot, pid, cell, 0u, 0u, 1.0f, 0.0f, q, d, tau);
                W.F[out].blk[slot] = 0u;
            } else {
                atomicOr(&W.st->overflow, 1u);
            }
        }
    }
}

__global__ void wf_init_kernel(WfState* st, unsigned cap)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->nf[0] = st->nf[1] = 0u;
        st->nv = 0u;
        st->fhead = st->vhead = 0u;
        st->need = cap;
        st->claimed = 0ull;
        st->done = 0u;
        st->overflow = 0u;
    }
}

// End of the stage kernels of a round that read F[in]: those flights and
// the vertex queue are used up; the start stage fills what F[out] left free,
// as far as paths are left to claim.
__global__ void wf_close_kernel(WfState* st, int in, unsigned cap, unsigned long long total)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int out = in ^ 1;
        st->nf[in] = 0u;
        st->nv = 0u;
        st->fhead = st->vhead = 0u;
        const unsigned queued = min(st->nf[out], cap);
        const unsigned long long left = st->claimed < total ? total - st->claimed : 0ull;
        st->need = (unsigned)min((unsigned long long)(cap - queued), left);
        if (queued == 0u && left == 0ull) st->done = 1u;
    }
}

// Bytes of one queue: the 8-byte ids, then 8 uint32 and 10 float arrays
// (80 B per entry, a multiple of 8, so every queue and the state after them
// stay 8-byte aligned for any capacity).
constexpr size_t kEntryBytes = 8 + 8 * 4 + 10 * 4;
static_assert(kEntryBytes % 8 == 0, "queue entries keep 8-byte alignment");
size_t queue_bytes(unsigned cap) { return (size_t)cap * kEntryBytes; }

void carve(WfQueue& Q, char* p, unsigned cap)
{
    Q.pid = reinterpret_cast<unsigned long long*>(p);
    p += (size_t)cap * 8;
    uint32_t** u[8] = {&Q.cell, &Q.ev, &Q.ground, &Q.blk, &Q.vox[0], &Q.vox[1], &Q.vox[2], &Q.steps};
    for (auto* f : u) { *f = reinterpret_cast<uint32_t*>(p); p += (size_t)cap * 4; }
    float** fl[10] = {&Q.w, &Q.score, &Q.x[0], &Q.x[1], &Q.x[2], &Q.d[0], &Q.d[1], &Q.d[2], &Q.aux, &Q.t};
    for (auto* f : fl) { *f = reinterpret_cast<float*>(p); p += (size_t)cap * 4; }
}

}  // namespace

int wavefront_blocks_per_sm(bool bf16)
{
    int a = 0, b = 0;
    if (bf16) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, wf_flight_kernel<true>, kWfBlock, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, wf_vertex_kernel<true>, kWfBlock, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, wf_flight_kernel<false>, kWfBlock, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, wf_vertex_kernel<false>, kWfBlock, 0);
    }
    return std::max(1, std::min(a, b));
}

cudaError_t wavefront_camera(const TraceParams& P, bool bf16, unsigned slots, int sm_count, cudaStream_t st,
                             WavefrontStats* stats)
{
    *stats = WavefrontStats{};
    const unsigned cap = slots;
    WfParams W{};
    W.P = P;
    W.cap = cap;
    char* buf = nullptr;
    const size_t qb = queue_bytes(cap);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), 3 * qb + 256, st);
    if (e != cudaSuccess) return e;
    carve(W.F[0], buf, cap);
    carve(W.F[1], buf + qb, cap);
    carve(W.V, buf + 2 * qb, cap);
    W.st = reinterpret_cast<WfState*>(buf + 3 * qb);
    const int grid = sm_count * wavefront_blocks_per_sm(bf16);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    unsigned long long launches = 0;
    auto stage = [&](int which, int q) {
        if (e != cudaSuccess) return;
        ++launches;
        if (which == 0) {
            if (bf16) wf_flight_kernel<true><<<grid, kWfBlock, 0, st>>>(W, q);
            else wf_flight_kernel<false><<<grid, kWfBlock, 0, st>>>(W, q);
        } else if (which == 1) {
            if (bf16) wf_vertex_kernel<true><<<grid, kWfBlock, 0, st>>>(W, q);
            else wf_vertex_kernel<false><<<grid, kWfBlock, 0, st>>>(W, q);
        } else if (which == 2) {
            wf_start_kernel<<<grid, kWfBlock, 0, st>>>(W, q);
        } else {
            wf_close_kernel<<<1, 32, 0, st>>>(W.st, q, cap, P.total);
        }
        e = cudaGetLastError();
    };
    if (e == cudaSuccess) {
        ++launches;
        wf_init_kernel<<<1, 32, 0, st>>>(W.st, cap);
        e = cudaGetLastError();
    }
    stage(2, 0);                                  // first paths into F[0]
    // rounds until nothing is queued and every path has been claimed; the
    // host reads the end flag after every 64 rounds (later rounds are empty)
    constexpr unsigned kCheck = 64, kMaxRounds = 1u << 24;
    unsigned r = 0;
    WfState hs{};
    while (e == cudaSuccess) {
        const int in = (int)(r & 1u);
        stage(0, in);
        stage(1, in ^ 1);
        stage(3, in);
        stage(2, in ^ 1);
        ++r;
        if (r % kCheck == 0) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, W.st, sizeof(hs), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess || hs.done || hs.overflow) break;
            if (r >= kMaxRounds) { hs.overflow = 2u; break; }
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(buf, st);
    stats->ms = ms;
    stats->rounds = r;
    stats->overflow = hs.overflow;
    stats->launches = launches;
    return e;
}

}  // namespace mcrt
