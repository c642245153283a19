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
// Random numbers: path id p, event e: stream (e, 0) for the flight, the new
// direction and roulette; (e, 1) for that vertex's sun ray; (0, 2) for the
// camera jitter / ground point; (0, 3) for the direct sun ray of a flux path.
#include "mcrt_internal.h"

namespace mcrt {

namespace {

constexpr unsigned kFull = 0xffffffffu;

enum Kind { kMain = 0, kSunLocal = 1, kSunDirect = 2 };

// Counter slots (see mcrt_tally_counters).
enum {
    C_PATHS = 0, C_TENT = 1, C_REAL = 2, C_GROUND = 3, C_LEAF = 4,
    C_SUN_TENT = 5, C_SUN_LEAF = 6, C_SUN_RAYS = 7, C_ABORT = 8, C_FLIGHTS = 9
};
constexpr int kCounters = 10;

template <int SENSOR, bool BF16, bool COUNT>
__global__ void __launch_bounds__(128) trace_kernel(const __grid_constant__ TraceParams P)
{
    const DevScene& S = P.S;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    // ---- per-lane path state ----------------------------------------------
    unsigned long long pid = 0, pend = 0;
    bool have = false;         // a path (or a chunk) is assigned
    bool exhausted = false;    // warp-uniform: no more work to claim
    Ray R;
    int kind = kMain;
    float tau = 0.0f, Ts = 1.0f;
    float w = 1.0f, score = 0.0f, cf = 0.0f, tdir = 0.0f;
    uint32_t ev = 0;
    bool term_after = false;
    float vx[3] = {0, 0, 0}, nd[3] = {0, 0, 1};
    Draws dm, ds;
    dm.reset(0, 0);
    ds.reset(0, 1);
    // tallies: camera chunk sums (flushed per chunk), flux lane sums
    double c1 = 0.0, c2 = 0.0;
    double f[6] = {0, 0, 0, 0, 0, 0};
    bool flush = false;
    unsigned flush_cell = 0;
    unsigned long long cnt[kCounters] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const float mu0 = S.sun[2];

    uint64_t t_start = 0;
    if (P.deadline_ns) t_start = globaltimer_ns();
    uint32_t iter = 0;

    // Start the sun ray from vx toward the sun (stream (event, stream)).
    auto begin_sun = [&](uint32_t event, uint32_t stream, int k) {
        const uint32_t plo = (uint32_t)pid, phi = (uint32_t)(pid >> 32);
        ds.reset(event, stream);
        ray_begin<BF16>(S, R, vx, S.sun);
        kind = k;
        Ts = 1.0f;
        tau = -__logf(ds.u(plo, phi, P.key));
        if (COUNT) cnt[C_SUN_RAYS]++;
    };
    // Start the free flight of event ev from vx along nd.
    auto begin_flight = [&]() {
        const uint32_t plo = (uint32_t)pid, phi = (uint32_t)(pid >> 32);
        dm.reset(ev, 0);
        ray_begin<BF16>(S, R, vx, nd);
        kind = kMain;
        tau = -__logf(dm.u(plo, phi, P.key));
        if (COUNT) cnt[C_FLIGHTS]++;
    };
    // Initialise path pid; returns false if it ends at once (camera miss).
    auto init_path = [&]() -> bool {
        const uint32_t plo = (uint32_t)pid, phi = (uint32_t)(pid >> 32);
        w = 1.0f; score = 0.0f; ev = 0; tdir = 0.0f;
        Draws dj;
        dj.reset(0, 2);
        if (SENSOR == kCamera) {
            const unsigned long long pix = pid / P.spp;
            const int px = (int)(pix % (unsigned long long)P.width);
            const int py = (int)(pix / (unsigned long long)P.width);
            const float jx = 1.0f - dj.u(plo, phi, P.key);
            const float jy = 1.0f - dj.u(plo, phi, P.key);
            const float sx = (2.0f * ((float)px + jx) / (float)P.width - 1.0f) * P.tan_half;
            const float sy = (2.0f * ((float)py + jy) / (float)P.height - 1.0f) * P.tan_half * P.aspect;
            float d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) d[a] = P.cam_f[a] + sx * P.cam_r[a] + sy * P.cam_u[a];
            const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            d[0] *= inv; d[1] *= inv; d[2] *= inv;
            float p[3] = {P.cam_pos[0], P.cam_pos[1], P.cam_pos[2]};
            if (p[2] > P.Lz) {
                if (!(d[2] < 0.0f)) return false;
                const float t = (P.Lz - p[2]) / d[2];
                p[0] += t * d[0];
                p[1] += t * d[1];
                p[2] = P.Lz;
            } else if (p[2] < 0.0f) {
                return false;
            }
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                p[a] -= floorf(p[a] / S.Lper[a]) * S.Lper[a];
                if (!(p[a] < S.Lper[a]) || p[a] < 0.0f) p[a] = 0.0f;
            }
            vx[0] = p[0]; vx[1] = p[1]; vx[2] = p[2];
            nd[0] = d[0]; nd[1] = d[1]; nd[2] = d[2];
            begin_flight();
        } else {
            const float u0 = dj.u(plo, phi, P.key), u1 = dj.u(plo, phi, P.key);
            const float u2 = dj.u(plo, phi, P.key), u3 = dj.u(plo, phi, P.key);
            vx[0] = (1.0f - u0) * S.Lper[0];
            vx[1] = (1.0f - u1) * S.Lper[1];
            vx[2] = 0.0f;
            if (!(vx[0] < S.Lper[0])) vx[0] = 0.0f;
            if (!(vx[1] < S.Lper[1])) vx[1] = 0.0f;
            cosine_up(u2, u3, nd);
            begin_sun(0, 3, kSunDirect);
        }
        return true;
    };
    // Score the finished path pid.
    auto score_path = [&]() {
        if (COUNT) cnt[C_PATHS]++;
        if (SENSOR == kCamera) {
            c1 += (double)score;
            c2 += (double)score * (double)score;
        } else {
            const double td = (double)tdir;
            const double tf = (double)kPi / (double)mu0 * (double)score;
            const double tt = td + tf;
            f[0] += td; f[1] += td * td;
            f[2] += tf; f[3] += tf * tf;
            f[4] += tt; f[5] += tt * tt;
        }
    };
    // Move on after path pid ended: next path of the chunk, or mark idle.
    auto next_path = [&]() {
        for (;;) {
            ++pid;
            if (pid >= pend) {
                have = false;
                if (SENSOR == kCamera) {
                    flush = true;
                    flush_cell = (unsigned)((pid - 1) / P.spp);
                }
                return;
            }
            if (init_path()) return;
            score_path();
        }
    };
    // After the sun ray of a vertex (or none): add the estimate, continue.
    auto after_vertex = [&]() {
        score += cf * Ts;
        if (term_after) {
            score_path();
            next_path();
        } else {
            ++ev;
            begin_flight();
        }
    };
    // Real collision (volume) or ground hit at point p of the flight.
    auto vertex = [&](const float p[3], bool ground, float k_tot) {
        const uint32_t plo = (uint32_t)pid, phi = (uint32_t)(pid >> 32);
        const int order = (int)ev + 1;
        const bool score_it = (P.max_order == 0) || (order <= P.max_order);
        if (!ground) {
            const float om = omega_at(S, k_tot);
            const float mu = R.d[0] * S.sun[0] + R.d[1] * S.sun[1] + R.d[2] * S.sun[2];
            cf = score_it ? w * om * hg_pdf(S.g, mu) : 0.0f;
            w *= om;
            const float xi1 = dm.u(plo, phi, P.key);
            const float xi2 = dm.u(plo, phi, P.key);
            rotate_dir(R.d, hg_sample_mu(S.g, xi1), xi2, nd);
            if (COUNT) cnt[C_REAL]++;
        } else {
            cf = score_it ? w * (S.albedo * (1.0f / kPi)) * fmaxf(S.sun[2], 0.0f) : 0.0f;
            w *= S.albedo;
            const float xi1 = dm.u(plo, phi, P.key);
            const float xi2 = dm.u(plo, phi, P.key);
            cosine_up(xi1, xi2, nd);
            if (COUNT) cnt[C_GROUND]++;
        }
        term_after = (P.max_order > 0) && (order >= P.max_order);
        if (!term_after && w < 0.01f) {
            if (dm.u(plo, phi, P.key) * 0.01f <= w) w = 0.01f;
            else term_after = true;
        }
        vx[0] = p[0]; vx[1] = p[1]; vx[2] = ground ? 0.0f : p[2];
        if (score_it) {
            begin_sun(ev, 1, kSunLocal);
        } else {
            Ts = 0.0f;
            after_vertex();
        }
    };
    // A sun ray ended with transmissivity Ts.
    auto end_sun = [&]() {
        if (kind == kSunDirect) {
            tdir = Ts;
            ev = 0;
            begin_flight();
        } else {
            after_vertex();
        }
    };

    for (;;) {
        // ---- convergent section: flush tallies, refill idle lanes ---------
        if (SENSOR == kCamera) {
            unsigned pend_mask = __ballot_sync(kFull, flush);
            while (pend_mask) {
                const int src = __ffs(pend_mask) - 1;
                const unsigned cell = __shfl_sync(kFull, flush_cell, src);
                const bool mine = flush && flush_cell == cell;
                double a = mine ? c1 : 0.0, b = mine ? c2 : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(kFull, a, o);
                    b += __shfl_xor_sync(kFull, b, o);
                }
                if (lane == src) {
                    atomicAdd(P.s1 + cell, a);
                    atomicAdd(P.s2 + cell, b);
                }
                if (mine) { flush = false; c1 = 0.0; c2 = 0.0; }
                pend_mask = __ballot_sync(kFull, flush);
            }
        }
        const unsigned idle = __ballot_sync(kFull, !have);
        if (idle && !exhausted) {
            const int nidle = __popc(idle);
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&P.work->next, (unsigned long long)nidle * P.chunk);
            base = __shfl_sync(kFull, base, leader);
            if (base + (unsigned long long)nidle * P.chunk >= P.total) exhausted = true;
            if (!have) {
                pid = base + (unsigned long long)__popc(idle & lt_mask) * P.chunk;
                if (pid < P.total) {
                    pend = min(pid + (unsigned long long)P.chunk, P.total);
                    have = true;
                    if (!init_path()) {
                        score_path();
                        next_path();
                    }
                }
            }
        }
        if (!__any_sync(kFull, have)) break;
        // ---- deadline / cancel, checked every 1024 iterations -------------
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
        if (!have) continue;

        // ---- one traversal step of the current ray --------------------------
        const uint32_t plo = (uint32_t)pid, phi = (uint32_t)(pid >> 32);
        const float seg = R.texit - R.t;
        const float Mseg = R.M * seg;
        if (R.M > 0.0f && tau < Mseg) {
            // tentative collision inside the leaf
            R.t = fminf(R.t + __fdividef(tau, R.M), R.texit);
            float p[3];
            int vi[3];
            point_in_leaf(S, R, p, vi);
            const float k = __fadd_rn(kfetch<BF16>(S, vi[0], vi[1], vi[2]), S.k_gas);
            if (kind == kMain) {
                if (COUNT) cnt[C_TENT]++;
                if (dm.u(plo, phi, P.key) * R.M <= k) {
                    vertex(p, false, k);
                } else {
                    tau = -__logf(dm.u(plo, phi, P.key));
                }
            } else {
                if (COUNT) cnt[C_SUN_TENT]++;
                bool ended = false;
                if (P.sun_mode == MCRT_SUN_DELTA) {
                    if (ds.u(plo, phi, P.key) * R.M <= k) { Ts = 0.0f; ended = true; }
                } else {
                    Ts *= 1.0f - __fdividef(k, R.M);
                    if (!(Ts > 0.0f)) { Ts = 0.0f; ended = true; }
                    else if (Ts < 0.1f) {
                        if (ds.u(plo, phi, P.key) * 0.1f <= Ts) Ts = 0.1f;
                        else { Ts = 0.0f; ended = true; }
                    }
                }
                if (ended) end_sun();
                else tau = -__logf(ds.u(plo, phi, P.key));
            }
        } else {
            // cross to the next leaf
            tau -= Mseg;
            float wdt;
            const int st = step_leaf<BF16>(S, R, &wdt);
            if (COUNT) {
                if (kind == kMain) cnt[C_LEAF]++;
                else cnt[C_SUN_LEAF]++;
            }
            if (st == kInside && R.steps > P.max_steps) {
                if (COUNT) cnt[C_ABORT]++;
                if (kind == kMain) { score_path(); next_path(); }
                else { Ts = 0.0f; end_sun(); }
            } else if (st == kTop) {
                if (kind == kMain) { score_path(); next_path(); }
                else end_sun();
            } else if (st == kGround) {
                if (kind == kMain) {
                    float p[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) p[a] = __fmaf_rn(R.t, R.d[a], R.o[a]);
                    p[0] = fminf(fmaxf(p[0], 0.0f), S.Lper[0]);
                    p[1] = fminf(fmaxf(p[1], 0.0f), S.Lper[1]);
                    if (!(p[0] < S.Lper[0])) p[0] = 0.0f;
                    if (!(p[1] < S.Lper[1])) p[1] = 0.0f;
                    vertex(p, true, 0.0f);
                } else {
                    Ts = 0.0f;
                    end_sun();
                }
            }
        }
    }

    // ---- end of work: flush lane sums ---------------------------------------
    if (SENSOR == kCamera) {
        // a deadline exit may leave chunk sums pending
        if (flush || (have && c1 != 0.0)) {
            const unsigned cell = flush ? flush_cell : (unsigned)(pid / P.spp);
            atomicAdd(P.s1 + cell, c1);
            atomicAdd(P.s2 + cell, c2);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            double a = f[q];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
            if (lane == 0 && a != 0.0) atomicAdd((q & 1) ? P.s2 + q / 2 : P.s1 + q / 2, a);
        }
    }
    if (COUNT) {
#pragma unroll
        for (int q = 0; q < kCounters; ++q) {
            unsigned long long a = cnt[q];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
            if (lane == 0 && a) atomicAdd(P.counters + q, a);
        }
    }
}

__global__ void finalize_kernel(const double* __restrict__ s1, const double* __restrict__ s2, double n, int count,
                                double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double m = s1[i] / n;
    double var = s2[i] / n - m * m;
    if (var < 0.0) var = 0.0;
    out[2 * i] = m;
    out[2 * i + 1] = n > 1.0 ? sqrt(var / (n - 1.0)) : 0.0;
}

// One thread walks one ray and records its leaves (traversal check).
template <bool BF16>
__global__ void debug_dda_kernel(DevScene S, float ox, float oy, float oz, float dx, float dy, float dz, int cap,
                                 int* cells, float* tio, int* count_status)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    Ray R;
    const float p[3] = {ox, oy, oz}, d[3] = {dx, dy, dz};
    ray_begin<BF16>(S, R, p, d);
    float tbase = 0.0f;
    int n = 0, status = 0;
    for (;;) {
        if (n >= cap) { status = 3; break; }
        cells[4 * n + 0] = R.lev;
        cells[4 * n + 1] = R.v[0] >> (3 * R.lev);
        cells[4 * n + 2] = R.v[1] >> (3 * R.lev);
        cells[4 * n + 3] = R.v[2] >> (3 * R.lev);
        tio[2 * n + 0] = __fadd_rn(tbase, R.t);
        tio[2 * n + 1] = __fadd_rn(tbase, R.texit);
        ++n;
        float wdt;
        const int st = step_leaf<BF16>(S, R, &wdt);
        if (wdt != 0.0f) tbase = __fadd_rn(tbase, wdt);
        if (st == kTop) { status = 1; break; }
        if (st == kGround) { status = 2; break; }
        if (R.steps > (1u << 22)) { status = 4; break; }
    }
    count_status[0] = n;
    count_status[1] = status;
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

template <int SENSOR, bool BF16, bool COUNT>
const void* kernel_ptr()
{
    return reinterpret_cast<const void*>(&trace_kernel<SENSOR, BF16, COUNT>);
}

const void* pick(int sensor, bool bf16, bool count)
{
    if (sensor == kCamera) {
        if (bf16) return count ? kernel_ptr<kCamera, true, true>() : kernel_ptr<kCamera, true, false>();
        return count ? kernel_ptr<kCamera, false, true>() : kernel_ptr<kCamera, false, false>();
    }
    if (bf16) return count ? kernel_ptr<kFlux, true, true>() : kernel_ptr<kFlux, true, false>();
    return count ? kernel_ptr<kFlux, false, true>() : kernel_ptr<kFlux, false, false>();
}

}  // namespace

cudaError_t launch_trace(const TraceParams& P, int sensor, bool bf16, bool count, int grid, int block,
                         cudaStream_t st)
{
    void* args[] = {const_cast<TraceParams*>(&P)};
    return cudaLaunchKernel(pick(sensor, bf16, count), dim3(grid), dim3(block), args, 0, st);
}

int trace_blocks_per_sm(int sensor, bool bf16, bool count, int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick(sensor, bf16, count), block, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_finalize(const double* s1, const double* s2, double n, int count, double* out, cudaStream_t st)
{
    finalize_kernel<<<(count + 255) / 256, 256, 0, st>>>(s1, s2, n, count, out);
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

cudaError_t launch_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    debug_philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, key, out, n);
    return cudaGetLastError();
}

}  // namespace mcrt
