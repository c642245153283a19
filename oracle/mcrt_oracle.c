/*
 * mcrt_oracle.c -- plain, slow, FP64 CPU oracle of the null-collision path
 * tracer (Villefranque et al. 2019, "Path-tracing Monte Carlo library for 3D
 * radiative transfer in highly resolved cloudy atmospheres").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the package's smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library; the only thing both sides see is the seeded scene data.
 *
 * What it computes (each function cites the passage it follows):
 *   - Philox4x32-10 (Salmon et al., SC'11), written from the published round
 *     definition; the method's random numbers come from it.
 *   - The majorant pyramid: exact max over 8^3 children, level by level
 *     (Sec. 3.1.1 "Construction": merged voxels store the max extinction).
 *   - The paper's octree (Sec. 3.1.1: groups of 2^3 cells tested
 *     recursively for merging): the max and min over every aligned 2^L
 *     voxel block, taken straight from the voxels.
 *   - The leaf criterion of the hierarchical grid: a cell is used for tracking
 *     when the vertical optical depth bound M * h_z of the merged region is
 *     below the threshold tau~ (Sec. 4.2, list after the coarse-graining text).
 *   - An FP32 traversal "spec" (bit-exact cell sequences) and an FP64
 *     brute-force ray/voxel-face intersection that pins it.
 *   - The null-collision free-path sampler (Sec. 2.3, steps 1-5 and Eq. 2),
 *     ratio / delta tracking toward the sun, the backward local-estimate
 *     radiance and ground-flux estimators with HG scattering and a Lambertian
 *     ground (Sec. 4.1), and a forward analog flux estimator (Sec. 5.2: a
 *     path is diffuse once it has been scattered).
 *
 * Everything floating point is double unless a function says it reproduces
 * the FP32 traversal spec.  Build with -ffp-contract=off so that the FP32
 * spec is not altered by fused multiply-adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_PI 3.14159265358979323846

/* ===================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4 "Philox").    */
/* Round: two 32x32->64 products of counter words with fixed multipliers, */
/* xor of the high halves with the other counter words and the key; the   */
/* key is bumped by the Weyl constants between rounds.                    */
/* ===================================================================== */
#define PHILOX_MUL0 0xD2511F53u
#define PHILOX_MUL1 0xCD9E8D57u
#define PHILOX_WEYL0 0x9E3779B9u
#define PHILOX_WEYL1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_WEYL0; k1 += PHILOX_WEYL1; }
        uint64_t p0 = (uint64_t)PHILOX_MUL0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_MUL1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_batch(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* Random numbers.  Every draw is addressed: stream s of event e of path p
 * evaluates Philox at counter (p low, p high, (e << 2) | s, block) and the
 * key (seed low, seed high), and takes a fixed word of that block:
 *   block 0, word 0            first optical depth of a flight (stream 0)
 *                              or of a flux path's direct sun ray (stream 3)
 *   block j >= 1, words 0, 1   j-th tentative collision of the ray: the
 *                              collision test (or roulette) draw, then the
 *                              next optical depth
 *   stream 1, block 0          the vertex that ends the flight of event e:
 *                              scattering/reflection direction (words 0, 1),
 *                              Russian roulette (word 2), and the first
 *                              optical depth of its sun ray (word 3)
 *   stream 2, block 0          path start (jitter, or ground point and
 *                              direction); word 2 of a camera path's: the
 *                              first optical depth of its first flight
 *   stream 0, blocks VERTEX    a learned vertex (direction, roulette and MIS
 *   and VERTEX - 1             draws; word 1 of block VERTEX - 1: its sun
 *                              ray's first optical depth); word 0 of block
 *                              VERTEX: the species at a Rayleigh vertex
 * Streams: 0 free flight, 1 vertex and its sun ray, 2 path start, 3 direct
 * sun ray of a flux path (event 0). */
#define BLOCK_VERTEX 0xFFFFFFFFu

typedef struct {
    uint32_t key[2];
    uint32_t c0, c1, c2;
} rng_t;

static void rng_init(rng_t* r, uint64_t seed, uint64_t path, uint32_t event, uint32_t stream)
{
    r->key[0] = (uint32_t)seed;
    r->key[1] = (uint32_t)(seed >> 32);
    r->c0 = (uint32_t)path;
    r->c1 = (uint32_t)(path >> 32);
    r->c2 = (event << 2) | (stream & 3u);
}

/* Uniform in (0, 1]: ((x >> 8) + 1) * 2^-24, exact in float and double. */
static double u01(uint32_t x) { return (double)((x >> 8) + 1u) * (1.0 / 16777216.0); }

/* The four uniforms of one block. */
static void rng_block(const rng_t* r, uint32_t block, double u[4])
{
    uint32_t ctr[4] = {r->c0, r->c1, r->c2, block}, out[4];
    orc_philox4x32_10(ctr, r->key, out);
    for (int i = 0; i < 4; ++i) u[i] = u01(out[i]);
}

double orc_u01_from_u32(uint32_t x) { return u01(x); }

/* ===================================================================== */
/* BF16 rounding of a finite, non-negative float (used for the optional    */
/* BF16 storage of the extinction field).                                 */
/* ===================================================================== */
static uint32_t f2u(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static float u2f(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

/* Round to nearest-even to the 8-bit mantissa of bfloat16. */
float orc_bf16_round_nearest(float x)
{
    if (isnan(x) || isinf(x)) return x;
    uint32_t u = f2u(x);
    uint32_t lsb = (u >> 16) & 1u;
    u = u + 0x7FFFu + lsb;
    return u2f(u & 0xFFFF0000u);
}

/* Smallest bfloat16 value >= x, for x >= 0 (majorants must stay bounds). */
float orc_bf16_round_up(float x)
{
    if (isnan(x) || isinf(x) || x <= 0.0f) return x <= 0.0f ? 0.0f : x;
    uint32_t u = f2u(x);
    if (u & 0xFFFFu) u = (u & 0xFFFF0000u) + 0x10000u;
    return u2f(u);
}

/* Largest bfloat16 value <= x, for x >= 0 (minorants must stay bounds). */
float orc_bf16_round_down(float x)
{
    if (isnan(x) || isinf(x) || x <= 0.0f) return x <= 0.0f ? 0.0f : x;
    return u2f(f2u(x) & 0xFFFF0000u);
}

/* ===================================================================== */
/* Majorant pyramid (Sec. 3.1.1, "Construction"; Sec. 2.4: the majorant   */
/* is piecewise uniform over the cells of a coarser grid).  Level 0 is   */
/* the voxel field; a level-L cell covers 8^L voxels per axis and stores  */
/* the exact max over its existing children.                             */
/* ===================================================================== */
static int ceil_div(int a, int b) { return (a + b - 1) / b; }

void orc_level_dims(int nx, int ny, int nz, int level, int out[3])
{
    int f = 1;
    for (int l = 0; l < level; ++l) f *= 8;
    out[0] = ceil_div(nx, f); out[1] = ceil_div(ny, f); out[2] = ceil_div(nz, f);
}

int64_t orc_pyramid_size(int nx, int ny, int nz, int levels)
{
    int64_t tot = 0;
    for (int l = 1; l <= levels; ++l) {
        int d[3]; orc_level_dims(nx, ny, nz, l, d);
        tot += (int64_t)d[0] * d[1] * d[2];
    }
    return tot;
}

/* out: levels 1..levels concatenated, each x fastest.  round_up_bf16 != 0
 * stores RU_bf16 of each max (the bound of a field stored as RN_bf16). */
int orc_build_pyramid(const float* k, int nx, int ny, int nz, int levels, int round_up_bf16, float* out)
{
    if (levels < 1) return -1;
    const float* prev = k;
    int pd[3] = {nx, ny, nz};
    float* cur = out;
    for (int l = 1; l <= levels; ++l) {
        int d[3]; orc_level_dims(nx, ny, nz, l, d);
        for (int cz = 0; cz < d[2]; ++cz)
            for (int cy = 0; cy < d[1]; ++cy)
                for (int cx = 0; cx < d[0]; ++cx) {
                    float m = 0.0f;
                    for (int z = 8 * cz; z < 8 * cz + 8 && z < pd[2]; ++z)
                        for (int y = 8 * cy; y < 8 * cy + 8 && y < pd[1]; ++y)
                            for (int x = 8 * cx; x < 8 * cx + 8 && x < pd[0]; ++x) {
                                float v = prev[((int64_t)z * pd[1] + y) * pd[0] + x];
                                if (l == 1 && round_up_bf16) v = orc_bf16_round_up(v);
                                if (v > m) m = v;
                            }
                    cur[((int64_t)cz * d[1] + cy) * d[0] + cx] = m;
                }
        prev = cur;
        pd[0] = d[0]; pd[1] = d[1]; pd[2] = d[2];
        cur += (int64_t)d[0] * d[1] * d[2];
    }
    return 0;
}

/* Minorant pyramid (the paper's octree keeps the min beside the max,
 * Sec. 3.1.1): a level-L cell stores the exact min over its existing
 * children.  round_nearest_bf16 != 0 takes the min over RN_bf16 of the
 * voxels (the values a BF16-stored field holds). */
int orc_build_pyramid_min(const float* k, int nx, int ny, int nz, int levels, int round_nearest_bf16, float* out)
{
    if (levels < 1) return -1;
    const float* prev = k;
    int pd[3] = {nx, ny, nz};
    float* cur = out;
    for (int l = 1; l <= levels; ++l) {
        int d[3]; orc_level_dims(nx, ny, nz, l, d);
        for (int cz = 0; cz < d[2]; ++cz)
            for (int cy = 0; cy < d[1]; ++cy)
                for (int cx = 0; cx < d[0]; ++cx) {
                    float m = INFINITY;
                    for (int z = 8 * cz; z < 8 * cz + 8 && z < pd[2]; ++z)
                        for (int y = 8 * cy; y < 8 * cy + 8 && y < pd[1]; ++y)
                            for (int x = 8 * cx; x < 8 * cx + 8 && x < pd[0]; ++x) {
                                float v = prev[((int64_t)z * pd[1] + y) * pd[0] + x];
                                if (l == 1 && round_nearest_bf16) v = orc_bf16_round_nearest(v);
                                if (v < m) m = v;
                            }
                    cur[((int64_t)cz * d[1] + cy) * d[0] + cx] = m;
                }
        prev = cur;
        pd[0] = d[0]; pd[1] = d[1]; pd[2] = d[2];
        cur += (int64_t)d[0] * d[1] * d[2];
    }
    return 0;
}

/* The paper's octree (Sec. 3.1.1): a level-L cell covers an aligned block
 * of 2^L voxels per axis (clipped at the field edges) and stores the max
 * and the min extinction of the voxels it holds.  Written as that
 * definition: every cell scans its voxels directly.  The stored values are
 * those of the field the tracer reads: with round_nearest_bf16 != 0 each
 * voxel is first rounded to nearest bfloat16, and both bounds are taken
 * over the rounded values. */
void orc_octree_dims(int nx, int ny, int nz, int level, int out[3])
{
    const int f = 1 << level;
    out[0] = ceil_div(nx, f); out[1] = ceil_div(ny, f); out[2] = ceil_div(nz, f);
}

int64_t orc_octree_size(int nx, int ny, int nz, int levels)
{
    int64_t tot = 0;
    for (int l = 1; l <= levels; ++l) {
        int d[3]; orc_octree_dims(nx, ny, nz, l, d);
        tot += (int64_t)d[0] * d[1] * d[2];
    }
    return tot;
}

int orc_build_octree(const float* k, int nx, int ny, int nz, int levels, int round_nearest_bf16, float* max_out,
                     float* min_out)
{
    if (levels < 1 || levels > 30) return -1;
    int64_t off = 0;
    for (int l = 1; l <= levels; ++l) {
        int d[3]; orc_octree_dims(nx, ny, nz, l, d);
        const int f = 1 << l;
        for (int cz = 0; cz < d[2]; ++cz)
            for (int cy = 0; cy < d[1]; ++cy)
                for (int cx = 0; cx < d[0]; ++cx) {
                    float mx = 0.0f, mn = INFINITY;
                    for (int z = f * cz; z < f * cz + f && z < nz; ++z)
                        for (int y = f * cy; y < f * cy + f && y < ny; ++y)
                            for (int x = f * cx; x < f * cx + f && x < nx; ++x) {
                                float v = k[((int64_t)z * ny + y) * nx + x];
                                if (round_nearest_bf16) v = orc_bf16_round_nearest(v);
                                if (v > mx) mx = v;
                                if (v < mn) mn = v;
                            }
                    const int64_t c = off + ((int64_t)cz * d[1] + cy) * d[0] + cx;
                    max_out[c] = mx;
                    min_out[c] = mn;
                }
        off += (int64_t)d[0] * d[1] * d[2];
    }
    return 0;
}

/* ===================================================================== */
/* Scene description shared by the traversal and the estimators.          */
/* ===================================================================== */
typedef struct {
    int32_t nx, ny, nz;
    float dx, dy, dz;          /* voxel size [km] (FP32, used exactly)    */
    const float* k;            /* extinction [km^-1], x fastest           */
    int32_t levels;            /* pyramid levels above the voxels         */
    const float* pyr;          /* concatenated levels 1..levels           */
    float tau_merge;           /* leaf threshold tau~ (INFINITY allowed)  */
    int32_t finest_level;      /* finest level used for tracking (0 or 1) */
    double k_clear;            /* uniform clear-sky extinction            */
    double ssa_clear, ssa_cloud;
    double g;                  /* HG asymmetry                            */
    double ground_albedo;
    double sun[3];             /* unit vector toward the sun              */
    int32_t sun_mode;          /* 0 ratio tracking, 1 delta tracking      */
    int32_t max_order;         /* 0: all orders; n: score orders <= n     */
    double k_gas;              /* extra uniform pure absorber             */
    int64_t max_steps;         /* traversal guard per ray                 */
    const double* mlp;         /* learned proposal parameters, or NULL    */
    int32_t n_learned;         /* volume vertices per path that use it    */
    double mis_alpha;          /* HG share of the one-sample MIS mixture  */
    const float* hf;           /* heightfield ground [km] (x fastest), or NULL: flat z = 0 */
    int32_t hnx, hny;          /* heightfield samples per axis (periodic)  */
    double hmax;               /* largest height                          */
    const float* pyr_min;      /* minorant levels 1..levels (layout of pyr), or NULL: 0 */
    int32_t clear_phase;       /* phase function of the clear-air part: 0 HG (g), 1 Rayleigh */
    int32_t grid;              /* grid tracked: 0 the 8^L pyramid, 1 the 2^L octree */
    int32_t oct_levels;        /* octree levels above the voxels (grid 1)  */
    const float* oct;          /* octree maxima, levels 1..oct_levels concatenated */
    const float* oct_min;      /* octree minima, same layout              */
} orc_scene;

/* Voxels per axis of a level-L cell of the tracked grid, as a shift. */
static int cell_shift(const orc_scene* S, int L) { return S->grid == 1 ? L : 3 * L; }

static const float* level_ptr(const orc_scene* S, int level, int dims[3])
{
    const float* p = S->pyr;
    for (int l = 1; l < level; ++l) {
        int d[3]; orc_level_dims(S->nx, S->ny, S->nz, l, d);
        p += (int64_t)d[0] * d[1] * d[2];
    }
    orc_level_dims(S->nx, S->ny, S->nz, level, dims);
    return p;
}

static float kvox(const orc_scene* S, const int v[3])
{
    return S->k[((int64_t)v[2] * S->ny + v[1]) * S->nx + v[0]];
}

/* Leaf containing voxel v: the coarsest cell at a level > finest_level
 * whose bound on the vertical optical depth, M * h_z (FP32 product), is
 * <= tau~; otherwise the cell of level finest_level.  (Sec. 4.2: cells are
 * merged while the merged vertical optical depth stays below tau~; the
 * merged cell stores the max, Sec. 3.1.1.)  *m_out (may be NULL) receives
 * the leaf's minorant: the voxel itself for a voxel leaf, else the cell's
 * min rounded down to bfloat16 (the leaf map holds it in 16 bits). */
static void leaf_of_m_octree(const orc_scene* S, const int v[3], int* lev_out, float* M_out, float* m_out);

static void leaf_of_m(const orc_scene* S, const int v[3], int* lev_out, float* M_out, float* m_out)
{
    if (S->grid == 1) { leaf_of_m_octree(S, v, lev_out, M_out, m_out); return; }
    for (int L = S->levels; L > S->finest_level; --L) {
        int d[3];
        const float* P = level_ptr(S, L, d);
        int64_t ci = ((int64_t)(v[2] >> (3 * L)) * d[1] + (v[1] >> (3 * L))) * d[0] + (v[0] >> (3 * L));
        float M = P[ci];
        float hz = S->dz * (float)(1 << (3 * L));
        float tz = M * hz;
        if (tz <= S->tau_merge) {
            *lev_out = L; *M_out = M;
            if (m_out) *m_out = S->pyr_min ? orc_bf16_round_down(S->pyr_min[P - S->pyr + ci]) : 0.0f;
            return;
        }
    }
    int L = S->finest_level;
    if (L == 0) {
        *lev_out = 0; *M_out = kvox(S, v);
        if (m_out) *m_out = *M_out;
        return;
    }
    int d[3];
    const float* P = level_ptr(S, L, d);
    int64_t ci = ((int64_t)(v[2] >> (3 * L)) * d[1] + (v[1] >> (3 * L))) * d[0] + (v[0] >> (3 * L));
    *lev_out = L;
    *M_out = P[ci];
    if (m_out) *m_out = S->pyr_min ? orc_bf16_round_down(S->pyr_min[P - S->pyr + ci]) : 0.0f;
}

/* The same rule over the octree: the coarsest octree cell at a level >
 * finest_level with M * h_z <= tau~, h_z = dz * 2^L (FP32 product). */
static void leaf_of_m_octree(const orc_scene* S, const int v[3], int* lev_out, float* M_out, float* m_out)
{
    int64_t off[31];
    off[1] = 0;
    for (int L = 1; L < S->oct_levels; ++L) {
        int d[3]; orc_octree_dims(S->nx, S->ny, S->nz, L, d);
        off[L + 1] = off[L] + (int64_t)d[0] * d[1] * d[2];
    }
    for (int L = S->oct_levels; L >= S->finest_level && L >= 1; --L) {
        int d[3]; orc_octree_dims(S->nx, S->ny, S->nz, L, d);
        int64_t ci = off[L] + ((int64_t)(v[2] >> L) * d[1] + (v[1] >> L)) * d[0] + (v[0] >> L);
        float M = S->oct[ci];
        float hz = S->dz * (float)(1 << L);
        if (L == S->finest_level || M * hz <= S->tau_merge) {
            *lev_out = L; *M_out = M;
            if (m_out) *m_out = orc_bf16_round_down(S->oct_min[ci]);
            return;
        }
    }
    *lev_out = 0; *M_out = kvox(S, v);
    if (m_out) *m_out = *M_out;
}

static void leaf_of(const orc_scene* S, const int v[3], int* lev_out, float* M_out)
{
    leaf_of_m(S, v, lev_out, M_out, NULL);
}

/* Voxel range [lo, hi] covered by the level-L cell containing voxel v. */
static void cell_range(const orc_scene* S, int L, const int v[3], int lo[3], int hi[3])
{
    const int n[3] = {S->nx, S->ny, S->nz};
    const int s = cell_shift(S, L);
    for (int a = 0; a < 3; ++a) {
        int c = v[a] >> s;
        lo[a] = c << s;
        int e = (c + 1) << s;
        hi[a] = (e < n[a] ? e : n[a]) - 1;
    }
}

/* ===================================================================== */
/* FP32 traversal spec.  The CUDA traversal is required to produce the    */
/* same leaf sequence and the same t values bit for bit.  Every operation */
/* is a single IEEE-754 binary32 operation with round-to-nearest; fmaf is */
/* the correctly rounded fused multiply-add.                              */
/*                                                                        */
/* State: voxel index v of the current point, leaf (level, majorant),     */
/* segment origin o, distance t along d.  Exit distance on axis a:        */
/*   B = hi+1 (d>0) or lo (d<0) in voxel units,                           */
/*   t_a = ((float)B * dx_a - o_a) * (1/d_a)       (three roundings),     */
/*   +inf when d_a == 0;  exit axis = first minimum in x, y, z order;     */
/*   t_exit = max(min_a t_a, t).                                          */
/* Step: on the exit axis v_a = hi+1 or lo-1.  On the other axes          */
/*   p_b = fmaf(t_exit, d_b, o_b), v_b = floor(p_b * (1/dx_b)), minus one */
/*   when d_b < 0 and (float)v_b * dx_b == p_b, clamped into the old      */
/*   leaf's voxel range.  z below 0 is the ground, z >= nz the top.       */
/*   x, y wrap periodically; on a wrap the segment restarts at the exit   */
/*   point (o_a set to 0 or L_a exactly) with t = 0.                      */
/* Recorded per leaf: level, leaf index (3), t_in, t_out measured from    */
/* the ray origin (tbase + t, one FP32 addition).                         */
/* ===================================================================== */
static int locate_f32(float p, float d, float dxa, float inv_dxa, int lo, int hi)
{
    int i = (int)floorf(p * inv_dxa);
    if (d < 0.0f && (float)i * dxa == p) i -= 1;
    if (i < lo) i = lo;
    if (i > hi) i = hi;
    return i;
}

/* Returns the number of leaves written; *status: 1 top, 2 ground,
 * 3 capacity reached, 4 step guard, -1 bad input. */
int orc_dda_spec(const orc_scene* S, const float o_in[3], const float d[3], int cap,
                 int32_t* cells, float* tio, int32_t* status)
{
    const int n[3] = {S->nx, S->ny, S->nz};
    const float h[3] = {S->dx, S->dy, S->dz};
    float inv_h[3], inv_d[3], Lper[2];
    float o[3] = {o_in[0], o_in[1], o_in[2]};
    for (int a = 0; a < 3; ++a) {
        inv_h[a] = 1.0f / h[a];
        inv_d[a] = (d[a] != 0.0f) ? 1.0f / d[a] : 0.0f;
    }
    Lper[0] = (float)n[0] * h[0];
    Lper[1] = (float)n[1] * h[1];
    if (d[0] == 0.0f && d[1] == 0.0f && d[2] == 0.0f) { *status = -1; return 0; }
    int v[3];
    for (int a = 0; a < 3; ++a) v[a] = locate_f32(o[a], d[a], h[a], inv_h[a], 0, n[a] - 1);
    float t = 0.0f, tbase = 0.0f;
    int count = 0;
    for (int64_t step = 0;; ++step) {
        if (step >= S->max_steps) { *status = 4; return count; }
        int L; float M;
        leaf_of(S, v, &L, &M);
        int lo[3], hi[3];
        cell_range(S, L, v, lo, hi);
        float ta[3];
        for (int a = 0; a < 3; ++a) {
            if (d[a] == 0.0f) { ta[a] = INFINITY; continue; }
            int B = d[a] > 0.0f ? hi[a] + 1 : lo[a];
            float bnd = (float)B * h[a];
            float diff = bnd - o[a];
            ta[a] = diff * inv_d[a];
        }
        int ax = 0;
        if (ta[1] < ta[ax]) ax = 1;
        if (ta[2] < ta[ax]) ax = 2;
        float texit = ta[ax] > t ? ta[ax] : t;
        if (count >= cap) { *status = 3; return count; }
        cells[4 * count + 0] = L;
        cells[4 * count + 1] = v[0] >> cell_shift(S, L);
        cells[4 * count + 2] = v[1] >> cell_shift(S, L);
        cells[4 * count + 3] = v[2] >> cell_shift(S, L);
        tio[2 * count + 0] = tbase + t;
        tio[2 * count + 1] = tbase + texit;
        ++count;
        (void)M;
        /* step across the face on axis ax */
        float p[3];
        for (int b = 0; b < 3; ++b) p[b] = fmaf(texit, d[b], o[b]);
        int nv[3];
        for (int b = 0; b < 3; ++b) {
            if (b == ax) continue;
            nv[b] = locate_f32(p[b], d[b], h[b], inv_h[b], lo[b], hi[b]);
        }
        nv[ax] = d[ax] > 0.0f ? hi[ax] + 1 : lo[ax] - 1;
        if (ax == 2) {
            if (nv[2] < 0) { *status = 2; return count; }
            if (nv[2] >= n[2]) { *status = 1; return count; }
            v[0] = nv[0]; v[1] = nv[1]; v[2] = nv[2];
            t = texit;
        } else {
            int wrapped = 0;
            if (nv[ax] < 0) { nv[ax] = n[ax] - 1; wrapped = 1; }
            else if (nv[ax] >= n[ax]) { nv[ax] = 0; wrapped = 2; }
            v[0] = nv[0]; v[1] = nv[1]; v[2] = nv[2];
            if (wrapped) {
                tbase = tbase + texit;
                for (int b = 0; b < 3; ++b) o[b] = p[b];
                o[ax] = (wrapped == 1) ? Lper[ax] : 0.0f;
                t = 0.0f;
            } else {
                t = texit;
            }
        }
    }
}

/* ===================================================================== */
/* Brute-force FP64 leaf sequence along a ray: every voxel face crossed   */
/* up to the top/ground (or tmax), sorted by distance, each voxel mapped  */
/* to its leaf, consecutive equal leaves merged.  No incremental state.   */
/* Used to pin the FP32 spec on small grids (away from near-ties).        */
/* ===================================================================== */
typedef struct { double t; } tcross;
static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

int orc_dda_bruteforce(const orc_scene* S, const double o[3], const double d[3], double tmax, int cap,
                       int32_t* cells, double* tio, int32_t* status)
{
    const int n[3] = {S->nx, S->ny, S->nz};
    const double h[3] = {S->dx, S->dy, S->dz};
    const double Lz = (double)n[2] * h[2];
    /* distance to the top or ground */
    double tend = tmax;
    int end_status = 3;
    if (d[2] > 0.0) { double tt = (Lz - o[2]) / d[2]; if (tt < tend) { tend = tt; end_status = 1; } }
    else if (d[2] < 0.0) { double tt = (0.0 - o[2]) / d[2]; if (tt < tend) { tend = tt; end_status = 2; } }
    /* all face crossings (x, y faces are unbounded because of periodicity) */
    int64_t cnt = 0, capx = 1024;
    double* ts = (double*)malloc(sizeof(double) * capx);
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        /* faces j*h; crossing t = (j*h - o)/d for j in range */
        double t0 = 0.0, t1 = tend;
        double p0 = o[a], p1 = o[a] + tend * d[a];
        double lo = p0 < p1 ? p0 : p1, hi = p0 < p1 ? p1 : p0;
        int64_t j0 = (int64_t)floor(lo / h[a]) - 1, j1 = (int64_t)ceil(hi / h[a]) + 1;
        for (int64_t j = j0; j <= j1; ++j) {
            double tc = ((double)j * h[a] - o[a]) / d[a];
            if (tc > t0 && tc < t1) {
                if (cnt == capx) { capx *= 2; ts = (double*)realloc(ts, sizeof(double) * capx); }
                ts[cnt++] = tc;
            }
        }
    }
    qsort(ts, (size_t)cnt, sizeof(double), cmp_double);
    int count = 0;
    double prev_t = 0.0;
    int prev_leaf[6] = {-1, -1, -1, -1, 0, 0};
    for (int64_t i = 0; i <= cnt; ++i) {
        double tb = (i < cnt) ? ts[i] : tend;
        double tm = 0.5 * (prev_t + tb);
        if (tb - prev_t <= 0.0) { prev_t = tb; continue; }
        int v[3];
        int image[2] = {0, 0};   /* periodic copy of the domain holding the point */
        for (int a = 0; a < 3; ++a) {
            double p = o[a] + tm * d[a];
            if (a < 2) {
                double L = (double)n[a] * h[a];
                image[a] = (int)floor(p / L);
                p = p - floor(p / L) * L;
            }
            int vi = (int)floor(p / h[a]);
            if (vi < 0) vi = 0;
            if (vi > n[a] - 1) vi = n[a] - 1;
            v[a] = vi;
        }
        int L; float M;
        leaf_of(S, v, &L, &M);
        /* a new record starts at every leaf change and at every periodic
         * wrap (the traversal restarts its segment there) */
        const int sh = cell_shift(S, L);
        int leaf[6] = {L, v[0] >> sh, v[1] >> sh, v[2] >> sh, image[0], image[1]};
        if (count > 0 && memcmp(leaf, prev_leaf, sizeof(leaf)) == 0) {
            tio[2 * (count - 1) + 1] = tb;
        } else {
            if (count >= cap) { free(ts); *status = 3; return count; }
            memcpy(cells + 4 * count, leaf, 4 * sizeof(int));
            tio[2 * count + 0] = prev_t;
            tio[2 * count + 1] = tb;
            memcpy(prev_leaf, leaf, sizeof(leaf));
            ++count;
        }
        prev_t = tb;
    }
    free(ts);
    *status = end_status;
    return count;
}

/* ===================================================================== */
/* FP64 traversal used by the estimators.  It works on the current point  */
/* p directly: find the leaf holding p (direction decides points on a     */
/* face), the distance to that leaf's exit face, then move p there with   */
/* the exit coordinate set exactly on the face.                           */
/* ===================================================================== */
typedef struct {
    double p[3];     /* current point, x,y in [0, L) */
    double d[3];
    int v[3];        /* voxel of p for the current leaf */
    int lev;         /* leaf level */
    double M;        /* leaf majorant (+ k_gas) */
    double m;        /* leaf minorant (+ k_gas) */
    int lo[3], hi[3];
    double seg;      /* distance from p to the leaf exit */
    int exit_axis;
    int64_t steps;
} trav64;

static int locate64(const orc_scene* S, double p, double d, int a)
{
    const int n[3] = {S->nx, S->ny, S->nz};
    const double h[3] = {S->dx, S->dy, S->dz};
    int i = (int)floor(p / h[a]);
    if (d < 0.0 && (double)i * h[a] == p) i -= 1;
    if (i < 0) i = 0;
    if (i > n[a] - 1) i = n[a] - 1;
    return i;
}

static void trav_setup_leaf(const orc_scene* S, trav64* T)
{
    const double h[3] = {S->dx, S->dy, S->dz};
    float Mf, mf;
    leaf_of_m(S, T->v, &T->lev, &Mf, &mf);
    T->M = (double)Mf + S->k_gas;
    T->m = (double)mf + S->k_gas;
    cell_range(S, T->lev, T->v, T->lo, T->hi);
    double best = INFINITY;
    int ax = 0;
    for (int a = 0; a < 3; ++a) {
        if (T->d[a] == 0.0) continue;
        double bnd = (T->d[a] > 0.0 ? (double)(T->hi[a] + 1) : (double)T->lo[a]) * h[a];
        double ta = (bnd - T->p[a]) / T->d[a];
        if (ta < 0.0) ta = 0.0;
        if (ta < best) { best = ta; ax = a; }
    }
    T->seg = best;
    T->exit_axis = ax;
}

static void trav_begin(const orc_scene* S, trav64* T, const double p[3], const double d[3])
{
    for (int a = 0; a < 3; ++a) { T->p[a] = p[a]; T->d[a] = d[a]; }
    for (int a = 0; a < 3; ++a) T->v[a] = locate64(S, T->p[a], T->d[a], a);
    T->steps = 0;
    trav_setup_leaf(S, T);
}

/* Advance p by s < seg inside the current leaf (a tentative collision). */
static void trav_move_inside(const orc_scene* S, trav64* T, double s)
{
    (void)S;
    for (int a = 0; a < 3; ++a) T->p[a] += s * T->d[a];
    T->seg -= s;
    if (T->seg < 0.0) T->seg = 0.0;
}

/* Voxel holding p, clamped into the current leaf (so k <= M holds). */
static double trav_k_here(const orc_scene* S, const trav64* T, int vox[3])
{
    for (int a = 0; a < 3; ++a) {
        int i = locate64(S, T->p[a], T->d[a], a);
        if (i < T->lo[a]) i = T->lo[a];
        if (i > T->hi[a]) i = T->hi[a];
        vox[a] = i;
    }
    return (double)kvox(S, vox) + S->k_gas;
}

/* Move to the exit face of the current leaf and enter the next one.
 * Returns 0 inside, 1 top of atmosphere, 2 ground, 4 step guard. */
static int trav_next_leaf(const orc_scene* S, trav64* T)
{
    const int n[3] = {S->nx, S->ny, S->nz};
    const double h[3] = {S->dx, S->dy, S->dz};
    if (++T->steps > S->max_steps) return 4;
    int ax = T->exit_axis;
    double s = T->seg;
    double bnd = (T->d[ax] > 0.0 ? (double)(T->hi[ax] + 1) : (double)T->lo[ax]) * h[ax];
    for (int a = 0; a < 3; ++a) T->p[a] += s * T->d[a];
    T->p[ax] = bnd;
    int nv_ax = T->d[ax] > 0.0 ? T->hi[ax] + 1 : T->lo[ax] - 1;
    if (ax == 2) {
        if (nv_ax < 0) { T->p[2] = 0.0; return 2; }
        if (nv_ax >= n[2]) { T->p[2] = (double)n[2] * h[2]; return 1; }
    } else {
        double L = (double)n[ax] * h[ax];
        if (nv_ax < 0) T->p[ax] = L;
        else if (nv_ax >= n[ax]) T->p[ax] = 0.0;
    }
    for (int a = 0; a < 3; ++a) T->v[a] = locate64(S, T->p[a], T->d[a], a);
    trav_setup_leaf(S, T);
    return 0;
}

/* ===================================================================== */
/* Phase functions and directions.                                        */
/* ===================================================================== */
/* HG phase function normalised to 1 over 4 pi sr. */
double orc_hg_pdf(double g, double mu)
{
    double den = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * ORC_PI * den * sqrt(den));
}

/* Rayleigh phase function normalised to 1 over 4 pi sr: 3 (1 + mu^2) / (16 pi). */
double orc_rayleigh_pdf(double mu)
{
    return 3.0 * (1.0 + mu * mu) / (16.0 * ORC_PI);
}

/* Inverse-CDF Rayleigh cosine for xi in (0, 1].  The cosine's CDF is
 * (mu^3 + 3 mu + 4) / 8, so mu solves the depressed cubic
 * mu^3 + 3 mu + 4 - 8 xi = 0, whose one real root (Cardano) is
 * A^(1/3) - A^(-1/3) with A = 4 xi - 2 + sqrt((4 xi - 2)^2 + 1). */
double orc_rayleigh_sample_mu(double xi)
{
    double b = 4.0 * xi - 2.0;
    double A = b + sqrt(b * b + 1.0);
    double c = cbrt(A);
    double mu = c - 1.0 / c;
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

/* Inverse-CDF cosine of the HG distribution for xi in (0, 1]. */
double orc_hg_sample_mu(double g, double xi)
{
    if (fabs(g) < 1e-4) return 1.0 - 2.0 * xi;
    double s = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
    double mu = (1.0 + g * g - s * s) / (2.0 * g);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

/* Orthonormal basis around a unit vector n (Duff et al., "Building an
 * orthonormal basis, revisited", JCGT 2017). */
static void onb(const double n[3], double b1[3], double b2[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a; b1[1] = sign * b; b1[2] = -sign * n[0];
    b2[0] = b; b2[1] = sign + n[1] * n[1] * a; b2[2] = -n[1];
}

/* Direction making cosine mu with d, azimuth phi in the basis of d. */
static void rotate_dir(const double d[3], double mu, double phi, double out[3])
{
    double b1[3], b2[3];
    onb(d, b1, b2);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double c = st * cos(phi), s = st * sin(phi);
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = c * b1[a] + s * b2[a] + mu * d[a];
    double nn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) out[a] = r[a] / nn;
}

/* Cosine-weighted direction about +z: cos(theta) = sqrt(xi1) > 0. */
static void cosine_up(double xi1, double xi2, double out[3])
{
    double st = sqrt(fmax(0.0, 1.0 - xi1));
    double phi = 2.0 * ORC_PI * xi2;
    out[0] = st * cos(phi); out[1] = st * sin(phi); out[2] = sqrt(xi1);
}

void orc_hg_sample_dirs(double g, const double* d_in, const double* xi, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        double mu = orc_hg_sample_mu(g, xi[2 * i]);
        rotate_dir(d_in + 3 * i, mu, 2.0 * ORC_PI * xi[2 * i + 1], out + 3 * i);
    }
}

/* ===================================================================== */
/* Heightfield ground (an extension of the paper's flat Lambertian        */
/* ground; the paper finds the ground's shape matters little for the      */
/* cloud estimates, Sec. 1).  Heights h[j][i] sit at the corners of a     */
/* periodic hnx x hny grid of cells of size Lx/hnx x Ly/hny.  Cell (i, j) */
/* is cut along its diagonal from corner (i, j) to corner (i+1, j+1):     */
/* with u, v the position in the cell scaled to [0, 1], triangle A        */
/* (u >= v) has corners 00, 10, 11 and triangle B (u < v) corners 00, 11, */
/* 01.  On a triangle the surface is the plane z = c + a u + b v.         */
/* ===================================================================== */
#define ORC_TERRAIN_OFFSET 1e-5      /* km: a path leaves the surface this far along its normal */
#define ORC_TERRAIN_MAX_CELLS 1000000

static int64_t wrap_index(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static double hf_at(const orc_scene* S, int64_t i, int64_t j)
{
    return (double)S->hf[wrap_index(j, S->hny) * S->hnx + wrap_index(i, S->hnx)];
}

static void tri_plane(const orc_scene* S, int64_t i, int64_t j, int tri, double* a, double* b, double* c)
{
    double h00 = hf_at(S, i, j), h10 = hf_at(S, i + 1, j), h01 = hf_at(S, i, j + 1), h11 = hf_at(S, i + 1, j + 1);
    *c = h00;
    if (tri == 0) { *a = h10 - h00; *b = h11 - h10; }
    else          { *a = h11 - h01; *b = h01 - h00; }
}

/* Unit upward normal of the plane z = c + a u + b v, u = x / hx - i. */
static void tri_normal(const orc_scene* S, int64_t i, int64_t j, int tri, double n[3])
{
    double a, b, c;
    tri_plane(S, i, j, tri, &a, &b, &c);
    double hx = (double)S->nx * S->dx / S->hnx, hy = (double)S->ny * S->dy / S->hny;
    double gx = a / hx, gy = b / hy;
    double inv = 1.0 / sqrt(gx * gx + gy * gy + 1.0);
    n[0] = -gx * inv; n[1] = -gy * inv; n[2] = inv;
}

/* Surface height and normal at (x, y). */
double orc_terrain_height(const orc_scene* S, double x, double y, double n[3])
{
    double hx = (double)S->nx * S->dx / S->hnx, hy = (double)S->ny * S->dy / S->hny;
    int64_t i = (int64_t)floor(x / hx), j = (int64_t)floor(y / hy);
    double u = x / hx - (double)i, v = y / hy - (double)j;
    int tri = u >= v ? 0 : 1;
    double a, b, c;
    tri_plane(S, i, j, tri, &a, &b, &c);
    if (n) tri_normal(S, i, j, tri, n);
    return c + a * u + b * v;
}

/* First point where the ray p + t d (t >= 0) meets the surface.  The
 * ray's horizontal projection is walked cell by cell (2D DDA over
 * unwrapped cell indices) over the part of the ray with z <= hmax (it
 * reaches z = 0, at or below every height, last); in each cell the ray
 * crosses at most two triangle pieces, split where u = v; on a piece the
 * ray's height above the plane, f(t), is linear, and the hit is the first
 * t where f reaches 0 (at the piece start if f is already <= 0 there).
 * Returns 1 with the distance, the (unwrapped) cell and the triangle;
 * 0 if the ray leaves the relief layer first. */
int orc_terrain_hit(const orc_scene* S, const double p[3], const double d[3], double* t_hit, int64_t cell[2],
                    int* tri_out)
{
    if (!S->hf) return 0;
    double hx = (double)S->nx * S->dx / S->hnx, hy = (double)S->ny * S->dy / S->hny;
    double t0 = 0.0, t1;
    if (p[2] > S->hmax) {
        if (d[2] >= 0.0) return 0;
        t0 = (S->hmax - p[2]) / d[2];
    }
    if (d[2] < 0.0) t1 = -p[2] / d[2];
    else if (d[2] > 0.0) t1 = (S->hmax - p[2]) / d[2];
    else t1 = INFINITY;
    if (t1 < t0) return 0;
    double x0 = p[0] + t0 * d[0], y0 = p[1] + t0 * d[1];
    int64_t i = (int64_t)floor(x0 / hx), j = (int64_t)floor(y0 / hy);
    if (d[0] < 0.0 && (double)i * hx == x0) i -= 1;
    if (d[1] < 0.0 && (double)j * hy == y0) j -= 1;
    double t = t0;
    for (int64_t step = 0; step < ORC_TERRAIN_MAX_CELLS; ++step) {
        double tx = d[0] > 0.0 ? ((double)(i + 1) * hx - p[0]) / d[0]
                  : d[0] < 0.0 ? ((double)i * hx - p[0]) / d[0] : INFINITY;
        double ty = d[1] > 0.0 ? ((double)(j + 1) * hy - p[1]) / d[1]
                  : d[1] < 0.0 ? ((double)j * hy - p[1]) / d[1] : INFINITY;
        double te = fmin(fmin(tx, ty), t1);
        if (te < t) te = t;
        /* pieces of [t, te] on either side of the diagonal u = v */
        double g0 = (p[0] / hx - (double)i) - (p[1] / hy - (double)j), g1 = d[0] / hx - d[1] / hy;
        double cut[3] = {t, te, te};
        int np = 1;
        if (g1 != 0.0) {
            double tm = -g0 / g1;
            if (tm > t && tm < te) { cut[1] = tm; cut[2] = te; np = 2; }
        }
        for (int q = 0; q < np; ++q) {
            double a0 = cut[q], b0 = cut[q + 1];
            double mid = 0.5 * (a0 + b0);
            int tri = (g0 + g1 * mid) >= 0.0 ? 0 : 1;
            double A, B, Cc;
            tri_plane(S, i, j, tri, &A, &B, &Cc);
            double fa = (p[2] + a0 * d[2]) - (Cc + A * ((p[0] + a0 * d[0]) / hx - (double)i) +
                                             B * ((p[1] + a0 * d[1]) / hy - (double)j));
            double fb = (p[2] + b0 * d[2]) - (Cc + A * ((p[0] + b0 * d[0]) / hx - (double)i) +
                                             B * ((p[1] + b0 * d[1]) / hy - (double)j));
            double th;
            if (fa <= 0.0) th = a0;
            else if (fb <= 0.0) th = a0 + fa * (b0 - a0) / (fa - fb);
            else continue;
            *t_hit = th;
            if (cell) { cell[0] = i; cell[1] = j; }
            if (tri_out) *tri_out = tri;
            return 1;
        }
        if (te >= t1) return 0;
        if (tx <= ty) i += d[0] > 0.0 ? 1 : -1;
        else j += d[1] > 0.0 ? 1 : -1;
        t = te;
    }
    return 0;
}

/* The ray's terrain hit with its normal, or 0. */
static int terrain_hit_normal(const orc_scene* S, const double p[3], const double d[3], double* t, double n[3])
{
    int64_t cell[2];
    int tri;
    if (!orc_terrain_hit(S, p, d, t, cell, &tri)) return 0;
    tri_normal(S, cell[0], cell[1], tri, n);
    return 1;
}

/* Cosine-weighted direction about the unit normal n (the flat ground's
 * cosine_up when n = +z). */
static void cosine_about(const double n[3], double xi1, double xi2, double out[3])
{
    double b1[3], b2[3];
    onb(n, b1, b2);
    double st = sqrt(fmax(0.0, 1.0 - xi1)), ct = sqrt(xi1);
    double phi = 2.0 * ORC_PI * xi2;
    double c = st * cos(phi), s = st * sin(phi);
    for (int a = 0; a < 3; ++a) out[a] = c * b1[a] + s * b2[a] + ct * n[a];
}

/* ===================================================================== */
/* Free flight with null collisions (Sec. 2.3, steps 4a-4g; Eq. 2): the   */
/* optical depth -ln(u) is spent across leaves of uniform majorant M;     */
/* at a tentative collision the true extinction k is read and the         */
/* collision is real with probability k / M, else null and the flight    */
/* goes on with a fresh optical depth.                                    */
/* ===================================================================== */
enum { EV_ESCAPE = 1, EV_GROUND = 2, EV_VOLUME = 3, EV_ABORT = 4 };

typedef struct { int64_t tentative, real, leaves; } orc_counts;

static void wrap_xy(const orc_scene* S, double p[3]);

/* With a heightfield the flight also ends where the ray meets the surface
 * (distance tg, found before the flight): the leaf holding that point is
 * cut there, and a flight that spends none of its optical depth before it
 * is a ground event with the triangle's normal in n_ground. */
static int free_flight(const orc_scene* S, double p[3], const double d[3], const rng_t* r,
                       double* k_at, int vox_at[3], orc_counts* C, double n_ground[3], double tau0)
{
    const double p0[3] = {p[0], p[1], p[2]};
    double tg = INFINITY, ng[3] = {0.0, 0.0, 1.0};
    const int has_tg = S->hf ? terrain_hit_normal(S, p0, d, &tg, ng) : 0;
    double dist = 0.0;
    if (n_ground) { n_ground[0] = 0.0; n_ground[1] = 0.0; n_ground[2] = 1.0; }
    trav64 T;
    trav_begin(S, &T, p, d);
    double u[4];
    double tau = tau0;                  /* given by the caller (>= 0), else word 0 of block 0 */
    if (!(tau >= 0.0)) {
        rng_block(r, 0, u);
        tau = -log(u[0]);
    }
    for (uint32_t j = 1;;) {
        double seg = T.seg;
        const int ground_here = has_tg && dist + seg >= tg;
        if (ground_here) seg = fmax(tg - dist, 0.0);
        if (T.M > 0.0 && tau < T.M * seg) {
            double s = tau / T.M;
            trav_move_inside(S, &T, s);
            dist += s;
            int vox[3];
            double k = trav_k_here(S, &T, vox);
            if (C) C->tentative++;
            rng_block(r, j++, u);
            if (u[0] * T.M <= k) {
                for (int a = 0; a < 3; ++a) p[a] = T.p[a];
                *k_at = k;
                if (vox_at) { vox_at[0] = vox[0]; vox_at[1] = vox[1]; vox_at[2] = vox[2]; }
                if (C) C->real++;
                return EV_VOLUME;
            }
            tau = -log(u[1]);
        } else if (ground_here) {
            for (int a = 0; a < 3; ++a) p[a] = p0[a] + tg * d[a];
            wrap_xy(S, p);
            if (n_ground) { n_ground[0] = ng[0]; n_ground[1] = ng[1]; n_ground[2] = ng[2]; }
            return EV_GROUND;
        } else {
            tau -= T.M * T.seg;
            dist += T.seg;
            int st = trav_next_leaf(S, &T);
            if (C) C->leaves++;
            if (st == 1) { for (int a = 0; a < 3; ++a) p[a] = T.p[a]; return EV_ESCAPE; }
            if (st == 2) {
                for (int a = 0; a < 3; ++a) p[a] = T.p[a];
                if (S->hf && n_ground) orc_terrain_height(S, p[0], p[1], n_ground);
                return EV_GROUND;
            }
            if (st == 4) return EV_ABORT;
        }
    }
}

/* Transmissivity from p toward direction s up to the top of atmosphere.
 * sun_mode 0: ratio tracking, t *= 1 - k/M at each tentative collision,
 * with Russian roulette below 0.1 (survive with prob t/0.1, t <- 0.1).
 * sun_mode 1: the 0/1 estimator of Sec. 2.3 (delta tracking).
 * sun_mode 2: decomposition (residual ratio) tracking: each leaf's
 * minorant m is a control extinction whose transmissivity exp(-m s) is
 * applied exactly over every distance s travelled, and ratio tracking runs
 * on the residual k - m with majorant M - m (t *= 1 - (k - m)/(M - m)).
 * A voxel leaf has m = M = k: it is crossed with no random draw at all.
 * Roulette below 0.1 as in ratio tracking; at a leaf crossing it draws
 * word 3 of the next block (the block is then used up). */
static double transmissivity(const orc_scene* S, const double p[3], const double s[3], const rng_t* r,
                             orc_counts* C, double tau0)
{
    if (S->hf) {                        /* shadow of the terrain */
        double tg;
        if (orc_terrain_hit(S, p, s, &tg, NULL, NULL)) return 0.0;
    }
    trav64 T;
    trav_begin(S, &T, p, s);
    double t = 1.0;
    double u[4];
    double tau = tau0;                  /* given by the caller (>= 0), else word 0 of block 0 */
    if (!(tau >= 0.0)) {
        rng_block(r, 0, u);
        tau = -log(u[0]);
    }
    const int decomp = S->sun_mode == 2;
    for (uint32_t j = 1;;) {
        double Mt = decomp ? T.M - T.m : T.M;      /* tracking majorant */
        if (Mt > 0.0 && tau < Mt * T.seg) {
            double ds = tau / Mt;
            trav_move_inside(S, &T, ds);
            int vox[3];
            double k = trav_k_here(S, &T, vox);
            if (C) C->tentative++;
            rng_block(r, j++, u);
            if (S->sun_mode == 1) {
                if (u[0] * T.M <= k) return 0.0;
            } else {
                if (decomp) t *= exp(-T.m * ds) * (1.0 - (k - T.m) / Mt);
                else t *= 1.0 - k / T.M;
                if (t <= 0.0) return 0.0;
                if (t < 0.1) {
                    if (u[0] * 0.1 <= t) t = 0.1;
                    else return 0.0;
                }
            }
            tau = -log(u[1]);
        } else {
            tau -= Mt * T.seg;
            if (decomp) t *= exp(-T.m * T.seg);
            int st = trav_next_leaf(S, &T);
            if (C) C->leaves++;
            if (st == 1) return t;
            if (st == 2 || st == 4) return 0.0;
            if (decomp && t < 0.1) {
                rng_block(r, j++, u);
                if (u[3] * 0.1 <= t) t = 0.1;
                else return 0.0;
            }
        }
    }
}

double orc_transmissivity(const orc_scene* S, const double p[3], const double s[3], uint64_t seed, uint64_t path)
{
    rng_t r;
    rng_init(&r, seed, path, 0, 1);
    return transmissivity(S, p, s, &r, NULL, -1.0);
}

/* Distance to the first real collision (for the mean-free-path pin). */
double orc_first_collision_distance(const orc_scene* S, const double p[3], const double d[3], uint64_t seed, uint64_t path)
{
    rng_t r;
    rng_init(&r, seed, path, 0, 0);
    double q[3] = {p[0], p[1], p[2]};
    trav64 T;
    trav_begin(S, &T, q, d);
    double dist = 0.0;
    double u[4];
    rng_block(&r, 0, u);
    double tau = -log(u[0]);
    for (uint32_t j = 1;;) {
        if (T.M > 0.0 && tau < T.M * T.seg) {
            double s = tau / T.M;
            trav_move_inside(S, &T, s);
            dist += s;
            int vox[3];
            double k = trav_k_here(S, &T, vox);
            rng_block(&r, j++, u);
            if (u[0] * T.M <= k) return dist;
            tau = -log(u[1]);
        } else {
            tau -= T.M * T.seg;
            dist += T.seg;
            int st = trav_next_leaf(S, &T);
            if (st != 0) return -dist;
        }
    }
}

/* ===================================================================== */
/* Backward path with local estimates toward the sun (Sec. 4.1).          */
/* Volume event at x: contribution w * omega(x) * p_HG(d . s) * T_sun(x); */
/* ground event: w * (rho / pi) * max(s_z, 0) * T_sun(x).  Then w *=      */
/* omega (or rho), a new direction is sampled (HG about d, or cosine      */
/* about +z), and Russian roulette applies below w = 0.01.  The path ends */
/* at the top of atmosphere.  The flight of event e draws from stream     */
/* (e, 0); its vertex and the vertex's sun ray from stream (e, 1).        */
/* ===================================================================== */
#define MLP_IN 9
#define MLP_OUT 40
void orc_mlp_forward(const double* params, const double* x, int64_t rows, double* out);
double orc_mis_sample(const double* raw, double g, double alpha, const double d[3], const double u[4], double out[3],
                      double* q_out, double* phg_out);

/* Features of a volume vertex for the learned proposal: position scaled to
 * [-1, 1] per axis, incoming direction, and ln(M + 1e-6) of the extinction
 * at the voxel and of the level-1 and level-2 majorants of its cells (the
 * top level when fewer levels exist). */
static void vertex_features(const orc_scene* S, const double p[3], const double d[3], double k_tot, const int vox[3],
                            double x[MLP_IN])
{
    double L[3] = {(double)S->nx * S->dx, (double)S->ny * S->dy, (double)S->nz * S->dz};
    for (int a = 0; a < 3; ++a) x[a] = 2.0 * p[a] / L[a] - 1.0;
    for (int a = 0; a < 3; ++a) x[3 + a] = d[a];
    x[6] = log(k_tot + 1e-6);
    for (int q = 1; q <= 2; ++q) {
        int lev = q <= S->levels ? q : S->levels;
        int dims[3];
        const float* P = level_ptr(S, lev, dims);
        int c[3] = {vox[0] >> (3 * lev), vox[1] >> (3 * lev), vox[2] >> (3 * lev)};
        double M = (double)P[((int64_t)c[2] * dims[1] + c[1]) * dims[0] + c[0]] + S->k_gas;
        x[6 + q] = log(M + 1e-6);
    }
}

/* Online-training record of one learned vertex (the training set of the
 * learned proposal): the vertex's features, the direction sampled there,
 * the path's score before the vertex, the weight times omega at the vertex,
 * the vertex's own local estimate, and the target of the KL estimator:
 * the score the path gained after the vertex, excluding its own estimate,
 * divided by w * omega.  That ratio equals p_HG(w') L(w') / q_mix(w'), the
 * density ratio p* / q_mix of the target distribution p* ~ p_HG L whose
 * KL divergence to the network's mixture is minimised. */
typedef struct {
    uint64_t path;
    int32_t vertex;             /* learned-vertex index along the path */
    int32_t pad;
    double x[MLP_IN];
    double dir[3];
    double before, w_omega, own, target;
} orc_record;

typedef struct {
    orc_record* rec;
    int64_t cap;
    int64_t n;                  /* records emitted (may exceed cap: the rest are dropped) */
} orc_rec_sink;

/* Share of the scattering at extinction k_total due to the cloud droplets
 * (the rest is the clear air): k_c omega_cloud / (k_c omega_cloud +
 * k_clear omega_clear). */
static double cloud_scatter_share(const orc_scene* S, double k_total)
{
    double k = k_total - S->k_gas;
    double kc = k - S->k_clear;
    if (kc < 0.0) kc = 0.0;
    double kcl = k - kc;
    double sc = kc * S->ssa_cloud, sr = kcl * S->ssa_clear;
    return (sc + sr > 0.0) ? sc / (sc + sr) : 1.0;
}

static double omega_at(const orc_scene* S, double k_total)
{
    double k = k_total - S->k_gas;          /* cloud + clear */
    double kc = k - S->k_clear;
    if (kc < 0.0) kc = 0.0;
    double kcl = k - kc;                    /* clear part actually present */
    if (k_total <= 0.0) return 0.0;
    return (kc * S->ssa_cloud + kcl * S->ssa_clear) / k_total;
}

/* d/dg of ln p_HG(mu) = -2g / (1 - g^2) - 3 (g - mu) / (1 + g^2 - 2 g mu). */
double orc_hg_dlog_dg(double g, double mu)
{
    return -2.0 * g / (1.0 - g * g) - 3.0 * (g - mu) / (1.0 + g * g - 2.0 * g * mu);
}

/* Backward path; *dscore (may be NULL) receives the derivative of the
 * score with respect to the HG asymmetry g, by the score-function method:
 * each local estimate c_j also contributes c_j (sum of d ln p_HG / dg of
 * the directions sampled before vertex j + d ln p_HG / dg of its own phase
 * value toward the sun); ground terms only carry the earlier sum.
 * *dalpha (may be NULL) receives the derivative with respect to the cloud
 * droplets' absorptivity alpha = 1 - omega_cloud at fixed extinction (the
 * sensitivity of Sec. 6.1): only the weights depend on it, through
 * omega = (k_c (1 - alpha) + k_clear omega_clear) / k, so each estimate c_j
 * contributes c_j times the sum over volume vertices up to and including j
 * of d ln omega / d alpha = -k_c / (k omega).  (Roulette keeps this form:
 * a survival's probability w / 0.01 carries the same logarithmic
 * derivative as the weight it replaces.) */
static double trace_backward_r(const orc_scene* S, double p[3], double d[3], uint64_t seed, uint64_t path,
                               orc_counts* C, int64_t* aborted, double* dscore, double* dalpha,
                               orc_rec_sink* sink, double tau_first);

static double trace_backward_d(const orc_scene* S, double p[3], double d[3], uint64_t seed, uint64_t path,
                               orc_counts* C, int64_t* aborted, double* dscore, double* dalpha)
{
    return trace_backward_r(S, p, d, seed, path, C, aborted, dscore, dalpha, NULL, -1.0);
}

static double trace_backward(const orc_scene* S, double p[3], double d[3], uint64_t seed, uint64_t path,
                             orc_counts* C, int64_t* aborted)
{
    return trace_backward_d(S, p, d, seed, path, C, aborted, NULL, NULL);
}

/* sink (may be NULL): receives one record per learned vertex of the path.
 * tau_first >= 0: the first flight's optical depth (a camera path draws it
 * with its start); else the flight draws it from its own stream. */
static double trace_backward_r(const orc_scene* S, double p[3], double d[3], uint64_t seed, uint64_t path,
                               orc_counts* C, int64_t* aborted, double* dscore, double* dalpha,
                               orc_rec_sink* sink, double tau_first)
{
    const int64_t rec0 = sink ? sink->n : 0;   /* this path's first record */
    double sg = 0.0, ds = 0.0;
    double sa = 0.0, da = 0.0;
    double w = 1.0, score = 0.0;
    int lv = 0;                 /* volume vertices so far */
    const double* s = S->sun;
    for (uint32_t e = 0;; ++e) {
        rng_t r;
        rng_init(&r, seed, path, e, 0);
        double k;
        int vox[3] = {0, 0, 0};
        double ng[3];
        int ev = free_flight(S, p, d, &r, &k, vox, C, ng, e == 0 ? tau_first : -1.0);
        if (ev == EV_ESCAPE) break;
        if (ev == EV_ABORT) { if (aborted) (*aborted)++; break; }
        int order = (int)e + 1;
        int score_it = (S->max_order == 0 || order <= S->max_order);
        rng_t rs;
        rng_init(&rs, seed, path, e, 1);
        /* the vertex draws from block 0 of its sun ray's stream (e, 1):
         * direction (words 0, 1), roulette (word 2) and the sun ray's first
         * optical depth (word 3); a learned vertex from blocks VERTEX and
         * VERTEX - 1 of the flight's stream (e, 0), its sun ray's first
         * optical depth from word 1 of the latter */
        const int learned_v = ev == EV_VOLUME && S->mlp && lv < S->n_learned;
        double uv[4], ul[4] = {0.0, 0.0, 0.0, 0.0};
        if (learned_v) {
            rng_block(&r, BLOCK_VERTEX, uv);
            rng_block(&r, BLOCK_VERTEX - 1u, ul);
        } else {
            rng_block(&rs, 0, uv);
        }
        const double sun_tau0 = -log(learned_v ? ul[1] : uv[3]);
        if (ev == EV_VOLUME) {
            const double before = score, w_vertex = w;
            double own = 0.0;
            double om = omega_at(S, k);
            if (om > 0.0) {
                double kc = k - S->k_gas - S->k_clear;
                if (kc < 0.0) kc = 0.0;
                sa += -kc / (k * om);
            }
            /* clear air with a Rayleigh phase function: the vertex's phase
             * function is the scattering-weighted mixture (used whole in
             * the local estimate); the new direction samples the species
             * first (word 0 of block VERTEX of the flight's stream), then
             * its phase function */
            const double pc = S->clear_phase == 1 ? cloud_scatter_share(S, k) : 1.0;
            if (score_it) {
                double Ts = transmissivity(S, p, s, &rs, C, sun_tau0);
                double mu = d[0] * s[0] + d[1] * s[1] + d[2] * s[2];
                double phg = orc_hg_pdf(S->g, mu);
                double ph = S->clear_phase == 1 ? pc * phg + (1.0 - pc) * orc_rayleigh_pdf(mu) : phg;
                double c = w * om * ph * Ts;
                score += c;
                own = c;
                /* d ln ph / dg: only the droplets' share depends on g */
                ds += c * (sg + pc * phg * orc_hg_dlog_dg(S->g, mu) / ph);
                da += c * sa;
            }
            w *= om;
            double nd[3];
            if (learned_v) {
                /* learned proposal: features, network, one-sample MIS */
                double x[MLP_IN], raw[MLP_OUT];
                vertex_features(S, p, d, k, vox, x);
                orc_mlp_forward(S->mlp, x, 1, raw);
                double um[4] = {uv[0], uv[1], uv[3], ul[0]};
                w *= orc_mis_sample(raw, S->g, S->mis_alpha, d, um, nd, NULL, NULL);
                if (sink) {
                    if (sink->n < sink->cap) {
                        orc_record* R = &sink->rec[sink->n];
                        R->path = path;
                        R->vertex = lv;
                        R->pad = 0;
                        for (int a = 0; a < MLP_IN; ++a) R->x[a] = x[a];
                        for (int a = 0; a < 3; ++a) R->dir[a] = nd[a];
                        R->before = before;
                        R->w_omega = w_vertex * om;
                        R->own = own;
                        R->target = 0.0;
                    }
                    sink->n++;
                }
            } else if (S->clear_phase == 1) {
                /* the direction's density is the mixture; its g-score too */
                double us[4];
                rng_block(&r, BLOCK_VERTEX, us);
                double mu = us[0] > pc ? orc_rayleigh_sample_mu(uv[0]) : orc_hg_sample_mu(S->g, uv[0]);
                rotate_dir(d, mu, 2.0 * ORC_PI * uv[1], nd);
                double phg = orc_hg_pdf(S->g, mu);
                sg += pc * phg * orc_hg_dlog_dg(S->g, mu) / (pc * phg + (1.0 - pc) * orc_rayleigh_pdf(mu));
            } else {
                double mu = orc_hg_sample_mu(S->g, uv[0]);
                double phi = 2.0 * ORC_PI * uv[1];
                rotate_dir(d, mu, phi, nd);
                sg += orc_hg_dlog_dg(S->g, mu);
            }
            ++lv;
            d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
        } else if (!S->hf) { /* flat ground */
            if (score_it) {
                double Ts = transmissivity(S, p, s, &rs, C, sun_tau0);
                double c = w * (S->ground_albedo / ORC_PI) * fmax(s[2], 0.0) * Ts;
                score += c;
                ds += c * sg;
                da += c * sa;
            }
            w *= S->ground_albedo;
            cosine_up(uv[0], uv[1], d);
        } else { /* heightfield: leave the surface along its normal, cosine about it */
            for (int a = 0; a < 3; ++a) p[a] += ORC_TERRAIN_OFFSET * ng[a];
            wrap_xy(S, p);
            if (score_it) {
                double ns = ng[0] * s[0] + ng[1] * s[1] + ng[2] * s[2];
                double Ts = ns > 0.0 ? transmissivity(S, p, s, &rs, C, sun_tau0) : 0.0;
                double c = w * (S->ground_albedo / ORC_PI) * fmax(ns, 0.0) * Ts;
                score += c;
                ds += c * sg;
                da += c * sa;
            }
            w *= S->ground_albedo;
            cosine_about(ng, uv[0], uv[1], d);
        }
        if (S->max_order > 0 && order >= S->max_order) break;
        if (w < 0.01) {
            if (uv[2] * 0.01 <= w) w = 0.01;
            else break;
        }
    }
    if (dscore) *dscore = ds;
    if (dalpha) *dalpha = da;
    if (sink) {
        /* targets: what the path scored after each learned vertex, per unit w * omega */
        for (int64_t i = rec0; i < sink->n && i < sink->cap; ++i) {
            orc_record* R = &sink->rec[i];
            R->target = R->w_omega > 0.0 ? (score - R->before - R->own) / R->w_omega : 0.0;
        }
    }
    return score;
}

/* ===================================================================== */
/* Sensors.                                                               */
/* ===================================================================== */
typedef struct {
    double pos[3], target[3], up[3];
    double fov_deg;                 /* horizontal field of view */
    int32_t width, height;
} orc_camera;

static void cam_basis(const orc_camera* C, double f[3], double rt[3], double u[3])
{
    double n;
    for (int a = 0; a < 3; ++a) f[a] = C->target[a] - C->pos[a];
    n = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int a = 0; a < 3; ++a) f[a] /= n;
    rt[0] = f[1] * C->up[2] - f[2] * C->up[1];
    rt[1] = f[2] * C->up[0] - f[0] * C->up[2];
    rt[2] = f[0] * C->up[1] - f[1] * C->up[0];
    n = sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
    for (int a = 0; a < 3; ++a) rt[a] /= n;
    u[0] = rt[1] * f[2] - rt[2] * f[1];
    u[1] = rt[2] * f[0] - rt[0] * f[2];
    u[2] = rt[0] * f[1] - rt[1] * f[0];
}

/* Wrap x, y into [0, L). */
static void wrap_xy(const orc_scene* S, double p[3])
{
    double Lx = (double)S->nx * S->dx, Ly = (double)S->ny * S->dy;
    p[0] -= floor(p[0] / Lx) * Lx;
    p[1] -= floor(p[1] / Ly) * Ly;
    if (p[0] >= Lx) p[0] = 0.0;
    if (p[1] >= Ly) p[1] = 0.0;
}

/* One camera path (Sec. 4.1: pinhole camera, direction jittered in the
 * pixel).  Stream (0, 2) gives the two jitter draws. */
static double camera_path_r(const orc_scene* S, const orc_camera* C, uint32_t spp, uint64_t seed, uint64_t path,
                            orc_counts* cnt, int64_t* aborted, orc_rec_sink* sink);

static double camera_path(const orc_scene* S, const orc_camera* C, uint32_t spp, uint64_t seed, uint64_t path,
                          orc_counts* cnt, int64_t* aborted)
{
    return camera_path_r(S, C, spp, seed, path, cnt, aborted, NULL);
}

static double camera_path_r(const orc_scene* S, const orc_camera* C, uint32_t spp, uint64_t seed, uint64_t path,
                            orc_counts* cnt, int64_t* aborted, orc_rec_sink* sink)
{
    uint64_t pix = path / spp;
    int px = (int)(pix % (uint64_t)C->width), py = (int)(pix / (uint64_t)C->width);
    rng_t r;
    rng_init(&r, seed, path, 0, 2);
    double uj[4];
    rng_block(&r, 0, uj);
    double jx = 1.0 - uj[0], jy = 1.0 - uj[1];
    double f[3], rt[3], u[3];
    cam_basis(C, f, rt, u);
    double tanh_ = tan(0.5 * C->fov_deg * ORC_PI / 180.0);
    double sx = (2.0 * (px + jx) / C->width - 1.0) * tanh_;
    double sy = (2.0 * (py + jy) / C->height - 1.0) * tanh_ * (double)C->height / (double)C->width;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = f[a] + sx * rt[a] + sy * u[a];
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) d[a] /= n;
    double p[3] = {C->pos[0], C->pos[1], C->pos[2]};
    double Lz = (double)S->nz * S->dz;
    if (p[2] > Lz) {
        if (d[2] >= 0.0) return 0.0;
        double t = (Lz - p[2]) / d[2];
        for (int a = 0; a < 2; ++a) p[a] += t * d[a];
        p[2] = Lz;
    } else if (p[2] < 0.0) {
        return 0.0;
    }
    wrap_xy(S, p);
    /* the first flight's optical depth: word 2 of the path-start block */
    return trace_backward_r(S, p, d, seed, path, cnt, aborted, NULL, NULL, sink, -log(uj[2]));
}

/* One ground-flux path: uniform ground point, cosine-weighted upward
 * direction (stream (0, 2): four draws); direct part from stream (0, 3).
 * out[0] = T_dir, out[1] = T_dif = pi / mu0 * sum of local estimates. */
static void flux_path_r(const orc_scene* S, uint64_t seed, uint64_t path, double out[4],
                        orc_counts* cnt, int64_t* aborted, orc_rec_sink* sink);

static void flux_path(const orc_scene* S, uint64_t seed, uint64_t path, double out[4],
                      orc_counts* cnt, int64_t* aborted)
{
    flux_path_r(S, seed, path, out, cnt, aborted, NULL);
}

static void flux_path_r(const orc_scene* S, uint64_t seed, uint64_t path, double out[4],
                        orc_counts* cnt, int64_t* aborted, orc_rec_sink* sink)
{
    rng_t r;
    rng_init(&r, seed, path, 0, 2);
    double u[4];
    rng_block(&r, 0, u);
    double u0 = u[0], u1 = u[1], u2 = u[2], u3 = u[3];
    double Lx = (double)S->nx * S->dx, Ly = (double)S->ny * S->dy;
    double p[3] = {(1.0 - u0) * Lx, (1.0 - u1) * Ly, 0.0};
    double d[3];
    rng_t rd;
    rng_init(&rd, seed, path, 0, 3);
    double mu0 = S->sun[2];
    if (S->hf) {
        /* heightfield: the point on the surface above (x, y), directions
         * cosine-weighted about its normal n; irradiance of the tilted
         * element per unit horizontal area: direct max(n.s, 0) / (n_z mu0)
         * T_sun, diffuse pi / (n_z mu0) times the local estimates */
        double n[3];
        p[2] = orc_terrain_height(S, p[0], p[1], n);
        for (int a = 0; a < 3; ++a) p[a] += ORC_TERRAIN_OFFSET * n[a];
        wrap_xy(S, p);
        cosine_about(n, u2, u3, d);
        double ns = n[0] * S->sun[0] + n[1] * S->sun[1] + n[2] * S->sun[2];
        double q[3] = {p[0], p[1], p[2]};
        double Tdir = ns > 0.0 ? transmissivity(S, q, S->sun, &rd, cnt, -1.0) : 0.0;
        double dsc = 0.0, dal = 0.0;
        double score = trace_backward_d(S, p, d, seed, path, cnt, aborted, &dsc, &dal);
        out[0] = fmax(ns, 0.0) / (n[2] * mu0) * Tdir;
        out[1] = ORC_PI / (n[2] * mu0) * score;
        out[2] = ORC_PI / (n[2] * mu0) * dsc;
        out[3] = ORC_PI / (n[2] * mu0) * dal;
        return;
    }
    cosine_up(u2, u3, d);
    double q[3] = {p[0], p[1], p[2]};
    double Tdir = transmissivity(S, q, S->sun, &rd, cnt, -1.0);
    double dsc = 0.0, dal = 0.0;
    double score = trace_backward_r(S, p, d, seed, path, cnt, aborted, &dsc, &dal, sink, -1.0);
    out[0] = Tdir;
    out[1] = ORC_PI / mu0 * score;
    out[2] = ORC_PI / mu0 * dsc;
    out[3] = ORC_PI / mu0 * dal;
}

/* ===================================================================== */
/* Forward analog flux (Sec. 5.2): photons enter uniformly at the top     */
/* along -s; weights carry absorption (w *= omega, w *= rho); arrivals    */
/* at the ground are direct until the photon has been scattered or        */
/* reflected once.  Used as an independent cross-check of the backward   */
/* estimator and for the energy balance R + T_abs + A = 1.                */
/* out per photon: [0] R (escape weight), [1] T_dir arrivals,             */
/* [2] T_dif arrivals, [3] volume absorption, [4] ground absorption,      */
/* [5] weight left at cutoff.                                             */
/* ===================================================================== */
static void forward_photon(const orc_scene* S, uint64_t seed, uint64_t path, double out[6], int64_t* aborted)
{
    for (int i = 0; i < 6; ++i) out[i] = 0.0;
    rng_t r0;
    rng_init(&r0, seed, path, 0, 2);
    double u0[4];
    rng_block(&r0, 0, u0);
    double Lx = (double)S->nx * S->dx, Ly = (double)S->ny * S->dy, Lz = (double)S->nz * S->dz;
    double p[3] = {(1.0 - u0[0]) * Lx, (1.0 - u0[1]) * Ly, Lz};
    double d[3] = {-S->sun[0], -S->sun[1], -S->sun[2]};
    double w = 1.0;
    int scattered = 0;
    for (uint32_t e = 0;; ++e) {
        rng_t r;
        rng_init(&r, seed, path, e, 0);
        double k;
        int ev = free_flight(S, p, d, &r, &k, NULL, NULL, NULL, -1.0);
        if (ev == EV_ESCAPE) { out[0] += w; return; }
        if (ev == EV_ABORT) { if (aborted) (*aborted)++; out[5] += w; return; }
        double uv[4];
        rng_block(&r, BLOCK_VERTEX, uv);
        if (ev == EV_VOLUME) {
            double om = omega_at(S, k);
            out[3] += w * (1.0 - om);
            w *= om;
            double mu = orc_hg_sample_mu(S->g, uv[0]);
            double phi = 2.0 * ORC_PI * uv[1];
            double nd[3];
            rotate_dir(d, mu, phi, nd);
            d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
            scattered = 1;
        } else {
            if (scattered) out[2] += w; else out[1] += w;
            out[4] += w * (1.0 - S->ground_albedo);
            w *= S->ground_albedo;
            cosine_up(uv[0], uv[1], d);
            scattered = 1;
        }
        if (w < 1e-6) { out[5] += w; return; }
    }
}

/* ===================================================================== */
/* Parallel drivers (pthreads).  Work is cut into fixed blocks whose       */
/* partial sums are combined in block order, so results do not depend on  */
/* the number of threads.                                                 */
/* ===================================================================== */
typedef struct {
    const orc_scene* S;
    const orc_camera* C;
    int kind;             /* 0 camera, 1 flux, 2 forward */
    uint32_t spp;
    uint64_t seed;
    uint64_t begin, end;  /* path ids */
    uint64_t block;       /* paths per block */
    int64_t nblocks;
    double* out;          /* per block partial sums (kind-dependent)  */
    int64_t* aborted;     /* per block */
    orc_counts* counts;   /* per block */
    int64_t next;         /* next block (protected by mu) */
    pthread_mutex_t mu;
} job_t;

static void run_block(job_t* J, int64_t b)
{
    uint64_t p0 = J->begin + (uint64_t)b * J->block;
    uint64_t p1 = p0 + J->block;
    if (p1 > J->end) p1 = J->end;
    int64_t ab = 0;
    orc_counts cnt = {0, 0, 0};
    if (J->kind == 0) {
        /* camera: the block is a set of whole pixels; out is per pixel */
        for (uint64_t path = p0; path < p1; ++path) {
            uint64_t pix = path / J->spp;
            double sc = camera_path(J->S, J->C, J->spp, J->seed, path, &cnt, &ab);
            J->out[2 * pix + 0] += sc;
            J->out[2 * pix + 1] += sc * sc;
        }
    } else if (J->kind == 1) {
        double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (uint64_t path = p0; path < p1; ++path) {
            double o[4];
            flux_path(J->S, J->seed, path, o, &cnt, &ab);
            double tot = o[0] + o[1];
            acc[0] += o[0]; acc[1] += o[0] * o[0];
            acc[2] += o[1]; acc[3] += o[1] * o[1];
            acc[4] += tot;  acc[5] += tot * tot;
            acc[6] += o[2]; acc[7] += o[2] * o[2];
            acc[8] += o[3]; acc[9] += o[3] * o[3];
        }
        for (int i = 0; i < 10; ++i) J->out[10 * b + i] = acc[i];
    } else {
        double acc[12];
        for (int i = 0; i < 12; ++i) acc[i] = 0.0;
        for (uint64_t path = p0; path < p1; ++path) {
            double o[6];
            forward_photon(J->S, J->seed, path, o, &ab);
            for (int i = 0; i < 6; ++i) { acc[2 * i] += o[i]; acc[2 * i + 1] += o[i] * o[i]; }
        }
        for (int i = 0; i < 12; ++i) J->out[12 * b + i] = acc[i];
    }
    J->aborted[b] = ab;
    J->counts[b] = cnt;
}

static void* worker(void* arg)
{
    job_t* J = (job_t*)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t b = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (b >= J->nblocks) return NULL;
        run_block(J, b);
    }
}

static void run_job(job_t* J, int nthreads)
{
    pthread_mutex_init(&J->mu, NULL);
    J->next = 0;
    if (nthreads < 1) nthreads = 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, worker, J);
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&J->mu);
}

/* Camera: paths [pix_begin*spp, pix_end*spp); sums (2 per pixel of the
 * whole image, only the range is touched); stats[0] aborted paths,
 * stats[1..3] tentative collisions, real collisions, leaf steps. */
int orc_trace_camera(const orc_scene* S, const orc_camera* C, uint32_t spp, uint64_t seed,
                     int64_t pix_begin, int64_t pix_end, double* sums, int nthreads, int64_t* stats)
{
    if (spp == 0 || pix_end < pix_begin) return -1;
    job_t J;
    memset(&J, 0, sizeof(J));
    J.S = S; J.C = C; J.kind = 0; J.spp = spp; J.seed = seed;
    J.begin = (uint64_t)pix_begin * spp; J.end = (uint64_t)pix_end * spp;
    J.block = spp;                      /* one pixel per block */
    J.nblocks = pix_end - pix_begin;
    J.out = sums;
    J.aborted = (int64_t*)calloc((size_t)(J.nblocks + 1), sizeof(int64_t));
    J.counts = (orc_counts*)calloc((size_t)(J.nblocks + 1), sizeof(orc_counts));
    run_job(&J, nthreads);
    int64_t ab = 0; orc_counts tot = {0, 0, 0};
    for (int64_t b = 0; b < J.nblocks; ++b) {
        ab += J.aborted[b];
        tot.tentative += J.counts[b].tentative; tot.real += J.counts[b].real; tot.leaves += J.counts[b].leaves;
    }
    if (stats) { stats[0] = ab; stats[1] = tot.tentative; stats[2] = tot.real; stats[3] = tot.leaves; }
    free(J.aborted); free(J.counts);
    return 0;
}

/* Flux: paths [begin, end); sums[10] = (sum, sum^2) of T_dir, T_dif, T_tot,
 * dT/dg (score-function derivative with respect to the HG asymmetry), dT/dalpha
 * (derivative with respect to the cloud droplets' absorptivity). */
int orc_trace_flux(const orc_scene* S, uint64_t seed, uint64_t begin, uint64_t end, double* sums,
                   int nthreads, int64_t* stats)
{
    if (end < begin) return -1;
    job_t J;
    memset(&J, 0, sizeof(J));
    J.S = S; J.kind = 1; J.seed = seed; J.begin = begin; J.end = end;
    J.block = 1024;
    J.nblocks = (int64_t)((end - begin + J.block - 1) / J.block);
    J.out = (double*)calloc((size_t)(10 * J.nblocks + 10), sizeof(double));
    J.aborted = (int64_t*)calloc((size_t)(J.nblocks + 1), sizeof(int64_t));
    J.counts = (orc_counts*)calloc((size_t)(J.nblocks + 1), sizeof(orc_counts));
    run_job(&J, nthreads);
    for (int i = 0; i < 10; ++i) sums[i] = 0.0;
    int64_t ab = 0; orc_counts tot = {0, 0, 0};
    for (int64_t b = 0; b < J.nblocks; ++b) {
        for (int i = 0; i < 10; ++i) sums[i] += J.out[10 * b + i];
        ab += J.aborted[b];
        tot.tentative += J.counts[b].tentative; tot.real += J.counts[b].real; tot.leaves += J.counts[b].leaves;
    }
    if (stats) { stats[0] = ab; stats[1] = tot.tentative; stats[2] = tot.real; stats[3] = tot.leaves; }
    free(J.out); free(J.aborted); free(J.counts);
    return 0;
}

/* Online-training records of the learned proposal (see orc_record) for
 * camera paths [begin, end) of a spp-per-pixel image (C != NULL) or for
 * ground-flux paths [begin, end) (C == NULL), traced one after another in
 * path order with the scene's network; at most cap records are stored,
 * scores[i] (may be NULL) receives path begin + i's backward score (the
 * sum of its local estimates).  Returns the number of records the paths
 * produced (all of them, also beyond cap). */
int64_t orc_learned_records(const orc_scene* S, const orc_camera* C, uint32_t spp, uint64_t seed, uint64_t begin,
                            uint64_t end, orc_record* out, int64_t cap, double* scores)
{
    if (!S->mlp || end < begin || (C && spp == 0)) return -1;
    orc_rec_sink sink = {out, cap, 0};
    orc_counts cnt = {0, 0, 0};
    int64_t ab = 0;
    for (uint64_t path = begin; path < end; ++path) {
        double sc;
        if (C) {
            sc = camera_path_r(S, C, spp, seed, path, &cnt, &ab, &sink);
        } else {
            double o[4];
            flux_path_r(S, seed, path, o, &cnt, &ab, &sink);
            sc = o[1] * S->sun[2] / ORC_PI;
        }
        if (scores) scores[path - begin] = sc;
    }
    return sink.n;
}

/* Forward analog: sums[12] = (sum, sum^2) of R, T_dir, T_dif, A_vol,
 * A_ground, cutoff weight, per photon. */
int orc_trace_forward(const orc_scene* S, uint64_t seed, uint64_t begin, uint64_t end, double* sums,
                      int nthreads, int64_t* stats)
{
    if (end < begin || S->hf) return -1;      /* the forward photon knows the flat ground only */
    job_t J;
    memset(&J, 0, sizeof(J));
    J.S = S; J.kind = 2; J.seed = seed; J.begin = begin; J.end = end;
    J.block = 1024;
    J.nblocks = (int64_t)((end - begin + J.block - 1) / J.block);
    J.out = (double*)calloc((size_t)(12 * J.nblocks + 12), sizeof(double));
    J.aborted = (int64_t*)calloc((size_t)(J.nblocks + 1), sizeof(int64_t));
    J.counts = (orc_counts*)calloc((size_t)(J.nblocks + 1), sizeof(orc_counts));
    run_job(&J, nthreads);
    for (int i = 0; i < 12; ++i) sums[i] = 0.0;
    int64_t ab = 0;
    for (int64_t b = 0; b < J.nblocks; ++b) {
        for (int i = 0; i < 12; ++i) sums[i] += J.out[12 * b + i];
        ab += J.aborted[b];
    }
    if (stats) stats[0] = ab;
    free(J.out); free(J.aborted); free(J.counts);
    return 0;
}

/* Per-photon energy balance check: returns max over photons of
 * |R + A_vol + A_ground + T_abs_part... - 1|, where the ground arrival
 * weight splits into absorbed and reflected parts.  Used by the
 * R + T + A = 1 pin (weights are exact, so the residual is rounding). */
double orc_forward_balance_residual(const orc_scene* S, uint64_t seed, uint64_t begin, uint64_t end)
{
    double worst = 0.0;
    for (uint64_t p = begin; p < end; ++p) {
        double o[6];
        forward_photon(S, seed, p, o, NULL);
        double res = fabs(o[0] + o[3] + o[4] + o[5] - 1.0);
        if (res > worst) worst = res;
    }
    return worst;
}

/* ===================================================================== */
/* Learned scattering proposal (no counterpart in the paper).             */
/* A multilayer perceptron maps 9 vertex features to an 8-lobe von       */
/* Mises-Fisher mixture; directions are drawn by defensive one-sample     */
/* multiple importance sampling with the HG phase function:               */
/*   q(w') = alpha p_HG(d.w') + (1 - alpha) sum_j pi_j f_j(w'),           */
/* and the path weight is multiplied by p_HG(d.w') / q(w'), which keeps   */
/* the estimator unbiased for any network.                                */
/* Parameter vector (11,560 doubles): W1[64][9], b1[64], W2[64][64],      */
/* b2[64], W3[64][64], b3[64], W4[40][64], b4[40] (row = output unit).    */
/* Outputs per lobe j: mu~ (3), kappa raw, logit.  GELU: tanh form.       */
/* ===================================================================== */
#define MLP_H 64
#define MLP_LOBES 8
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_OUT * MLP_H + MLP_OUT)

int orc_mlp_nparam(void) { return MLP_NPARAM; }

static double gelu(double x)
{
    const double c = 0.7978845608028654; /* sqrt(2/pi) */
    return 0.5 * x * (1.0 + tanh(c * (x + 0.044715 * x * x * x)));
}

static double gelu_grad(double x)
{
    const double c = 0.7978845608028654;
    double u = c * (x + 0.044715 * x * x * x);
    double t = tanh(u);
    double du = c * (1.0 + 3.0 * 0.044715 * x * x);
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * du;
}

/* One dense layer y = W x + b (W row-major [nout][nin]). */
static void dense(const double* W, const double* b, const double* x, int nin, int nout, double* y)
{
    for (int o = 0; o < nout; ++o) {
        double s = b[o];
        for (int i = 0; i < nin; ++i) s += W[o * nin + i] * x[i];
        y[o] = s;
    }
}

typedef struct { const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4; } mlp_view;

static mlp_view mlp_split(const double* p)
{
    mlp_view v;
    v.W1 = p; p += MLP_H * MLP_IN;
    v.b1 = p; p += MLP_H;
    v.W2 = p; p += MLP_H * MLP_H;
    v.b2 = p; p += MLP_H;
    v.W3 = p; p += MLP_H * MLP_H;
    v.b3 = p; p += MLP_H;
    v.W4 = p; p += MLP_OUT * MLP_H;
    v.b4 = p;
    return v;
}

/* Forward pass of one row; z[3][64] pre-activations and h[3][64]
 * activations are returned for the backward pass when non-NULL. */
static void mlp_row(const mlp_view* v, const double* x, double* out, double z[3][MLP_H], double h[3][MLP_H])
{
    double zz[3][MLP_H], hh[3][MLP_H];
    dense(v->W1, v->b1, x, MLP_IN, MLP_H, zz[0]);
    for (int i = 0; i < MLP_H; ++i) hh[0][i] = gelu(zz[0][i]);
    dense(v->W2, v->b2, hh[0], MLP_H, MLP_H, zz[1]);
    for (int i = 0; i < MLP_H; ++i) hh[1][i] = gelu(zz[1][i]);
    dense(v->W3, v->b3, hh[1], MLP_H, MLP_H, zz[2]);
    for (int i = 0; i < MLP_H; ++i) hh[2][i] = gelu(zz[2][i]);
    dense(v->W4, v->b4, hh[2], MLP_H, MLP_OUT, out);
    if (z) memcpy(z, zz, sizeof(zz));
    if (h) memcpy(h, hh, sizeof(hh));
}

void orc_mlp_forward(const double* params, const double* x, int64_t rows, double* out)
{
    mlp_view v = mlp_split(params);
    for (int64_t r = 0; r < rows; ++r) mlp_row(&v, x + MLP_IN * r, out + MLP_OUT * r, NULL, NULL);
}

static double softplus(double x) { return x > 30.0 ? x : log1p(exp(x)); }

/* Mixture parameters from the 40 raw outputs: unit axes, concentrations
 * kappa = softplus + 1e-3, weights = softmax of the logits. */
void orc_mixture(const double* raw, double mu[MLP_LOBES][3], double kappa[MLP_LOBES], double pi[MLP_LOBES])
{
    double mx = -INFINITY;
    for (int j = 0; j < MLP_LOBES; ++j) if (raw[5 * j + 4] > mx) mx = raw[5 * j + 4];
    double s = 0.0;
    for (int j = 0; j < MLP_LOBES; ++j) {
        const double* q = raw + 5 * j;
        double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (n < 1e-12) { mu[j][0] = 0.0; mu[j][1] = 0.0; mu[j][2] = 1.0; }
        else { mu[j][0] = q[0] / n; mu[j][1] = q[1] / n; mu[j][2] = q[2] / n; }
        kappa[j] = softplus(q[3]) + 1e-3;
        pi[j] = exp(q[4] - mx);
        s += pi[j];
    }
    for (int j = 0; j < MLP_LOBES; ++j) pi[j] /= s;
}

/* vMF density over the sphere, kappa / (2 pi (1 - exp(-2 kappa))) exp(kappa (mu.x - 1)). */
double orc_vmf_pdf(const double mu[3], double kappa, const double x[3])
{
    double c = mu[0] * x[0] + mu[1] * x[1] + mu[2] * x[2];
    return kappa / (2.0 * ORC_PI * (-expm1(-2.0 * kappa))) * exp(kappa * (c - 1.0));
}

/* vMF sample (Wood 1994): cosine w = 1 + ln(xi + (1 - xi) exp(-2 kappa)) / kappa. */
void orc_vmf_sample(const double mu[3], double kappa, double xi1, double xi2, double out[3])
{
    double w = 1.0 + log(xi1 + (1.0 - xi1) * exp(-2.0 * kappa)) / kappa;
    if (w > 1.0) w = 1.0;
    if (w < -1.0) w = -1.0;
    rotate_dir(mu, w, 2.0 * ORC_PI * xi2, out);
}

static double mixture_pdf(double mu[MLP_LOBES][3], const double kappa[MLP_LOBES], const double pi[MLP_LOBES],
                          const double x[3])
{
    double q = 0.0;
    for (int j = 0; j < MLP_LOBES; ++j) q += pi[j] * orc_vmf_pdf(mu[j], kappa[j], x);
    return q;
}

/* One-sample MIS direction at a vertex with incoming direction d.
 * u[0]: HG cosine or vMF cosine draw, u[1]: azimuth, u[2]: HG-vs-mixture
 * choice (HG when u[2] <= alpha), u[3]: lobe choice.  Returns the weight
 * factor p_HG / q; *q_out and *phg_out receive q(w') and p_HG(d.w'). */
double orc_mis_sample(const double* raw, double g, double alpha, const double d[3], const double u[4], double out[3],
                      double* q_out, double* phg_out)
{
    double mu[MLP_LOBES][3], kappa[MLP_LOBES], pi[MLP_LOBES];
    orc_mixture(raw, mu, kappa, pi);
    if (u[2] <= alpha) {
        rotate_dir(d, orc_hg_sample_mu(g, u[0]), 2.0 * ORC_PI * u[1], out);
    } else {
        int j = MLP_LOBES - 1;
        double c = 0.0;
        for (int i = 0; i < MLP_LOBES; ++i) {
            c += pi[i];
            if (u[3] <= c) { j = i; break; }
        }
        orc_vmf_sample(mu[j], kappa[j], u[0], u[1], out);
    }
    double phg = orc_hg_pdf(g, d[0] * out[0] + d[1] * out[1] + d[2] * out[2]);
    double q = alpha * phg + (1.0 - alpha) * mixture_pdf(mu, kappa, pi, out);
    if (q_out) *q_out = q;
    if (phg_out) *phg_out = phg;
    return phg / q;
}

double orc_mixture_pdf(const double* raw, const double x[3])
{
    double mu[MLP_LOBES][3], kappa[MLP_LOBES], pi[MLP_LOBES];
    orc_mixture(raw, mu, kappa, pi);
    return mixture_pdf(mu, kappa, pi, x);
}

/* Loss over `rows` training records: mean of -t_r log q_vMF(w'_r), where
 * t_r is the record's target weight (the radiance the sampled direction
 * brought back, weighted so that the expectation is the KL divergence
 * between the ideal product p_HG L and the mixture, up to a constant).
 * x: rows x 9 features, dir: rows x 3 directions, t: rows targets.
 * grad (11,560) receives d loss / d params; returns the loss. */
double orc_mlp_loss_grad(const double* params, const double* x, const double* dir, const double* t, int64_t rows,
                         double* grad)
{
    mlp_view v = mlp_split(params);
    memset(grad, 0, sizeof(double) * MLP_NPARAM);
    double* gW1 = grad;
    double* gb1 = gW1 + MLP_H * MLP_IN;
    double* gW2 = gb1 + MLP_H;
    double* gb2 = gW2 + MLP_H * MLP_H;
    double* gW3 = gb2 + MLP_H;
    double* gb3 = gW3 + MLP_H * MLP_H;
    double* gW4 = gb3 + MLP_H;
    double* gb4 = gW4 + MLP_OUT * MLP_H;
    double loss = 0.0;
    const double inv_rows = 1.0 / (double)rows;
    for (int64_t r = 0; r < rows; ++r) {
        const double* xr = x + MLP_IN * r;
        const double* w = dir + 3 * r;
        double out[MLP_OUT], z[3][MLP_H], h[3][MLP_H];
        mlp_row(&v, xr, out, z, h);
        double mu[MLP_LOBES][3], kappa[MLP_LOBES], pi[MLP_LOBES], f[MLP_LOBES];
        orc_mixture(out, mu, kappa, pi);
        double q = 0.0;
        for (int j = 0; j < MLP_LOBES; ++j) { f[j] = orc_vmf_pdf(mu[j], kappa[j], w); q += pi[j] * f[j]; }
        const double tr = t[r] * inv_rows;
        loss += -tr * log(q);
        /* d(-t log q)/d raw */
        double dout[MLP_OUT];
        for (int j = 0; j < MLP_LOBES; ++j) {
            const double* raw = out + 5 * j;
            double resp = pi[j] * f[j] / q;                     /* responsibility */
            double n = sqrt(raw[0] * raw[0] + raw[1] * raw[1] + raw[2] * raw[2]);
            double c = mu[j][0] * w[0] + mu[j][1] * w[1] + mu[j][2] * w[2];
            double k = kappa[j];
            /* d log f / d mu~ = kappa (w - (mu.w) mu) / |mu~| */
            for (int a = 0; a < 3; ++a) {
                double dmu = (n < 1e-12) ? 0.0 : k * (w[a] - c * mu[j][a]) / n;
                dout[5 * j + a] = -tr * resp * dmu;
            }
            /* d log f / d kappa = 1/kappa - 2 e^{-2k} / (1 - e^{-2k}) + (c - 1) */
            double e2 = exp(-2.0 * k);
            double dk = 1.0 / k - 2.0 * e2 / (-expm1(-2.0 * k)) + (c - 1.0);
            double sig = 1.0 / (1.0 + exp(-raw[3]));             /* softplus' */
            dout[5 * j + 3] = -tr * resp * dk * sig;
            dout[5 * j + 4] = -tr * (resp - pi[j]);
        }
        /* backward through the layers */
        double dh[MLP_H], dz[MLP_H], dprev[MLP_H];
        for (int o = 0; o < MLP_OUT; ++o) {
            gb4[o] += dout[o];
            for (int i = 0; i < MLP_H; ++i) gW4[o * MLP_H + i] += dout[o] * h[2][i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double s = 0.0;
            for (int o = 0; o < MLP_OUT; ++o) s += v.W4[o * MLP_H + i] * dout[o];
            dh[i] = s;
        }
        const double* Ws[3] = {v.W1, v.W2, v.W3};
        double* gWs[3] = {gW1, gW2, gW3};
        double* gbs[3] = {gb1, gb2, gb3};
        for (int L = 2; L >= 0; --L) {
            int nin = (L == 0) ? MLP_IN : MLP_H;
            const double* inp = (L == 0) ? xr : h[L - 1];
            for (int o = 0; o < MLP_H; ++o) dz[o] = dh[o] * gelu_grad(z[L][o]);
            for (int o = 0; o < MLP_H; ++o) {
                gbs[L][o] += dz[o];
                for (int i = 0; i < nin; ++i) gWs[L][o * nin + i] += dz[o] * inp[i];
            }
            if (L > 0) {
                for (int i = 0; i < MLP_H; ++i) {
                    double s = 0.0;
                    for (int o = 0; o < MLP_H; ++o) s += Ws[L][o * MLP_H + i] * dz[o];
                    dprev[i] = s;
                }
                memcpy(dh, dprev, sizeof(dh));
            }
        }
    }
    return loss;
}

/* Adam (Kingma and Ba 2015) with bias correction; step t >= 1. */
void orc_adam_step(double* params, double* m, double* v, const double* grad, int64_t n, int64_t t, double lr,
                   double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        params[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
