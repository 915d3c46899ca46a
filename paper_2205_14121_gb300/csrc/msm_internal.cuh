// Internal declarations of libmsm: system state, device helpers, kernel entry
// points shared between the translation units.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "msm.h"

#define MSM_TPB 256

// ---------------------------------------------------------------------------
// control words (device int32 array), see md_system::ctl
// ---------------------------------------------------------------------------
enum {
    CTL_REBUILD = 0,     // displacement check tripped / build requested
    CTL_OVERFLOW = 1,    // bit per list kind
    CTL_UNSTABLE = 2,    // NaN/Inf or escape seen by the integrator
    CTL_NPLT = 3,        // subset compaction counters
    CTL_NREC = 4,
    CTL_NFAST = 5,       // plasma particles listed for the fast-particle pair pass
    CTL_MAXROW = 8,      // 4 slots: longest row per list kind (this build)
    CTL_WORDS = 16
};

// Step-dependent values read by the kernels; written on the device so that a
// captured multi-step graph needs no host updates.
struct md_dstate {
    int64_t step;        // completed fluid steps n
    int32_t sub;         // completed interface substeps c within the step
    int32_t pad;
    double  time;        // n dt + c dt_m
    double  le_offset;   // Lees-Edwards image offset in [0, Lx)
    float   le_offset_f; // its FP32 copy
    float   le_build_f;  // offset at the last list build
    int64_t n_builds;
    int64_t steps_left;  // countdown of a captured loop
    int64_t base;        // fluid steps completed when the current outer step began
    int64_t done;        // outer steps begun (next base)
    int64_t ring_count;  // per-platelet feature records appended so far
    uint32_t fast_stamp; // marks the particles of the current fast list (fast_flag)
    uint32_t pad2;
};

struct md_grid {
    int   nc[3];
    float lo[3];
    float h[3];
    float inv_h[3];
    int64_t ncell;
    int32_t *start;  // ncell + 1
    int32_t *count;  // ncell
};

struct md_geom {
    float L[3], hL[3];
    int   walls, le;
    float shear_v;   // shear_rate * Ly (image velocity jump)
};

struct md_system {
    md_config cfg;
    cudaStream_t stream;
    int device;
    std::string err;

    int64_t n, n_plt, n_rec, nb;
    int cap[4];

    // particle arrays (cell-sorted)
    double *xs, *ys, *zs;        // FP64 master positions
    float4 *x32;                 // xyz + id bits
    float4 *v;                   // v + tag bits
    float4 *f[3];                // level forces (fluid, iface, platelet)
    float4 *xb;                  // positions at the last build
    // plasma particles that moved beyond skin/2 (but within the skin) since
    // the build: their pairs missing from the lists are evaluated by a pass
    // of their own instead of a rebuild
    int32_t *fast_idx;           // [fast_max] slots
    uint32_t *fast_flag;         // [n] == ds->fast_stamp: listed now
    int64_t fast_max;
    // deterministic mode (MD_FORCE_DETERMINISTIC): fixed-point sums per level
    unsigned long long *fdet[3];  // [3 n] each
    unsigned det_levels = 0;      // levels of the last deterministic md_forces (0: none current)
    bool det_step = false;        // md_mts_step with MD_SCHED_DETERMINISTIC: every force from fixed-point sums
    int32_t *tag_s;              // tags in sorted order
    int32_t *cellid, *slot, *perm, *pos_of_id;
    double *alt64;               // 3n
    float4 *altv, *altx, *altf[3];
    int32_t *alt_tag;
    int32_t *tag_id;             // tags in id order, as last given to md_set_particles
    float4 *X0;                  // rest positions, id order

    // grids
    md_grid gmain, gplt, grec;

    // subsets
    int32_t *plt_idx, *plt_sorted, *plt_cell, *plt_slot;
    int32_t *rec_idx, *rec_sorted, *rec_cell, *rec_slot;

    // lists (row-major ELL: entry k of row r at r*cap + k)
    int32_t *nl[4], *nc[4];

    // bonds (stored grouped by platelet: bonds of p are [bond_off[p], bond_off[p+1]))
    int32_t *bond_id, *bond_ij;
    float *bond_r0;
    // angle triplets (ids; slots remapped at each sort) and rest angles
    int64_t na = 0;
    int32_t *angle_id = nullptr, *angle_ijk = nullptr;
    float *angle_t0 = nullptr;
    int2 *bond_blk = nullptr, *angle_blk = nullptr;   // per block of MSM_TPB terms: first and last platelet
    // AI-MTS: step ratios (bit k - 1) of the platelets each platelet has LJ
    // or receptor pairs with, and its drift stride on the K-substep grid
    unsigned long long *plt_cmask = nullptr;
    int32_t *plt_stride = nullptr;
    int32_t *plt_row_stride = nullptr;   // the stride of each platelet row (plt_sorted order)
    bool have_angles = false;

    // per-platelet measurements (K8)
    int32_t *plt_off, *plt_ids;  // member ids of platelet p: plt_ids[plt_off[p] .. plt_off[p+1])
    int32_t *bond_off;
    int32_t *plt_contacts;
    float4 *plt_bound;           // per platelet at the last build: centre of mass, radius
    double *feat_sums;           // [P][25] FP64 partial sums of the measurements, then [P] strain bits
    int32_t *plt_near;           // bit 0 / 1: another platelet within LJ / Morse reach
    int2 *cell_pid;              // per platelet (receptor) sub-grid cell: lowest, highest platelet id
    double *feat;                // [P][12]
    float *ring;                 // [P][ring_T][12] time series of the measurements
    int ring_T = 128;
    std::vector<int32_t> h_tag;  // tags in id order (host copy)

    // per-platelet step ratios (AI-MTS): platelet p takes k_p substeps per
    // interface step on a fine grid of K = lcm(k_p) substeps
    int32_t *plt_k = nullptr;    // device [P]
    std::vector<int32_t> h_plt_k;
    int plt_K = 1;
    // AI-MTS evaluation point of the next platelet-level launch_forces (due_on
    // false: plain forces)
    int due_q = 0;
    bool due_on = false;
    double due_dtm = 0.0;

    // scan scratch
    int32_t *scan_sums;
    int64_t scan_cap;

    // reductions
    double *red_part;            // partial sums [RED_BLOCKS][RED_WORDS]
    double *red_out;             // [RED_WORDS]
    double *prof_part;           // flow-profile partials [PROF_BLOCKS][2 * PROF_BINS_MAX], then the result
    double *vir_acc;             // 9 doubles (conservative virial)
    int red_blocks;

    // control
    int32_t *ctl;
    md_dstate *ds;
    int32_t *h_ctl;              // pinned host mirror
    md_dstate *h_ds;

    md_geom geom;
    float cut2[4];               // list cut-offs squared (FP32)
    double skin_p;               // skin of the platelet particles (cfg.skin_plt, else cfg.skin)
    float excl2;
    float disp2;                 // rebuild threshold on displacement^2

    bool lists_stale = true;
    bool forces_stale = true;
    bool have_particles = false;
    bool have_bonds = false;
    bool have_levels = false;
    int64_t host_step = 0;
    int32_t host_sub = 0;
    unsigned forces_levels = 0;  // levels whose buffers hold current forces
    int cfg_k_m = 1;             // interface substeps of the active schedule
    float margin = 0.0f;         // extra slack in the rebuild trigger (MTS)

    // kernel accounting (md_profile_*)
    int64_t nlaunch = 0;                      // every kernel launched
    int64_t cls_launch[MD_PROF_CLASSES] = {};
    double cls_ms[MD_PROF_CLASSES] = {};
    bool prof_on = false;
    struct prof_rec { int cls; cudaEvent_t a, b; };
    std::vector<prof_rec> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    int prof_cls = -1;
    cudaEvent_t prof_a = nullptr;
    int64_t prof_mark = 0;

    // captured outer step: WHILE(steps_left) { step with IF(rebuild) nodes }
    cudaGraphExec_t step_exec = nullptr;
    cudaGraph_t step_graph = nullptr;
    int graph_key[4] = {-1, -1, -1, -1};
    int64_t graph_body_launches = 0;     // kernels per body iteration
    int64_t graph_chain_launches = 0;    // kernels per taken rebuild
    bool graph_failed = false;
};

// kernel accounting helpers (diag.cu)
void prof_begin(md_system *s, int cls);
void prof_end(md_system *s);
#define MSM_COUNT(s, k) ((s)->nlaunch += (k))

// reductions layout
enum { RED_WORDS = 16, RED_BLOCKS_MAX = 1024, PROF_BINS_MAX = 256, PROF_BLOCKS = 304 };

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tag_of(float4 v) { return __float_as_int(v.w); }
// x32.w holds the particle id in bits 0-29 and its class in bits 30-31
// (0 plasma, 1 wall, 2 platelet), so list builds need no tag load.
#define MSM_ID_MASK 0x3FFFFFFFu
// Plasma-list entries in the warp-stream layout: partner index in the low 27
// bits, the row's lane within its warp of 32 rows above
#define MSM_STREAM_SHIFT 27
#define MSM_STREAM_JMASK 0x07FFFFFF
enum { CLS_FLUID = 0, CLS_WALL = 1, CLS_PLT = 2 };
__device__ __host__ __forceinline__ uint32_t pack_w(uint32_t id, int32_t tag)
{
    const uint32_t cls = tag >= 0 ? CLS_PLT : (tag == MD_TAG_WALL ? CLS_WALL : CLS_FLUID);
    return (id & MSM_ID_MASK) | (cls << 30);
}
__device__ __forceinline__ uint32_t id_of(float4 x) { return (uint32_t)__float_as_int(x.w) & MSM_ID_MASK; }
__device__ __forceinline__ int class_of(float4 x) { return (int)((uint32_t)__float_as_int(x.w) >> 30); }

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the two multiply-xor
// S-boxes with the Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Standard normal from two 32-bit words: Box-Muller on their top 24 bits,
// u1 = (k+1) 2^-24 in (0,1], u2 in [0,1), zeta = sqrt(-2 ln u1) cos(2 pi u2).
// -2 ln u1 comes from the hardware log2 except near u1 = 1 (v = 1 - u1 below
// 2^-6, v exact), where the absolute error of that approximation would
// dominate its small result; there the Taylor series of -ln(1 - v) is summed
// to v^5 (relative truncation below 2^-30).  Both are evaluated and one is
// selected, with no branch: a lane near u1 = 1 would otherwise make its whole
// warp run both paths.  cos(2 pi u2) = -cos(2 pi (u2 - 1/2)) keeps the
// hardware cosine's argument in [-pi, pi).
__device__ __forceinline__ float gauss_from_bits(uint32_t r0, uint32_t r1);

// Uniform variate of zero mean and unit variance from the top 24 bits b of
// one word: sqrt(3) (2 (b + 1/2) 2^-24 - 1), as one FMA on the exact float b.
// The 2^24 values are symmetric about zero, so the mean is exactly zero.
__device__ __forceinline__ float uniform_from_bits(uint32_t r0)
{
    return fmaf((float)(r0 >> 8), 1.7320508075688772f / 8388608.0f,
                1.7320508075688772f * (1.0f / 16777216.0f - 1.0f));
}

__device__ __forceinline__ float gauss_from_bits(uint32_t r0, uint32_t r1)
{
    const uint32_t k = r0 >> 8;
    const float v = (float)(0xFFFFFFu - k) * (1.0f / 16777216.0f);
    const float ser = 2.0f * v * (1.0f + v * (0.5f + v * (0.33333334f + v * (0.25f + v * 0.2f))));
    const float lg = -1.38629436f * __log2f((float)(k + 1u) * (1.0f / 16777216.0f));
    const float t = v < 0.015625f ? ser : lg;
    const float u2 = (float)(r1 >> 8) * (1.0f / 16777216.0f) - 0.5f;
    return -(t * rsqrtf(fmaxf(t, 1e-30f))) * __cosf(6.28318531f * u2);
}

// The first Philox round applied to the counter words that do not depend on
// the pair, (nt, cs) with the key: the round's multiply of the third word and
// the key-mixed fourth word.  philox_pre + the pair words reproduce
// philox4x32_10 bit for bit.
struct philox_pre {
    uint32_t hi1k, lo1, cwk;
    uint2 k1;                      // key after the first round's bump
    int uniform;                   // MD_CFG_UNIFORM_NOISE: zeta from uniform_from_bits
};
__device__ __forceinline__ philox_pre philox_prepare(uint32_t nt, uint32_t cs, uint2 key)
{
    philox_pre q;
    q.hi1k = __umulhi(0xCD9E8D57u, nt) ^ key.x;
    q.lo1 = 0xCD9E8D57u * nt;
    q.cwk = cs ^ key.y;
    q.k1 = make_uint2(key.x + 0x9E3779B9u, key.y + 0xBB67AE85u);
    q.uniform = 0;
    return q;
}
// NOISE: 1 the uniform variate, 0 the Gaussian, -1 as q.uniform says
template <int NOISE = -1>
__device__ __forceinline__ float pair_zeta_pre(uint32_t a, uint32_t b, const philox_pre &q)
{
    const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
    uint4 c = make_uint4(q.hi1k ^ hi, q.lo1, __umulhi(0xD2511F53u, lo) ^ q.cwk, 0xD2511F53u * lo);
    uint2 k = q.k1;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    const bool uni = NOISE < 0 ? q.uniform != 0 : NOISE == 1;
    return uni ? uniform_from_bits(c.x) : gauss_from_bits(c.x, c.y);
}

// Pair noise zeta_ij at time index (nt, cs).
__device__ __forceinline__ float pair_zeta(uint32_t a, uint32_t b, uint32_t nt, uint32_t cs, uint2 key)
{
    const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
    const uint4 r = philox4x32_10(make_uint4(lo, hi, nt, cs), key);
    return gauss_from_bits(r.x, r.y);
}

// FP32 periodic difference with an exact shift of the far coordinate.
__device__ __forceinline__ float img_sub(float a, float b, float L, float hL)
{
    float d = __fsub_rn(a, b);
    if (d > hL) d = __fsub_rn(__fsub_rn(a, L), b);
    else if (d < -hL) d = __fsub_rn(a, __fsub_rn(b, L));
    return d;
}

// Minimum-image separation r_ij = x_i - x_j in FP32, the same operation
// sequence as the list predicate.  *vshift gets the image velocity jump in x
// to subtract from v_i - v_j (Lees-Edwards), 0 otherwise.
__device__ __forceinline__ void min_image_f32(const md_geom &g, float delta, float4 xi, float4 xj,
                                              float &dx, float &dy, float &dz, float &vshift)
{
    float xj0 = xj.x;
    vshift = 0.0f;
    if (g.walls) {
        dy = __fsub_rn(xi.y, xj.y);
    } else if (g.le) {
        dy = __fsub_rn(xi.y, xj.y);
        if (dy > g.hL[1]) {
            dy = __fsub_rn(__fsub_rn(xi.y, g.L[1]), xj.y);
            xj0 = __fadd_rn(xj0, delta);
            if (xj0 >= g.L[0]) xj0 = __fsub_rn(xj0, g.L[0]);
            vshift = g.shear_v;
        } else if (dy < -g.hL[1]) {
            dy = __fsub_rn(xi.y, __fsub_rn(xj.y, g.L[1]));
            xj0 = __fsub_rn(xj0, delta);
            if (xj0 < 0.0f) xj0 = __fadd_rn(xj0, g.L[0]);
            vshift = -g.shear_v;
        }
    } else {
        dy = img_sub(xi.y, xj.y, g.L[1], g.hL[1]);
    }
    dx = img_sub(xi.x, xj0, g.L[0], g.hL[0]);
    dz = img_sub(xi.z, xj.z, g.L[2], g.hL[2]);
}

__device__ __forceinline__ float r2_f32(float dx, float dy, float dz)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}


__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int cell_coord(const md_grid &g, int d, float x)
{
    return clampi(__float2int_rd((x - g.lo[d]) * g.inv_h[d]), 0, g.nc[d] - 1);
}

__device__ __forceinline__ int64_t cell_index(const md_grid &g, int cx, int cy, int cz)
{
    return ((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx;
}

// ---------------------------------------------------------------------------
// Cell scans of the list builders and of the fast-particle pair pass
// ---------------------------------------------------------------------------
// Periodic cell wrap; the integer division only runs for the few cells
// outside the grid.
__device__ __forceinline__ int wrapc(int c, int n)
{
    if (c >= 0 && c < n) return c;
    c %= n;
    return c < 0 ? c + n : c;
}

__device__ __forceinline__ int cell_index32(const md_grid &g, int cx, int cy, int cz)
{
    return (cz * g.nc[1] + cy) * g.nc[0] + cx;
}

// Cells [lo, hi] within reach R of coordinate x along one axis, clamped to
// [-n, 2n - 1] (one period either side: a reach may span several cells) and
// to at most n cells, so that a non-finite or escaped position (reported by
// the integrator's unstable flag) still gives a bounded scan.
__device__ __forceinline__ void cell_span(float x, float lo0, float R, float inv_h, int n, int &lo, int &hi)
{
    lo = __float2int_rd((x - lo0 - R) * inv_h);
    hi = __float2int_rd((x - lo0 + R) * inv_h);
    lo = min(max(lo, -n), 2 * n - 1);
    hi = min(max(hi, -n), 2 * n - 1);
    if (hi - lo + 1 > n) hi = lo + n - 1;
}

// Distance from x to the slab [c0, c0 + h] along one axis, less a slack that
// covers the rounding of the cell assignment (positions sit within a few ulp
// of their cell's nominal bounds).
__device__ __forceinline__ float slab_gap(float x, float c0, float h)
{
    const float gap = fmaxf(fmaxf(c0 - x, x - (c0 + h)), 0.0f);
    return fmaxf(gap - 1e-4f, 0.0f);
}

// Emit (sb, se) for every non-empty run of member positions in the cells
// within reach R of xi.  Cells are at least R/2 wide; each (y, z) row of
// cells is one or two contiguous member runs, rows out of reach are skipped
// and the x extent of a row is trimmed to the sphere of radius R.
// Lees-Edwards rows that cross the y boundary are shifted by the image
// offset.  half: skip cells with a lower index than xi's own cell, and in
// that cell the members up to r.
template <bool HALF, class E, class K>
__device__ __forceinline__ void for_ranges(const md_grid &g, const md_geom &geom, float delta, float4 xi, float R,
                                           int32_t r, E emit, K skip_cell)
{
    const int ox = cell_coord(g, 0, xi.x);
    const int own_row = cell_coord(g, 2, xi.z) * g.nc[1] + cell_coord(g, 1, xi.y);
    const float R2 = R * R;
    const int nx = g.nc[0];
    int zlo, zhi, ylo, yhi;
    cell_span(xi.z, g.lo[2], R, g.inv_h[2], g.nc[2], zlo, zhi);
    cell_span(xi.y, g.lo[1], R, g.inv_h[1], g.nc[1], ylo, yhi);
    if (geom.walls) {
        ylo = max(ylo, 0);
        yhi = min(yhi, g.nc[1] - 1);
    }
    for (int cz = zlo; cz <= zhi; ++cz) {
        const int wz = wrapc(cz, g.nc[2]);
        const float gz = slab_gap(xi.z, g.lo[2] + cz * g.h[2], g.h[2]);
        for (int cy = ylo; cy <= yhi; ++cy) {
            int wy = cy;
            float sx = 0.0f;
            if (!geom.walls) {
                if (cy < 0) {
                    wy = wrapc(cy, g.nc[1]);
                    if (geom.le) sx = delta;
                } else if (cy >= g.nc[1]) {
                    wy = wrapc(cy, g.nc[1]);
                    if (geom.le) sx = -delta;
                }
            }
            const int row = wz * g.nc[1] + wy;
            if (HALF && row < own_row) continue;
            const float gy = slab_gap(xi.y, g.lo[1] + cy * g.h[1], g.h[1]);
            const float rem = R2 - (gy * gy + gz * gz);
            if (rem < 0.0f) continue;
            int xlo, xhi;
            cell_span(xi.x + sx, g.lo[0], sqrtf(rem) + 1e-4f, g.inv_h[0], nx, xlo, xhi);
            // the span as at most two runs of wrapped cell indices
            int a0 = xlo, b0 = xhi, a1 = 0, b1 = -1;
            if (xhi < 0) { a0 += nx; b0 += nx; }
            else if (xlo >= nx) { a0 -= nx; b0 -= nx; }
            else if (xlo < 0) { a0 = xlo + nx; b0 = nx - 1; a1 = 0; b1 = xhi; }
            else if (xhi >= nx) { a0 = xlo; b0 = nx - 1; a1 = 0; b1 = xhi - nx; }
            const int rowc = row * nx;
            // one run of cells [a, b] of this row
            auto run = [&](int a, int b) {
                if (HALF && row == own_row) a = max(a, ox);
                if (a > b) return;
                // cells that cannot hold a partner are cut out of the run
                while (a <= b && skip_cell(rowc + a)) ++a;
                int bb = b;
                while (bb >= a && skip_cell(rowc + bb)) --bb;
                for (int c = a; c <= bb;) {
                    int d = c;
                    while (d < bb && !skip_cell(rowc + d + 1)) ++d;
                    int32_t sb = g.start[rowc + c];
                    const int32_t se = g.start[rowc + d + 1];
                    if (HALF && row == own_row && sb <= r) sb = r + 1;
                    if (sb < se) emit(sb, se);
                    c = d + 1;
                    while (c <= bb && skip_cell(rowc + c)) ++c;
                }
            };
            run(a0, b0);
            if (a1 <= b1) run(a1, b1);
        }
    }
}

// Visit (member position s, particle index) of every candidate of xi.
template <bool HALF, class F, class K>
__device__ __forceinline__ void for_candidates(const md_grid &g, const md_geom &geom, float delta, float4 xi,
                                               float R, const int32_t *__restrict__ members, int32_t r, F fn, K skip)
{
    for_ranges<HALF>(g, geom, delta, xi, R, r, [&](int32_t sb, int32_t se) {
        for (int32_t s = sb; s < se; ++s) fn(s, members ? members[s] : s);
    }, skip);
}

__device__ __forceinline__ bool gate_closed(const int32_t *gate) { return gate && *gate == 0; }

// AI-MTS (Sec. 3.3): every platelet-level term (a bond, an LJ or a Morse pair)
// lives on the grid of the finer of its platelets, c = max(k_i, k_j), of the
// K = lcm(k) substeps per interface step.  At evaluation point qe (1..K) the
// term is due when qe is a multiple of K/c, and it is stored as the impulse
// (dt_m / c) F it applies; terms not due contribute nothing.
struct md_due {
    const int32_t *plt_k;   // null: plain forces (STS, fixed-k RESPA)
    int qe, K;
    float dtm;
    // the drift stride K / lcm(k_p, k of p's listed contact partners), per
    // platelet and per platelet row (plt_sorted order); null: not in use
    const int32_t *stride, *row_stride;
};

// AI-MTS: whether any platelet of a block of terms is due at this point
// (r: the first and last platelet of the block's terms, which are stored
// grouped by platelet); a block with none skips its loads.
__device__ __forceinline__ bool block_due(const md_due &d, int2 r)
{
    for (int p = r.x; p <= r.y; ++p)
        if ((d.qe % (d.K / d.plt_k[p])) == 0) return true;
    return false;
}

__device__ __forceinline__ float term_scale(const md_due &d, int32_t ti, int32_t tj)
{
    if (!d.plt_k) return 1.0f;
    const int c = max(d.plt_k[ti & ~MD_RECEPTOR_BIT], d.plt_k[tj & ~MD_RECEPTOR_BIT]);
    return (d.qe % (d.K / c)) == 0 ? d.dtm / (float)c : 0.0f;
}

// ---------------------------------------------------------------------------
// host-side launchers (one translation unit each)
// ---------------------------------------------------------------------------
// sort.cu
// carry: force levels whose values survive the re-sort (the others are zero
// at that point and stay so)
cudaError_t launch_rebuild(md_system *s, const int32_t *gate, unsigned carry = MD_LEVEL_ALL);
cudaError_t launch_scan(md_system *s, const int32_t *in, int32_t *out, int64_t count, int32_t *total_out,
                        const int32_t *gate);
// neighbor.cu
cudaError_t launch_build_lists(md_system *s, const int32_t *gate);
// AI-MTS drift strides from the current LJ / receptor lists and step ratios
// (run after every build and every change of the ratios)
cudaError_t launch_strides(md_system *s, const int32_t *gate);
// forces.cu
// with_fast: also the fast-particle pass of the DPD levels (launch_fast_pairs);
// fdet: deterministic mode, every pair term added to these 64-bit fixed-point
// sums (3 per particle, units of 2^-32) instead of out
cudaError_t launch_forces(md_system *s, unsigned level_mask, float4 *const out[3], bool virial,
                          bool with_fast = true, unsigned long long *fdet = nullptr);
// pairs of the listed fast plasma particles that the plasma / interface lists lack
cudaError_t launch_fast_pairs(md_system *s, unsigned level_mask, float4 *const out[3], bool virial,
                              unsigned long long *fdet = nullptr);
// a level's fixed-point sums to its FP32 buffer
cudaError_t launch_fixed_to_f4(md_system *s, const unsigned long long *q, float4 *f);
// integrate.cu
// stride_q >= 0: AI-MTS substep stride_q of the K grid, platelet particles
// kicked and drifted by their platelet's stride (launch_strides)
cudaError_t launch_kick_drift(md_system *s, const float h[3], int kick_which, double dt, int drift_which,
                              unsigned zero_levels, bool plt_rows, int stride_q = -1);
cudaError_t launch_set_time(md_system *s, int64_t n, int32_t c, double t);
cudaError_t launch_outer_begin(md_system *s, cudaGraphConditionalHandle loop, bool use_loop);
cudaError_t launch_time_rel(md_system *s, int dn, int c, double t_off);
cudaError_t launch_cond_rebuild(md_system *s, cudaGraphConditionalHandle h);
cudaError_t launch_set_loop(md_system *s, int64_t n);
cudaError_t launch_zero_forces(md_system *s, unsigned levels);
// md_set_xv keeping the lists: scatter an id-order state (device AoS, 3n
// doubles) into the storage slots, then the rebuild check of every particle
cudaError_t launch_place_state(md_system *s, const double *aos_dev, bool velocities);
cudaError_t launch_check_placed(md_system *s, int64_t step0);
// reduce.cu
cudaError_t launch_kinetics(md_system *s);
// y-binned v_x sums and counts into prof_part + PROF_BLOCKS * 2 * PROF_BINS_MAX:
// plasma, edge slabs clamped (mobile false); mobile particles inside [0, Ly)
// (mobile true, the local flow of the wall temperature)
cudaError_t launch_flow_profile(md_system *s, int nbins, bool mobile = false);
// slabs of the local flow subtracted from the wall-bounded kinetic tensor
constexpr int KIN_BINS = 20;
// features.cu
// f_plt: platelet-level forces to use (null: s->f[2]); hk: half kicks per
// level still pending on the stored velocities (null: none)
cudaError_t launch_features(md_system *s, double *out_dev, const float4 *f_plt = nullptr,
                            const float *hk = nullptr);
// append feat to the ring at the device record counter, then advance it
cudaError_t launch_feature_ring(md_system *s, const double *feat);
// ai.cu: the denoising filter (raw [B][T][F] -> normalised time-major
// [T][B][F]) and an Adam step (b1 0.9, b2 0.999, eps 1e-8, step count t)
cudaError_t ai_launch_denoise(const float *raw, int B, int T, int F, const float *mean, const float *stdv, float *out,
                              cudaStream_t st);
cudaError_t ai_launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, int64_t t,
                           cudaStream_t st);
// api.cu helpers
int set_error(md_system *s, int code, const char *msg);
int cuda_fail(md_system *s, cudaError_t e, const char *where);

// kick-drift subsets
enum { DRIFT_ALL = 0, DRIFT_FLUID = 1, DRIFT_PLT = 2 };
