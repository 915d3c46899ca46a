// K3-K5: pair and bond forces of the three levels.
//
//  K3  DPD (Eq. 1 plasma-plasma / plasma-wall on MD_LIST_FLUID; Eq. 3
//      interface on MD_LIST_IFACE):
//        F_ij = [a w - gamma w^2 (e.v_ij) + sigma w zeta_ij / sqrt(dt)] e_ij,
//        w = 1 - r/rc, zeta_ij ~ N(0,1) from Philox4x32-10 keyed on
//        (min id, max id, n, c) so that F^R_ji = -F^R_ij exactly.
//  K4  harmonic bonds (Eq. 2): F_i = -2 k_b (r - r0) e_ij.
//  K5  LJ 12-6 (Eq. 2) on MD_LIST_LJ and the printed-form Morse plus the
//      receptor term f_A (1 - r/r0) (Eq. 2, Eq. 4) on MD_LIST_MORSE.
//
// Partner j's contribution is scattered with one vector atomic
// (red.global.add.v4.f32); a row's own sum is added once at the end.  The
// conservative virial (pressure, Sec. 4.2) is accumulated in FP32 per thread
// and reduced in FP64 when requested.
#include "msm_internal.cuh"

namespace {

struct pair_args {
    int64_t rows;
    const int32_t *row_idx;
    const int32_t *nl, *nc;
    int cap;
    const float4 *x32, *v;
    float4 *f;
    md_geom geom;
    const md_dstate *ds;
    uint2 key;
    // DPD
    float a_same, a_wall, gamma, sig_isdt, rc2, inv_rc;
    // LJ / Morse
    float lj_eps24, lj_sig2, lj_rc2;
    float m_Da_r0, m_alpha, m_inv_r0, m_rc2, f_A;
    double *vir;
    // AI-MTS: platelet-level pairs scaled to impulses, or skipped, per term_scale
    md_due due;
    const int32_t *tag;
    // deterministic mode: every pair term added in 64-bit fixed point here
    unsigned long long *fdet;
    // interface level, Eq. 3 with an LJ conservative term (MD_CFG_IFACE_LJ):
    // 24 eps / s^2 and s^2 of the LJ, cut at its minimum (wca_rc2 0: off)
    float wca_eps24, wca_sig2, wca_rc2;
    // MD_CFG_UNIFORM_NOISE: zeta_ij a unit-variance uniform variate
    int uniform_noise;
};

// Conservative part of a DPD-level pair: a (1 - r/rc), or on the interface
// level the repulsive LJ when selected (force magnitude along e_ij)
template <bool IF>
__device__ __forceinline__ float dpd_conservative(const pair_args &a, float aij, float wr, float r2, float inv_r)
{
    if (IF && a.wca_rc2 > 0.0f) {
        if (!(r2 < a.wca_rc2)) return 0.0f;
        const float s2 = a.wca_sig2 / r2;
        const float s6 = s2 * s2 * s2;
        return a.wca_eps24 * (2.0f * s6 * s6 - s6) * inv_r;
    }
    return aij * wr;
}

struct vir6 {
    float xx, yy, zz, xy, xz, yz;
    __device__ void add(float dx, float dy, float dz, float s)  // r (x) (s r)
    {
        xx += dx * dx * s; yy += dy * dy * s; zz += dz * dz * s;
        xy += dx * dy * s; xz += dx * dz * s; yz += dy * dz * s;
    }
    __device__ void add_rf(float rx, float ry, float rz, float fx, float fy, float fz)  // sym(r (x) F)
    {
        xx += rx * fx; yy += ry * fy; zz += rz * fz;
        xy += 0.5f * (rx * fy + ry * fx); xz += 0.5f * (rx * fz + rz * fx); yz += 0.5f * (ry * fz + rz * fy);
    }
};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void flush_virial(double *vir, const vir6 &w)
{
    const double c[6] = {w.xx, w.yy, w.zz, w.xy, w.xz, w.yz};
    double s[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = warp_sum_d(c[k]);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&vir[0], s[0]); atomicAdd(&vir[4], s[1]); atomicAdd(&vir[8], s[2]);
        atomicAdd(&vir[1], s[3]); atomicAdd(&vir[3], s[3]);
        atomicAdd(&vir[2], s[4]); atomicAdd(&vir[6], s[4]);
        atomicAdd(&vir[5], s[5]); atomicAdd(&vir[7], s[5]);
    }
}

__device__ __forceinline__ void scatter(float4 *f, int32_t j, float fx, float fy, float fz)
{
    atomicAdd(&f[j], make_float4(fx, fy, fz, 0.0f));
}

// Deterministic mode: a pair term in units of 2^-32 (exact scaling, rounding
// to the nearest integer, symmetric under negation), added as a 64-bit
// integer: the sums are independent of the order of the atomic updates, and
// +q and -q of a pair cancel exactly.
__device__ __forceinline__ void put_fixed(unsigned long long *f, int32_t j, float fx, float fy, float fz)
{
    const float s = 4294967296.0f;
    atomicAdd(&f[3 * (int64_t)j], (unsigned long long)__float2ll_rn(fx * s));
    atomicAdd(&f[3 * (int64_t)j + 1], (unsigned long long)__float2ll_rn(fy * s));
    atomicAdd(&f[3 * (int64_t)j + 2], (unsigned long long)__float2ll_rn(fz * s));
}

// A pair term on i (+) and j (-), evaluated with the particle of lower id
// first so that its FP32 value does not depend on which of the two owns the
// list row (the minimum image rounds differently in the two orientations).
__device__ __forceinline__ void put_pair(const pair_args &a, int32_t i, int32_t j, float px, float py, float pz)
{
    put_fixed(a.fdet, i, px, py, pz);
    put_fixed(a.fdet, j, -px, -py, -pz);
}

// ---------------------------------------------------------------------------
// K3: DPD pair forces over one list (fluid level or interface level).
//
// A warp owns 32 consecutive rows and streams their concatenated candidate
// lists 32 entries at a time, so every lane has work whatever the row
// lengths (the row of flat entry f is found by a shuffle binary search over
// the rows' prefix offsets).  Candidates inside rc are appended to a per-warp
// ring queue in shared memory (ballot + popc give the slots); whenever 32 pairs
// are queued each lane evaluates one -- Philox, Box-Muller and Eq. 1 -- and
// scatters -F_ij to j.  Queue entries keep their row order, so the row sums
// are a segmented shuffle reduction over each batch.
// ---------------------------------------------------------------------------
constexpr int DPD_WARPS = MSM_TPB / 32;
constexpr int DPD_QCAP = 64;

struct dpd_smem {
    float4 xi[DPD_WARPS][32];          // row positions (w: id)
    float4 vi[DPD_WARPS][32];          // row velocities (w: tag)
    float4 fi[DPD_WARPS][32];          // row force sums
    float4 qa[DPD_WARPS][DPD_QCAP];    // queued pairs (a ring): dx, dy, dz, image v-shift
    int2 qb[DPD_WARPS][DPD_QCAP];      // j | source row (lane) << 27, id_j (id_i: the row's xi.w)
};

// Eq. 1 for one pair, the particle with the lower id first (deterministic
// mode): the pair's FP32 terms then do not depend on which particle owns the
// list row; the cut-off is decided here too.
template <bool VIR, bool IF>
__device__ __forceinline__ void dpd_pair_fixed(const pair_args &a, int32_t i, int32_t j, const philox_pre &pq,
                                               vir6 &w)
{
    const float4 xi = a.x32[i], xj = a.x32[j];
    const bool sw = id_of(xi) > id_of(xj);
    const int32_t p = sw ? j : i, q = sw ? i : j;
    const float4 xp = sw ? xj : xi, xq = sw ? xi : xj;
    const float4 vp = a.v[p], vq = a.v[q];
    float dx, dy, dz, vsh;
    min_image_f32(a.geom, a.ds->le_offset_f, xp, xq, dx, dy, dz, vsh);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < a.rc2) || r2 == 0.0f) return;
    const bool wall = tag_of(vp) == MD_TAG_WALL || tag_of(vq) == MD_TAG_WALL;
    const float aij = wall ? a.a_wall : a.a_same;
    const float inv_r = rsqrtf(r2);
    const float wr = 1.0f - r2 * inv_r * a.inv_rc;
    const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
    const float edv = ex * (vp.x - vq.x - vsh) + ey * (vp.y - vq.y) + ez * (vp.z - vq.z);
    const float zeta = pair_zeta_pre(id_of(xp), id_of(xq), pq);
    const float fc = dpd_conservative<IF>(a, aij, wr, r2, inv_r);
    const float fp = fc - a.gamma * wr * wr * edv + a.sig_isdt * wr * zeta;
    put_pair(a, p, q, fp * ex, fp * ey, fp * ez);
    if (VIR) w.add(dx, dy, dz, fc * inv_r);
}

template <bool VIR, bool DET, bool IF, bool UNI>
__device__ __forceinline__ void dpd_batch(const pair_args &a, dpd_smem &sm, int warp, int lane, bool valid,
                                          int slot, const philox_pre &pq, vir6 &w, int64_t r0)
{
    if (DET) {
        if (valid) {
            const int2 b = sm.qb[warp][slot];
            const int rr = (int)((uint32_t)b.x >> MSM_STREAM_SHIFT);
            const int32_t i = a.row_idx ? a.row_idx[r0 + rr] : (int32_t)(r0 + rr);
            dpd_pair_fixed<VIR, IF>(a, i, b.x & MSM_STREAM_JMASK, pq, w);
        }
        return;
    }
    float px = 0.f, py = 0.f, pz = 0.f;
    int src = -1;
    if (valid) {
        const float4 q = sm.qa[warp][slot];
        const int2 b = sm.qb[warp][slot];
        const int32_t jq = b.x & MSM_STREAM_JMASK;
        src = (int)((uint32_t)b.x >> MSM_STREAM_SHIFT);
        const uint32_t id_iq = (uint32_t)__float_as_int(sm.xi[warp][src].w) & MSM_ID_MASK;
        const float4 vi = sm.vi[warp][src];
        const float4 vj = a.v[jq];
        const float r2 = q.x * q.x + q.y * q.y + q.z * q.z;
        const bool wall = tag_of(vi) == MD_TAG_WALL || tag_of(vj) == MD_TAG_WALL;
        const float aij = wall ? a.a_wall : a.a_same;
        const float inv_r = rsqrtf(r2);
        const float wr = 1.0f - r2 * inv_r * a.inv_rc;
        const float ex = q.x * inv_r, ey = q.y * inv_r, ez = q.z * inv_r;
        const float edv = ex * (vi.x - vj.x - q.w) + ey * (vi.y - vj.y) + ez * (vi.z - vj.z);
        const float zeta = pair_zeta_pre<UNI ? 1 : 0>(id_iq, (uint32_t)b.y, pq);
        const float fc = dpd_conservative<IF>(a, aij, wr, r2, inv_r);
        const float fp = fc - a.gamma * wr * wr * edv + a.sig_isdt * wr * zeta;
        px = fp * ex; py = fp * ey; pz = fp * ez;
        scatter(a.f, jq, -px, -py, -pz);
        if (VIR) w.add(q.x, q.y, q.z, fc * inv_r);
    }
    // segmented sum over runs of equal src (entries are in row order): lane
    // l adds lane l + o's partial while no run starts in (l, l + o]
    const int prev = __shfl_up_sync(0xffffffffu, src, 1);
    const bool head = lane == 0 || prev != src;
    const unsigned hm = __ballot_sync(0xffffffffu, head);
    const unsigned above = lane == 31 ? 0xffffffffu : (hm >> (lane + 1));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float ox = __shfl_down_sync(0xffffffffu, px, o);
        const float oy = __shfl_down_sync(0xffffffffu, py, o);
        const float oz = __shfl_down_sync(0xffffffffu, pz, o);
        if (lane + o < 32 && (above & ((1u << o) - 1u)) == 0u) { px += ox; py += oy; pz += oz; }
    }
    if (valid && head) {     // head of a run holds its total
        float4 t = sm.fi[warp][src];
        t.x += px; t.y += py; t.z += pz;
        sm.fi[warp][src] = t;
    }
}

// STREAM: the list is in the warp-stream layout (the plasma list): entry f
// of the warp's concatenated rows is word f of the first row's slot, with the
// row's lane in its top bits; otherwise ELL rows (the interface list) and the
// row of an entry comes from a binary search over the rows' prefix offsets.
// UNI: the noise variate (MD_CFG_UNIFORM_NOISE) fixed at compile time; the
// kernel picks the instance once.
template <bool VIR, bool STREAM, bool DET, bool UNI>
__device__ __forceinline__ void dpd_rows(const pair_args &a, dpd_smem &sm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = r - lane;
    const bool active = r < a.rows;
    const int32_t i = active ? (a.row_idx ? a.row_idx[r] : (int32_t)r) : 0;
    const int cnt = active ? min(a.nc[r], a.cap) : 0;
    const float4 xi = active ? a.x32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    sm.xi[warp][lane] = xi;
    sm.vi[warp][lane] = active ? a.v[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    sm.fi[warp][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    philox_pre pq = philox_prepare((uint32_t)a.ds->step, (uint32_t)a.ds->sub, a.key);
    pq.uniform = a.uniform_noise;
    const float delta = a.ds->le_offset_f;
    const unsigned lt = (1u << lane) - 1u;
    vir6 w = {0, 0, 0, 0, 0, 0};
    // exclusive prefix of the row lengths: row L owns flat entries [pre_L, pre_L + cnt_L)
    int pre = cnt, total;
    if (STREAM) {
        total = __reduce_add_sync(0xffffffffu, cnt);
    } else {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += t;
        }
        total = __shfl_sync(0xffffffffu, pre, 31);
        pre -= cnt;
    }
    const int32_t *wst = a.nl + r0 * a.cap;
    int qn = 0, qh = 0;     // queued pairs, ring slot of the oldest
    // row of flat entry f (the last lane whose prefix is <= f) and its list entry
    auto locate = [&](int f, int &row, int32_t &j) {
        if (STREAM) {
            const uint32_t e = f < total ? (uint32_t)wst[f] : 0u;
            row = (int)(e >> MSM_STREAM_SHIFT);
            j = (int32_t)(e & MSM_STREAM_JMASK);
            return;
        }
        row = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int p = __shfl_sync(0xffffffffu, pre, row + step);
            if (p <= f) row += step;
        }
        const int k = f - __shfl_sync(0xffffffffu, pre, row);
        j = f < total ? a.nl[(r0 + row) * a.cap + k] : 0;
    };
    // software pipeline over rounds of 32 entries: the list entries of round
    // t + 2 and the positions of round t + 1 are in flight while round t is
    // tested and its queued pairs evaluated
    int row_c, row_n, row_nn;
    int32_t j_c, j_n, j_nn;
    locate(lane, row_c, j_c);
    float4 xj_c = lane < total ? a.x32[j_c] : make_float4(0.f, 0.f, 0.f, 0.f);
    locate(32 + lane, row_n, j_n);
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
        const bool valid = base + lane < total;
        const float4 xj_n = base + 32 + lane < total ? a.x32[j_n] : make_float4(0.f, 0.f, 0.f, 0.f);
        locate(base + 64 + lane, row_nn, j_nn);
        bool hit = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, vsh = 0.f;
        uint32_t id_i = 0;
        if (valid) {
            const float4 xi = sm.xi[warp][row_c];
            id_i = id_of(xi);
            min_image_f32(a.geom, delta, xi, xj_c, dx, dy, dz, vsh);
            const float r2 = dx * dx + dy * dy + dz * dz;
            // deterministic mode: a slightly wider net, the cut-off decided
            // again in the pair's canonical orientation
            hit = r2 < (DET ? a.rc2 * 1.000002f : a.rc2) && r2 > 0.0f;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int pos = (qh + qn + __popc(m & lt)) & (DPD_QCAP - 1);
            sm.qa[warp][pos] = make_float4(dx, dy, dz, vsh);
            sm.qb[warp][pos] = make_int2(j_c | (row_c << MSM_STREAM_SHIFT), (int)id_of(xj_c));
        }
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
            dpd_batch<VIR, DET, !STREAM, UNI>(a, sm, warp, lane, true, (qh + lane) & (DPD_QCAP - 1), pq, w, r0);
            qh = (qh + 32) & (DPD_QCAP - 1);
            qn -= 32;
            __syncwarp();
        }
        row_c = row_n; j_c = j_n; xj_c = xj_n;
        row_n = row_nn; j_n = j_nn;
    }
    if (qn > 0) dpd_batch<VIR, DET, !STREAM, UNI>(a, sm, warp, lane, lane < qn, (qh + lane) & (DPD_QCAP - 1), pq, w, r0);
    __syncwarp();
    if (!DET && active && cnt > 0) {
        const float4 t = sm.fi[warp][lane];
        scatter(a.f, i, t.x, t.y, t.z);
    }
    if (VIR) flush_virial(a.vir, w);
}

template <bool VIR, bool STREAM, bool DET = false>
__global__ void __launch_bounds__(MSM_TPB, 5) k_dpd(pair_args a)
{
    __shared__ dpd_smem sm;
    if (a.uniform_noise) dpd_rows<VIR, STREAM, DET, true>(a, sm);
    else dpd_rows<VIR, STREAM, DET, false>(a, sm);
}

// K3 for the fast plasma particles: those that moved beyond skin/2 (but
// within the skin) since the list build, listed by the kick-drift instead of
// triggering a rebuild.  A pair of two particles within skin/2 of their build
// positions that came within rc was within rc + skin at the build, so it is
// in the list; a pair with a fast particle may not be.  For every fast
// particle i this pass scans the cells within rc + skin (its partners, at most
// a skin from their build cells), keeps the partners now within rc, and
// evaluates those that the list lacks -- decided by the builder's predicate
// on the build positions, row particle first (plasma list: the lower storage
// index; interface list: the platelet particle), so no pair is counted twice.
// Two fast particles meet once, from the lower index.  Eq. 1 as in k_dpd.
struct fast_args {
    const int32_t *fast_idx;
    const uint32_t *fast_flag;
    const int32_t *ctl;
    int64_t fast_max;
    md_grid g;                 // cells of the candidates: main grid, or the platelet sub-grid
    const int32_t *members;    // null: main grid (storage order); else platelet rows
    const float4 *xb;          // positions at the build
    float R;                   // scan reach
    float cut2;                // the list's cut-off squared (the builder's predicate)
};

// One warp per fast particle: lane t takes (y, z) stencil row t of the cells
// within reach (at most 25 rows for cells at least half the reach wide) and
// its one or two runs of members, then the warp tests the concatenated
// candidates 32 at a time; a few dependent loads per particle instead of one
// per candidate.
template <bool VIR, bool IFACE, bool DET = false>
__global__ void __launch_bounds__(128) k_dpd_fast(pair_args a, fast_args fa)
{
    const int64_t nf = min((int64_t)fa.ctl[CTL_NFAST], fa.fast_max);
    const float delta = a.ds->le_offset_f, dbuild = a.ds->le_build_f;
    const uint32_t stamp = a.ds->fast_stamp;
    philox_pre pq = philox_prepare((uint32_t)a.ds->step, (uint32_t)a.ds->sub, a.key);
    pq.uniform = a.uniform_noise;
    const int lane = threadIdx.x & 31;
    const md_grid &g = fa.g;
    vir6 w = {0, 0, 0, 0, 0, 0};
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = warp0; q < nf; q += nwarps) {
        const int32_t i = fa.fast_idx[q];
        const float4 xi = a.x32[i], vi = a.v[i], xbi = fa.xb[i];
        const uint32_t idi = id_of(xi);
        int zlo, zhi, ylo, yhi;
        cell_span(xi.z, g.lo[2], fa.R, g.inv_h[2], g.nc[2], zlo, zhi);
        cell_span(xi.y, g.lo[1], fa.R, g.inv_h[1], g.nc[1], ylo, yhi);
        if (a.geom.walls) {
            ylo = max(ylo, 0);
            yhi = min(yhi, g.nc[1] - 1);
        }
        const int ny = max(yhi - ylo + 1, 0), nrows = ny * max(zhi - zlo + 1, 0);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int r0 = 0; r0 < nrows; r0 += 32) {
            // this lane's stencil row: up to two runs [sb0, se0), [sb1, se1)
            int32_t sb0 = 0, se0 = 0, sb1 = 0, se1 = 0;
            const int t = r0 + lane;
            if (t < nrows) {
                const int cz = zlo + t / ny, cy = ylo + t % ny;
                const int wz = wrapc(cz, g.nc[2]);
                int wy = cy;
                float sx = 0.0f;
                if (!a.geom.walls) {
                    if (cy < 0) {
                        wy = wrapc(cy, g.nc[1]);
                        if (a.geom.le) sx = delta;
                    } else if (cy >= g.nc[1]) {
                        wy = wrapc(cy, g.nc[1]);
                        if (a.geom.le) sx = -delta;
                    }
                }
                const float gz = slab_gap(xi.z, g.lo[2] + cz * g.h[2], g.h[2]);
                const float gy = slab_gap(xi.y, g.lo[1] + cy * g.h[1], g.h[1]);
                const float rem = fa.R * fa.R - (gy * gy + gz * gz);
                if (rem >= 0.0f) {
                    const int nx = g.nc[0];
                    int xlo, xhi;
                    cell_span(xi.x + sx, g.lo[0], sqrtf(rem) + 1e-4f, g.inv_h[0], nx, xlo, xhi);
                    int a0 = xlo, b0 = xhi, a1 = 0, b1 = -1;
                    if (xhi < 0) { a0 += nx; b0 += nx; }
                    else if (xlo >= nx) { a0 -= nx; b0 -= nx; }
                    else if (xlo < 0) { a0 = xlo + nx; b0 = nx - 1; b1 = xhi; }
                    else if (xhi >= nx) { b0 = nx - 1; b1 = xhi - nx; }
                    const int rowc = (wz * g.nc[1] + wy) * nx;
                    sb0 = g.start[rowc + a0];
                    se0 = g.start[rowc + b0 + 1];
                    if (a1 <= b1) {
                        sb1 = g.start[rowc + a1];
                        se1 = g.start[rowc + b1 + 1];
                    }
                }
            }
            const int len0 = se0 - sb0, len = len0 + (se1 - sb1);
            int pre = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += u;
            }
            const int total = __shfl_sync(0xffffffffu, pre, 31);
            pre -= len;
            for (int base = 0; base < total; base += 32) {
                const int f = base + lane;
                int owner = 0;     // the last lane whose prefix is <= f
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int pv = __shfl_sync(0xffffffffu, pre, owner + st);
                    if (pv <= f) owner += st;
                }
                const int k = f - __shfl_sync(0xffffffffu, pre, owner);
                const int l0 = __shfl_sync(0xffffffffu, len0, owner);
                const int32_t b_0 = __shfl_sync(0xffffffffu, sb0, owner), b_1 = __shfl_sync(0xffffffffu, sb1, owner);
                if (f >= total) continue;
                const int32_t sm = k < l0 ? b_0 + k : b_1 + (k - l0);
                const int32_t j = fa.members ? fa.members[sm] : sm;
                if (j == i) continue;
                const float4 xj = a.x32[j];
                if (IFACE) {
                    if (class_of(xj) != CLS_PLT) continue;
                } else {
                    if (class_of(xj) == CLS_PLT) continue;
                    if (fa.fast_flag[j] == stamp && j < i) continue;
                }
                float dx, dy, dz, vsh;
                min_image_f32(a.geom, delta, xi, xj, dx, dy, dz, vsh);
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < (DET ? a.rc2 * 1.000002f : a.rc2)) || r2 == 0.0f) continue;
                float ex, ey, ez, es;
                const float4 xbj = fa.xb[j];
                if (IFACE || j < i) min_image_f32(a.geom, dbuild, xbj, xbi, ex, ey, ez, es);
                else min_image_f32(a.geom, dbuild, xbi, xbj, ex, ey, ez, es);
                if (r2_f32(ex, ey, ez) < fa.cut2) continue;       // in the list
                if (DET) {
                    dpd_pair_fixed<VIR, IFACE>(a, i, j, pq, w);
                    continue;
                }
                const float4 vj = a.v[j];
                const bool wall = tag_of(vj) == MD_TAG_WALL;
                const float aij = wall ? a.a_wall : a.a_same;
                const float inv_r = rsqrtf(r2);
                const float wr = 1.0f - r2 * inv_r * a.inv_rc;
                const float nx = dx * inv_r, ny_ = dy * inv_r, nz = dz * inv_r;
                const float edv = nx * (vi.x - vj.x - vsh) + ny_ * (vi.y - vj.y) + nz * (vi.z - vj.z);
                const float zeta = pair_zeta_pre(idi, id_of(xj), pq);
                const float fc = dpd_conservative<IFACE>(a, aij, wr, r2, inv_r);
                const float fp = fc - a.gamma * wr * wr * edv + a.sig_isdt * wr * zeta;
                const float px = fp * nx, py = fp * ny_, pz = fp * nz;
                fx += px; fy += py; fz += pz;
                scatter(a.f, j, -px, -py, -pz);
                if (VIR) w.add(dx, dy, dz, fc * inv_r);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (lane == 0 && (fx != 0.f || fy != 0.f || fz != 0.f)) scatter(a.f, i, fx, fy, fz);
    }
    if (VIR) flush_virial(a.vir, w);
}

// K5a: LJ 12-6 (Eq. 2), shifted potential: the force is unshifted.
template <bool VIR>
__global__ void __launch_bounds__(MSM_TPB) k_lj(pair_args a)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    vir6 w = {0, 0, 0, 0, 0, 0};
    if (r < a.rows) {
        // AI-MTS: off its platelet's stride points no term of the row is due
        // (the stride divides K / max(k_i, k_j) for every partner j listed),
        // so the row's list is not read
        const bool idle = a.due.row_stride && (a.due.qe % a.due.row_stride[r]) != 0;
        const int32_t i = a.row_idx[r];
        const int cnt = idle ? 0 : min(a.nc[r], a.cap);
        if (cnt > 0) {
            const float4 xi = a.x32[i];
            const float delta = a.ds->le_offset_f;
            const int32_t ti = a.due.plt_k ? a.tag[i] : 0;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            for (int k = 0; k < cnt; ++k) {
                const int32_t j = a.nl[r * a.cap + k];
                const float sc = a.due.plt_k ? term_scale(a.due, ti, a.tag[j]) : 1.0f;
                if (sc == 0.0f) continue;
                const float4 xj = a.x32[j];
                // deterministic mode: the particle of lower id first
                const bool sw = a.fdet && id_of(xi) > id_of(xj);
                float dx, dy, dz, vsh;
                min_image_f32(a.geom, delta, sw ? xj : xi, sw ? xi : xj, dx, dy, dz, vsh);
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 >= a.lj_rc2 || r2 == 0.0f) continue;
                const float inv_r2 = 1.0f / r2;
                const float s2 = a.lj_sig2 * inv_r2;
                const float s6 = s2 * s2 * s2;
                const float fr = a.lj_eps24 * (2.0f * s6 * s6 - s6) * inv_r2 * sc;
                const float px = fr * dx, py = fr * dy, pz = fr * dz;
                if (a.fdet) {
                    put_pair(a, sw ? j : i, sw ? i : j, px, py, pz);
                } else {
                    fx += px; fy += py; fz += pz;
                    scatter(a.f, j, -px, -py, -pz);
                }
                if (VIR) w.add(dx, dy, dz, fr);
            }
            if (!a.fdet) scatter(a.f, i, fx, fy, fz);
        }
    }
    if (VIR) flush_virial(a.vir, w);
}

// K5b: Morse in the printed form of Eq. 2 plus the receptor term of Eq. 4.
template <bool VIR>
__global__ void __launch_bounds__(MSM_TPB) k_morse(pair_args a)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    vir6 w = {0, 0, 0, 0, 0, 0};
    if (r < a.rows) {
        const int32_t i = a.row_idx[r];
        const int32_t ti = a.due.plt_k ? a.tag[i] : 0;
        // AI-MTS: as for the LJ rows, by the stride of the row's platelet
        const bool idle = a.due.stride && (a.due.qe % a.due.stride[ti & ~MD_RECEPTOR_BIT]) != 0;
        const int cnt = idle ? 0 : min(a.nc[r], a.cap);
        if (cnt > 0) {
            const float4 xi = a.x32[i];
            const float delta = a.ds->le_offset_f;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            for (int k = 0; k < cnt; ++k) {
                const int32_t j = a.nl[r * a.cap + k];
                const float sc = a.due.plt_k ? term_scale(a.due, ti, a.tag[j]) : 1.0f;
                if (sc == 0.0f) continue;
                const float4 xj = a.x32[j];
                const bool sw = a.fdet && id_of(xi) > id_of(xj);
                float dx, dy, dz, vsh;
                min_image_f32(a.geom, delta, sw ? xj : xi, sw ? xi : xj, dx, dy, dz, vsh);
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 >= a.m_rc2 || r2 == 0.0f) continue;
                const float inv_r = rsqrtf(r2);
                const float rr = r2 * inv_r;
                const float t = a.m_alpha * (1.0f - rr * a.m_inv_r0);
                const float fm = a.m_Da_r0 * (expf(t) - expf(0.5f * t)) + a.f_A * (1.0f - rr * a.m_inv_r0);
                const float s = fm * inv_r * sc;
                const float px = s * dx, py = s * dy, pz = s * dz;
                if (a.fdet) {
                    put_pair(a, sw ? j : i, sw ? i : j, px, py, pz);
                } else {
                    fx += px; fy += py; fz += pz;
                    scatter(a.f, j, -px, -py, -pz);
                }
                if (VIR) w.add(dx, dy, dz, s);
            }
            if (!a.fdet) scatter(a.f, i, fx, fy, fz);
        }
    }
    if (VIR) flush_virial(a.vir, w);
}

// K4: harmonic bonds, one thread per bond.
template <bool VIR>
__global__ void __launch_bounds__(MSM_TPB) k_bonds(int64_t nb, const int32_t *__restrict__ ij,
                                                  const float *__restrict__ r0, float kb2, const float4 *__restrict__ x32,
                                                  float4 *f, md_geom geom, const md_dstate *ds, double *vir, md_due due,
                                                  const int32_t *tag, unsigned long long *fdet,
                                                  const int2 *__restrict__ blk)
{
    vir6 w = {0, 0, 0, 0, 0, 0};
    // the CTAs stride over the blocks of MSM_TPB bonds: an AI-MTS substep
    // that skips most blocks costs a pass over their table, not a launch of
    // them all
    const int64_t nblk = (nb + MSM_TPB - 1) / MSM_TPB;
    for (int64_t vb = blockIdx.x; vb < nblk; vb += gridDim.x) {
        // AI-MTS substep: a block whose platelets are all off this grid point
        // skips its loads (the decision is uniform over the CTA)
        if (due.plt_k && !block_due(due, blk[vb])) continue;
        const int64_t b = vb * MSM_TPB + threadIdx.x;
        // both ends belong to one platelet: the bond lives on that platelet's grid
        const float sc = (b < nb && due.plt_k) ? term_scale(due, tag[ij[2 * b]], tag[ij[2 * b]]) : 1.0f;
        if (b < nb && sc != 0.0f) {
            const int32_t i = ij[2 * b], j = ij[2 * b + 1];
            float dx, dy, dz, vsh;
            min_image_f32(geom, ds->le_offset_f, x32[i], x32[j], dx, dy, dz, vsh);
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0.0f) {
                const float inv_r = rsqrtf(r2);
                const float rr = r2 * inv_r;
                const float s = -kb2 * (rr - r0[b]) * inv_r * sc;
                if (fdet) {     // a bond's orientation is fixed by its definition
                    put_fixed(fdet, i, s * dx, s * dy, s * dz);
                    put_fixed(fdet, j, -s * dx, -s * dy, -s * dz);
                } else {
                    scatter(f, i, s * dx, s * dy, s * dz);
                    scatter(f, j, -s * dx, -s * dy, -s * dz);
                }
                if (VIR) w.add(dx, dy, dz, s);
            }
        }
    }
    if (VIR) flush_virial(vir, w);
}

// K4b: angle term of Eq. 2, U = k (theta - theta0)^2, one thread per
// triplet (i, vertex j, k).  theta = atan2(|a x b|, a.b) for the arms
// a = x_i - x_j, b = x_k - x_j (accurate near 0 and pi, where arccos of the
// cosine loses digits); F_i = 2 k (theta - theta0) / sin(theta)
// (e_b - cos(theta) e_a) / |a|, F_k likewise, F_j = -F_i - F_k, with
// sin(theta) held at 1e-3 at least.
template <bool VIR>
__global__ void __launch_bounds__(MSM_TPB) k_angles(int64_t na, const int32_t *__restrict__ ijk,
                                                   const float *__restrict__ t0, float k2,
                                                   const float4 *__restrict__ x32, float4 *f, md_geom geom,
                                                   const md_dstate *ds, double *vir, md_due due, const int32_t *tag,
                                                   unsigned long long *fdet, const int2 *__restrict__ blk)
{
    vir6 w = {0, 0, 0, 0, 0, 0};
    // the CTAs stride over the blocks of MSM_TPB triplets, as in k_bonds
    const int64_t nblk = (na + MSM_TPB - 1) / MSM_TPB;
    for (int64_t vb = blockIdx.x; vb < nblk; vb += gridDim.x) {
        if (due.plt_k && !block_due(due, blk[vb])) continue;
        const int64_t q = vb * MSM_TPB + threadIdx.x;
        // the triplet lies on one platelet: it lives on that platelet's grid
        const float sc = (q < na && due.plt_k) ? term_scale(due, tag[ijk[3 * q + 1]], tag[ijk[3 * q + 1]]) : 1.0f;
        if (q < na && sc != 0.0f) {
            const int32_t i = ijk[3 * q], j = ijk[3 * q + 1], k = ijk[3 * q + 2];
            const float4 xj = x32[j];
            float ax, ay, az, bx, by, bz, vs;
            min_image_f32(geom, ds->le_offset_f, x32[i], xj, ax, ay, az, vs);
            min_image_f32(geom, ds->le_offset_f, x32[k], xj, bx, by, bz, vs);
            const float ia = rsqrtf(ax * ax + ay * ay + az * az), ib = rsqrtf(bx * bx + by * by + bz * bz);
            const float dot = ax * bx + ay * by + az * bz;
            const float cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
            const float crs = sqrtf(cx * cx + cy * cy + cz * cz);
            const float th = atan2f(crs, dot);
            const float c = dot * ia * ib;
            const float sn = fmaxf(crs * ia * ib, 1e-3f);
            const float g = k2 * (th - t0[q]) / sn * sc;
            const float eax = ax * ia, eay = ay * ia, eaz = az * ia, ebx = bx * ib, eby = by * ib, ebz = bz * ib;
            const float fix = g * (ebx - c * eax) * ia, fiy = g * (eby - c * eay) * ia, fiz = g * (ebz - c * eaz) * ia;
            const float fkx = g * (eax - c * ebx) * ib, fky = g * (eay - c * eby) * ib, fkz = g * (eaz - c * ebz) * ib;
            if (fdet) {     // a triplet's orientation is fixed by its definition
                // the vertex takes minus the sum of the two rounded ends, so the
                // triplet's terms cancel exactly
                const float S = 4294967296.0f;
                const long long qi[3] = {__float2ll_rn(fix * S), __float2ll_rn(fiy * S), __float2ll_rn(fiz * S)};
                const long long qk[3] = {__float2ll_rn(fkx * S), __float2ll_rn(fky * S), __float2ll_rn(fkz * S)};
    #pragma unroll
                for (int d = 0; d < 3; ++d) {
                    atomicAdd(&fdet[3 * (int64_t)i + d], (unsigned long long)qi[d]);
                    atomicAdd(&fdet[3 * (int64_t)k + d], (unsigned long long)qk[d]);
                    atomicAdd(&fdet[3 * (int64_t)j + d], (unsigned long long)(-(qi[d] + qk[d])));
                }
            } else {
                scatter(f, i, fix, fiy, fiz);
                scatter(f, k, fkx, fky, fkz);
                scatter(f, j, -(fix + fkx), -(fiy + fky), -(fiz + fkz));
            }
            if (VIR) {
                w.add_rf(ax, ay, az, fix, fiy, fiz);
                w.add_rf(bx, by, bz, fkx, fky, fkz);
            }
        }
    }
    if (VIR) flush_virial(vir, w);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)(n > 0 ? (n + MSM_TPB - 1) / MSM_TPB : 1); }
// bond and angle CTAs striding over their blocks of terms: eight resident
// per SM of the 152
constexpr unsigned TERM_BLOCKS = 1216;
inline unsigned term_grid(int64_t n) { return blocks_for(n) < TERM_BLOCKS ? blocks_for(n) : TERM_BLOCKS; }

}  // namespace

// Forces of the levels in level_mask, accumulated into out[level] (the
// buffers must be zero or hold partial sums of the same evaluation).
constexpr int FAST_BLOCKS = 608;   // warps grid-striding over the fast list (four blocks of 4 warps per SM)

static fast_args fast_for(md_system *s, const md_grid &g, const int32_t *members, float cut2)
{
    fast_args fa;
    fa.fast_idx = s->fast_idx;
    fa.fast_flag = s->fast_flag;
    fa.ctl = s->ctl;
    fa.fast_max = s->fast_max;
    fa.g = g;
    fa.members = members;
    fa.xb = s->xb;
    // partners at most a skin (plasma) or skin_plt / 2 (platelets) from their build cells
    fa.R = (float)(s->cfg.rc + (s->cfg.skin > s->skin_p ? s->cfg.skin : s->skin_p)) * (1.0f + 1e-5f);
    fa.cut2 = cut2;
    return fa;
}

// pair_args of the DPD levels (the fields the pair kernels read)
// The selectable variants of the DPD levels: the interface level's LJ
// conservative term (MD_CFG_IFACE_LJ) and the uniform noise variate
// (MD_CFG_UNIFORM_NOISE).
static void set_variants(md_system *s, pair_args &a, bool iface)
{
    const md_config &c = s->cfg;
    a.uniform_noise = (c.flags & MD_CFG_UNIFORM_NOISE) ? 1 : 0;
    const bool on = iface && (c.flags & MD_CFG_IFACE_LJ);
    const double rmin = pow(2.0, 1.0 / 6.0) * c.lj_sigma;
    a.wca_eps24 = (float)(24.0 * c.lj_eps);
    a.wca_sig2 = (float)(c.lj_sigma * c.lj_sigma);
    a.wca_rc2 = on ? (float)(rmin * rmin) : 0.0f;
}

// Deterministic mode: a level's fixed-point sums to its FP32 buffer.
__global__ void k_fixed_to_f4(int64_t n, const unsigned long long *__restrict__ q, float4 *f)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double u = 1.0 / 4294967296.0;
    f[k] = make_float4((float)((double)(long long)q[3 * k] * u), (float)((double)(long long)q[3 * k + 1] * u),
                       (float)((double)(long long)q[3 * k + 2] * u), 0.0f);
}

cudaError_t launch_fixed_to_f4(md_system *s, const unsigned long long *q, float4 *f)
{
    k_fixed_to_f4<<<blocks_for(s->n), MSM_TPB, 0, s->stream>>>(s->n, q, f);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

static pair_args dpd_args(md_system *s)
{
    const md_config &c = s->cfg;
    pair_args a;
    a.x32 = s->x32;
    a.v = s->v;
    a.geom = s->geom;
    a.ds = s->ds;
    a.key = make_uint2((uint32_t)(c.seed & 0xffffffffu), (uint32_t)(c.seed >> 32));
    a.gamma = (float)c.gamma;
    a.rc2 = (float)(c.rc * c.rc);
    a.inv_rc = (float)(1.0 / c.rc);
    a.vir = s->vir_acc;
    a.tag = s->tag_s;
    a.fdet = nullptr;
    set_variants(s, a, false);
    return a;
}

cudaError_t launch_fast_pairs(md_system *s, unsigned level_mask, float4 *const out[3], bool virial,
                              unsigned long long *fdet)
{
    const md_config &c = s->cfg;
    pair_args a = dpd_args(s);
    a.fdet = fdet;
    if (level_mask & MD_LEVEL_FLUID) {
        a.f = out[0];
        a.a_same = (float)c.a_ff;
        a.a_wall = (float)c.a_fw;
        a.sig_isdt = (float)(c.sigma / sqrt(c.dt));
        const fast_args fa = fast_for(s, s->gmain, nullptr, s->cut2[MD_LIST_FLUID]);
        if (fdet && virial) k_dpd_fast<true, false, true><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        else if (fdet) k_dpd_fast<false, false, true><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        else if (virial) k_dpd_fast<true, false><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        else k_dpd_fast<false, false><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        MSM_COUNT(s, 1);
    }
    if ((level_mask & MD_LEVEL_IFACE) && s->n_plt > 0) {
        const int km = s->cfg_k_m > 0 ? s->cfg_k_m : 1;
        a.f = out[1];
        a.a_same = (float)c.a_fp;
        a.a_wall = (float)c.a_fp;
        a.sig_isdt = (float)(c.sigma / sqrt(c.dt / km));
        set_variants(s, a, true);
        const fast_args fa = fast_for(s, s->gplt, s->plt_sorted, s->cut2[MD_LIST_IFACE]);
        if (fdet && virial) k_dpd_fast<true, true, true><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        else if (fdet) k_dpd_fast<false, true, true><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        else if (virial) k_dpd_fast<true, true><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        else k_dpd_fast<false, true><<<FAST_BLOCKS, 128, 0, s->stream>>>(a, fa);
        MSM_COUNT(s, 1);
    }
    return cudaGetLastError();
}

cudaError_t launch_forces(md_system *s, unsigned level_mask, float4 *const out[3], bool virial, bool with_fast,
                          unsigned long long *fdet)
{
    const md_config &c = s->cfg;
    pair_args a;
    a.fdet = fdet;
    a.x32 = s->x32;
    a.v = s->v;
    a.geom = s->geom;
    a.ds = s->ds;
    a.key = make_uint2((uint32_t)(c.seed & 0xffffffffu), (uint32_t)(c.seed >> 32));
    a.gamma = (float)c.gamma;
    a.rc2 = (float)(c.rc * c.rc);
    a.inv_rc = (float)(1.0 / c.rc);
    a.lj_eps24 = (float)(24.0 * c.lj_eps);
    a.lj_sig2 = (float)(c.lj_sigma * c.lj_sigma);
    a.lj_rc2 = (float)(c.lj_rc * c.lj_rc);
    // the printed form's alpha; MD_CFG_MORSE_STANDARD gives the standard
    // form's range a, and the printed form with alpha = 2 a r0 is the same curve
    const double m_alpha = (c.flags & MD_CFG_MORSE_STANDARD) ? 2.0 * c.morse_alpha * c.morse_r0 : c.morse_alpha;
    a.m_Da_r0 = (float)(c.morse_D * m_alpha / c.morse_r0);
    a.m_alpha = (float)m_alpha;
    a.m_inv_r0 = (float)(1.0 / c.morse_r0);
    a.m_rc2 = (float)(c.morse_rc * c.morse_rc);
    a.f_A = (float)c.f_A;
    a.vir = s->vir_acc;
    a.tag = s->tag_s;
    a.due.plt_k = s->due_on ? s->plt_k : nullptr;
    a.due.qe = s->due_q;
    a.due.K = s->plt_K;
    a.due.dtm = (float)s->due_dtm;
    const bool strided = a.due.plt_k && s->have_levels;      // the strides follow every build and ratio change
    a.due.stride = strided ? s->plt_stride : nullptr;
    a.due.row_stride = strided ? s->plt_row_stride : nullptr;
    const int km = s->cfg_k_m > 0 ? s->cfg_k_m : 1;
    set_variants(s, a, false);

    if (level_mask & MD_LEVEL_FLUID) {
        a.rows = s->n;
        a.row_idx = nullptr;
        a.nl = s->nl[MD_LIST_FLUID];
        a.nc = s->nc[MD_LIST_FLUID];
        a.cap = s->cap[MD_LIST_FLUID];
        a.f = out[0];
        a.a_same = (float)c.a_ff;
        a.a_wall = (float)c.a_fw;
        a.sig_isdt = (float)(c.sigma / sqrt(c.dt));
        if (fdet && virial) k_dpd<true, true, true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        else if (fdet) k_dpd<false, true, true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        else if (virial) k_dpd<true, true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        else k_dpd<false, true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        MSM_COUNT(s, 1);
    }
    if ((level_mask & MD_LEVEL_IFACE) && s->n_plt > 0) {
        a.rows = s->n_plt;
        a.row_idx = s->plt_sorted;
        a.nl = s->nl[MD_LIST_IFACE];
        a.nc = s->nc[MD_LIST_IFACE];
        a.cap = s->cap[MD_LIST_IFACE];
        a.f = out[1];
        a.a_same = (float)c.a_fp;
        a.a_wall = (float)c.a_fp;
        a.sig_isdt = (float)(c.sigma / sqrt(c.dt / km));
        set_variants(s, a, true);
        if (fdet && virial) k_dpd<true, false, true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        else if (fdet) k_dpd<false, false, true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        else if (virial) k_dpd<true, false><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        else k_dpd<false, false><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        MSM_COUNT(s, 1);
    }
    if ((level_mask & MD_LEVEL_PLT) && s->n_plt > 0) {
        if (s->nb > 0) {
            if (virial)
                k_bonds<true><<<term_grid(s->nb), MSM_TPB, 0, s->stream>>>(s->nb, s->bond_ij, s->bond_r0,
                                                                           (float)(2.0 * c.k_bond), s->x32, out[2],
                                                                           s->geom, s->ds, s->vir_acc, a.due, s->tag_s,
                                                                           a.fdet, s->bond_blk);
            else
                k_bonds<false><<<term_grid(s->nb), MSM_TPB, 0, s->stream>>>(s->nb, s->bond_ij, s->bond_r0,
                                                                            (float)(2.0 * c.k_bond), s->x32, out[2],
                                                                            s->geom, s->ds, s->vir_acc, a.due, s->tag_s,
                                                                           a.fdet, s->bond_blk);
        }
        if (s->na > 0) {
            if (virial)
                k_angles<true><<<term_grid(s->na), MSM_TPB, 0, s->stream>>>(
                    s->na, s->angle_ijk, s->angle_t0, (float)(2.0 * c.k_angle), s->x32, out[2], s->geom, s->ds,
                    s->vir_acc, a.due, s->tag_s, a.fdet, s->angle_blk);
            else
                k_angles<false><<<term_grid(s->na), MSM_TPB, 0, s->stream>>>(
                    s->na, s->angle_ijk, s->angle_t0, (float)(2.0 * c.k_angle), s->x32, out[2], s->geom, s->ds,
                    s->vir_acc, a.due, s->tag_s, a.fdet, s->angle_blk);
            MSM_COUNT(s, 1);
        }
        a.rows = s->n_plt;
        a.row_idx = s->plt_sorted;
        a.nl = s->nl[MD_LIST_LJ];
        a.nc = s->nc[MD_LIST_LJ];
        a.cap = s->cap[MD_LIST_LJ];
        a.f = out[2];
        if (virial) k_lj<true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        else k_lj<false><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        MSM_COUNT(s, 1 + (s->nb > 0 ? 1 : 0) + (s->n_rec > 0 ? 1 : 0));
        if (s->n_rec > 0) {
            a.rows = s->n_rec;
            a.row_idx = s->rec_sorted;
            a.nl = s->nl[MD_LIST_MORSE];
            a.nc = s->nc[MD_LIST_MORSE];
            a.cap = s->cap[MD_LIST_MORSE];
            if (virial) k_morse<true><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
            else k_morse<false><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && with_fast && (level_mask & (MD_LEVEL_FLUID | MD_LEVEL_IFACE)))
        e = launch_fast_pairs(s, level_mask, out, virial, fdet);
    return e;
}
