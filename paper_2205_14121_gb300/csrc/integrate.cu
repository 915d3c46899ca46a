// K6/K7: velocity-Verlet kicks and drifts of the multi-level loop (Table 1)
// with the rebuild check fused into the drift.
//
//  kick   v += sum_l h_l f_l  (+ h_fluid g x^: the body force belongs to the
//         fluid level)
//  drift  x64 += dt v (FP64 master positions), then the boundary:
//           walls   bounce-back at y = 0 and y = Ly (position mirrored,
//                   velocity reversed: no-slip, Sec. 3.1)
//           LE      crossing y moves x by -/+ delta and v_x by -/+ rate*Ly
//           periodic wrap in x, z (and y without walls)
//         x32 = (float)x64; |x32 - x_build| (minimum image) against the
//         skin threshold -> rebuild flag; NaN / escape -> unstable flag.
//  zero   the level buffers the next force evaluation accumulates into.
#include "msm_internal.cuh"

namespace {

struct kd_args {
    int64_t n;
    const int32_t *idx;    // null: thread k handles particle k; else particle idx[k]
    double *xs, *ys, *zs;
    float4 *x32, *v;
    float4 *f[3];
    const float4 *xb;
    const int32_t *tag;
    float h[3];            // kick factor per level (0: level not kicked)
    int kick_which;        // DRIFT_* selector of kicked particles, -1: none
    int drift_which;       // DRIFT_* selector of drifted particles, -1: none
    unsigned zero_levels;
    int nf;
    float g;
    double dt;
    double L[3];
    double wall;
    double shear_v;
    float skin_half, margin, skin;
    float skin_p;          // skin of the platelet particles
    md_geom geom;
    const md_dstate *ds;
    int32_t *ctl;
    int sparse_level;      // >= 0: a pure kick with this level only (most forces zero)
    int32_t *fast_idx;     // plasma beyond skin/2 and within the skin: listed here
    uint32_t *fast_flag;
    int64_t fast_max;
    const int32_t *row_stride;  // AI-MTS substep q of the K grid: drift stride of each platelet row (null: every substep)
    int q;
};

__device__ __forceinline__ bool selected(int which, int32_t t)
{
    if (which < 0 || t == MD_TAG_WALL) return false;
    if (which == DRIFT_ALL) return true;
    if (which == DRIFT_FLUID) return t < 0;
    return t >= 0;
}

// Rebuild check of particle k (storage slot, tag t) at position xn against
// its position at the last build.  The margin covers platelet particles,
// which keep drifting in the inner substeps after this check and before the
// rebuild point at the end of the interface substep; plasma does not move in
// between.  Plasma up to twice the threshold keeps the lists: its pairs that
// they lack are evaluated by the fast-particle pass (every partner within rc
// is then in a list or found there).
__device__ __forceinline__ void check_moved(const kd_args &a, int64_t k, int32_t t, float4 xn)
{
    float dx, dy, dz, vs;
    min_image_f32(a.geom, a.ds->le_offset_f, xn, a.xb[k], dx, dy, dz, vs);
    const float d2 = dx * dx + dy * dy + dz * dz;
    const float mg = t >= 0 ? a.margin : 0.0f;
    const float sk = t >= 0 ? a.skin_p : a.skin;
    float thr = 0.5f * sk - mg;
    if (a.geom.le) {
        float dd = fabsf(a.ds->le_offset_f - a.ds->le_build_f);
        dd = fminf(dd, a.geom.L[0] - dd);
        thr = 0.5f * (sk - dd) - mg;
    }
    if (!(d2 <= thr * thr) || thr <= 0.0f) {
        int q = -1;
        if (t == MD_TAG_FLUID && thr > 0.0f && d2 <= 4.0f * thr * thr) {
            q = atomicAdd(&a.ctl[CTL_NFAST], 1);
            if (q < a.fast_max) {
                a.fast_idx[q] = (int32_t)k;
                a.fast_flag[k] = a.ds->fast_stamp;
            }
        }
        if (q < 0 || q >= a.fast_max) a.ctl[CTL_REBUILD] = 1;
    }
}

__global__ void __launch_bounds__(MSM_TPB) k_kick_drift(kd_args a)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n) return;
    double dt = a.dt;
    if (a.row_stride) {
        // AI-MTS platelet rows: every term that involves this row's platelet
        // is due at multiples of its stride only, so no force acts on it in
        // between: it is kicked and moved there, by stride substeps at once
        const int st = a.row_stride[r];
        if (a.q % st != 0) return;
        dt *= st;
    }
    const int64_t k = a.idx ? a.idx[r] : r;
    if (a.sparse_level >= 0) {
        // interface half kicks: only particles near a platelet carry a force
        const float4 fl = a.f[a.sparse_level][k];
        if (fl.x == 0.0f && fl.y == 0.0f && fl.z == 0.0f) return;
    }
    const int32_t t = a.tag[k];
    const bool kick = selected(a.kick_which, t);
    const bool drift = selected(a.drift_which, t);
    unsigned zero_seen = 0u;   // levels read as exactly zero: no need to clear them
    if (kick || drift) {
        float4 vv = a.v[k];
        if (kick) {
            float ax = 0.f, ay = 0.f, az = 0.f;
            for (int l = 0; l < a.nf; ++l) {
                if (a.h[l] == 0.0f || (l == 2 && t < 0)) continue;   // platelet-level forces act on platelets only
                const float4 fl = a.f[l][k];
                if (fl.x == 0.0f && fl.y == 0.0f && fl.z == 0.0f) zero_seen |= 1u << l;
                ax += a.h[l] * fl.x; ay += a.h[l] * fl.y; az += a.h[l] * fl.z;
            }
            ax += a.h[0] * a.g;
            vv.x += ax;
            vv.y += ay;
            vv.z += az;
        }
        if (drift) {
            // FP64 master update; FP64 instructions are rare on this part, so
            // the wrap decisions are taken on the rounded FP32 copies (a
            // double >= L always rounds to a float >= (float)L) and the FP64
            // arithmetic is redone only for the few particles that wrap.
            double x = fma(dt, (double)vv.x, a.xs[k]);
            double y = fma(dt, (double)vv.y, a.ys[k]);
            double z = fma(dt, (double)vv.z, a.zs[k]);
            const double Lx = a.L[0], Ly = a.L[1], Lz = a.L[2];
            float xf = (float)x, yf = (float)y, zf = (float)z;
            if (a.geom.walls) {
                // bounce-back: retrace the overshoot beyond the wall with the
                // reversed velocity (independent of drift substepping)
                if (yf < 0.0f || yf >= a.geom.L[1]) {
                    const double wall = y < 0.0 ? 0.0 : (y >= Ly ? Ly : -1.0);
                    if (wall >= 0.0) {
                        const double tau = vv.y != 0.0f ? (y - wall) / (double)vv.y : 0.0;
                        x -= 2.0 * (double)vv.x * tau;
                        z -= 2.0 * (double)vv.z * tau;
                        y = 2.0 * wall - y;
                        vv.x = -vv.x; vv.y = -vv.y; vv.z = -vv.z;
                        xf = (float)x; yf = (float)y; zf = (float)z;
                    }
                }
            } else if (a.geom.le) {
                const double delta = a.ds->le_offset;
                if (y >= Ly) {
                    y -= Ly; x -= delta; vv.x -= (float)a.shear_v;
                } else if (y < 0.0) {
                    y += Ly; x += delta; vv.x += (float)a.shear_v;
                }
                xf = (float)x; yf = (float)y;
            } else if (yf >= a.geom.L[1] || yf < 0.0f) {
                y += yf < 0.0f ? Ly : -Ly;
                yf = (float)y;
            }
            for (int rep = 0; rep < 2 && (xf >= a.geom.L[0] || xf < 0.0f); ++rep) {
                x += xf < 0.0f ? Lx : -Lx;   // a Lees-Edwards shift can add one more period
                xf = (float)x;
            }
            if (zf >= a.geom.L[2] || zf < 0.0f) {
                z += zf < 0.0f ? Lz : -Lz;
                zf = (float)z;
            }
            a.xs[k] = x; a.ys[k] = y; a.zs[k] = z;
            float4 xn = a.x32[k];
            xn.x = xf; xn.y = yf; xn.z = zf;
            a.x32[k] = xn;
            check_moved(a, k, t, xn);
            const bool bad = !(fabsf(xf) + fabsf(yf) + fabsf(zf) < 1e30f) ||
                             !(fabsf(vv.x) + fabsf(vv.y) + fabsf(vv.z) < 1e30f) ||
                             (a.geom.walls && (yf < -(float)a.wall || yf > a.geom.L[1] + (float)a.wall));
            if (bad) a.ctl[CTL_UNSTABLE] = 1;
        }
        a.v[k] = vv;
    }
    for (int l = 0; l < a.nf; ++l)
        if (((a.zero_levels & ~zero_seen) & (1u << l)) && !(l == 2 && t < 0)) a.f[l][k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Set the device time index (n, c) and the time n dt + c dt_m + q dt_p;
// recompute the Lees-Edwards offset and check its drift since the build.
__global__ void k_set_time(md_dstate *ds, int64_t n, int32_t c, double t, double rate_Ly, double Lx, int le,
                           float skin, float margin, int32_t *ctl)
{
    ds->step = n;
    ds->sub = c;
    ds->time = t;
    if (le) {
        double d = fmod(rate_Ly * t, Lx);
        if (d < 0.0) d += Lx;
        ds->le_offset = d;
        ds->le_offset_f = (float)d;
        float dd = fabsf(ds->le_offset_f - ds->le_build_f);
        dd = fminf(dd, (float)Lx - dd);
        if (0.5f * (skin - dd) - margin <= 0.0f) ctl[CTL_REBUILD] = 1;
    }
}

// Start of an outer step: its base index is the count of steps begun; in a
// captured loop, also count down and steer the WHILE node.
__global__ void k_outer_begin(md_dstate *ds, cudaGraphConditionalHandle loop, int use_loop)
{
    ds->base = ds->done;
    ds->done += 1;
    if (use_loop) {
        ds->steps_left -= 1;
        cudaGraphSetConditional(loop, ds->steps_left > 0 ? 1u : 0u);
    }
}

// Time index relative to the current outer step: (base + dn, c), time
// base*dt + t_off; Lees-Edwards offset and its drift check as k_set_time.
__global__ void k_time_rel(md_dstate *ds, int dn, int c, double t_off, double dt, double rate_Ly, double Lx,
                           int le, float skin, float margin, int32_t *ctl)
{
    const int64_t n = ds->base + dn;
    const double t = (double)ds->base * dt + t_off;
    ds->step = n;
    ds->sub = c;
    ds->time = t;
    if (le) {
        double d = fmod(rate_Ly * t, Lx);
        if (d < 0.0) d += Lx;
        ds->le_offset = d;
        ds->le_offset_f = (float)d;
        float dd = fabsf(ds->le_offset_f - ds->le_build_f);
        dd = fminf(dd, (float)Lx - dd);
        if (0.5f * (skin - dd) - margin <= 0.0f) ctl[CTL_REBUILD] = 1;
    }
}

__global__ void k_cond_rebuild(const int32_t *ctl, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, ctl[CTL_REBUILD] ? 1u : 0u);
}

__global__ void k_set_loop(md_dstate *ds, int64_t n) { ds->steps_left = n; }

// Outer-step counters at step n (a new state set at time index n).
__global__ void k_set_counters(md_dstate *ds, int64_t n)
{
    ds->base = n;
    ds->done = n;
}

// Before a drift of the plasma: an empty fast list under a new stamp.
__global__ void k_fast_reset(md_dstate *ds, int32_t *ctl)
{
    ds->fast_stamp += 1;
    ctl[CTL_NFAST] = 0;
}

__global__ void k_zero_f4(float4 *p, int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// A new state in the current storage order (md_set_xv keeping the lists):
// slot q takes the values of the particle it holds (id from the position
// word), read from the id-ordered upload; the id / tag bits stay.  Gathered
// by slot, so the random accesses are reads and every write is coalesced.
__global__ void k_place_x(int64_t n, const double *__restrict__ aos, double *xs, double *ys, double *zs, float4 *x32)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float4 p = x32[q];
    const int64_t k = id_of(p);
    const double x = aos[3 * k], y = aos[3 * k + 1], z = aos[3 * k + 2];
    xs[q] = x; ys[q] = y; zs[q] = z;
    p.x = (float)x; p.y = (float)y; p.z = (float)z;
    x32[q] = p;
}

__global__ void k_place_v(int64_t n, const double *__restrict__ aos, const float4 *__restrict__ x32, float4 *v)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t k = id_of(x32[q]);
    float4 u = v[q];
    u.x = (float)aos[3 * k]; u.y = (float)aos[3 * k + 1]; u.z = (float)aos[3 * k + 2];
    v[q] = u;
}

// The rebuild check of the kick-drift on every particle of a placed state
// (walls included, held to the plasma threshold); NaN / escape -> unstable.
__global__ void __launch_bounds__(MSM_TPB) k_check_placed(kd_args a)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const float4 xn = a.x32[k];
    check_moved(a, k, a.tag[k], xn);
    const float4 vv = a.v[k];
    const bool bad = !(fabsf(xn.x) + fabsf(xn.y) + fabsf(xn.z) < 1e30f) ||
                     !(fabsf(vv.x) + fabsf(vv.y) + fabsf(vv.z) < 1e30f) ||
                     (a.geom.walls && (xn.y < -(float)a.wall || xn.y > a.geom.L[1] + (float)a.wall));
    if (bad) a.ctl[CTL_UNSTABLE] = 1;
}

inline unsigned blocks_for(int64_t n) { return (unsigned)(n > 0 ? (n + MSM_TPB - 1) / MSM_TPB : 1); }

kd_args base_args(md_system *s)
{
    kd_args a;
    a.n = s->n;
    a.idx = nullptr;
    a.xs = s->xs; a.ys = s->ys; a.zs = s->zs;
    a.x32 = s->x32; a.v = s->v;
    for (int l = 0; l < 3; ++l) { a.f[l] = s->f[l]; a.h[l] = 0.0f; }
    a.nf = s->n_plt > 0 ? 3 : 1;
    a.xb = s->xb;
    a.tag = s->tag_s;
    a.g = (float)s->cfg.body_force;
    a.dt = 0.0;
    for (int d = 0; d < 3; ++d) a.L[d] = s->cfg.box[d];
    a.wall = s->cfg.wall;
    a.shear_v = s->cfg.shear_rate * s->cfg.box[1];
    a.skin = (float)s->cfg.skin;
    a.skin_half = 0.5f * (float)s->cfg.skin;
    a.skin_p = (float)s->skin_p;
    a.margin = s->margin;
    a.geom = s->geom;
    a.ds = s->ds;
    a.ctl = s->ctl;
    a.kick_which = -1;
    a.drift_which = -1;
    a.zero_levels = 0;
    a.sparse_level = -1;
    a.fast_idx = s->fast_idx;
    a.fast_flag = s->fast_flag;
    a.fast_max = s->fast_max;
    a.row_stride = nullptr;
    a.q = 0;
    return a;
}

}  // namespace

// Kick (per-level factors h[3], selector kick_which) + drift by dt of the
// drift_which subset + zeroing of zero_levels.  plt_rows: iterate only over
// the platelet particles (the subset rows) instead of every particle.
cudaError_t launch_kick_drift(md_system *s, const float h[3], int kick_which, double dt, int drift_which,
                              unsigned zero_levels, bool plt_rows, int stride_q)
{
    kd_args a = base_args(s);
    if (stride_q >= 0 && plt_rows && s->have_levels && s->plt_row_stride) {
        a.row_stride = s->plt_row_stride;
        a.q = stride_q;
    }
    for (int l = 0; l < 3; ++l) a.h[l] = h[l];
    a.kick_which = kick_which;
    a.drift_which = drift_which;
    a.dt = dt;
    a.zero_levels = zero_levels;
    a.sparse_level = -1;
    if (drift_which < 0 && zero_levels == 0u && h[0] == 0.0f && h[2] == 0.0f && h[1] != 0.0f) a.sparse_level = 1;
    if (plt_rows) {
        a.idx = s->plt_sorted;
        a.n = s->n_plt;
    }
    if (a.n <= 0) return cudaSuccess;
    if (!plt_rows && (drift_which == DRIFT_ALL || drift_which == DRIFT_FLUID)) {
        k_fast_reset<<<1, 1, 0, s->stream>>>(s->ds, s->ctl);
        MSM_COUNT(s, 1);
    }
    k_kick_drift<<<blocks_for(a.n), MSM_TPB, 0, s->stream>>>(a);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_place_state(md_system *s, const double *x_dev, bool velocities)
{
    if (velocities) k_place_v<<<blocks_for(s->n), MSM_TPB, 0, s->stream>>>(s->n, x_dev, s->x32, s->v);
    else k_place_x<<<blocks_for(s->n), MSM_TPB, 0, s->stream>>>(s->n, x_dev, s->xs, s->ys, s->zs, s->x32);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_check_placed(md_system *s, int64_t step0)
{
    k_set_counters<<<1, 1, 0, s->stream>>>(s->ds, step0);
    MSM_COUNT(s, 1);
    kd_args a = base_args(s);
    a.margin = 0.05f;        // the larger of the two schedules' margins
    k_fast_reset<<<1, 1, 0, s->stream>>>(s->ds, s->ctl);
    k_check_placed<<<blocks_for(s->n), MSM_TPB, 0, s->stream>>>(a);
    MSM_COUNT(s, 2);
    return cudaGetLastError();
}

cudaError_t launch_set_time(md_system *s, int64_t n, int32_t c, double t)
{
    const md_config &cf = s->cfg;
    k_set_time<<<1, 1, 0, s->stream>>>(s->ds, n, c, t, cf.shear_rate * cf.box[1], cf.box[0], s->geom.le,
                                       (float)(cf.skin < s->skin_p ? cf.skin : s->skin_p), s->margin, s->ctl);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_outer_begin(md_system *s, cudaGraphConditionalHandle loop, bool use_loop)
{
    k_outer_begin<<<1, 1, 0, s->stream>>>(s->ds, loop, use_loop ? 1 : 0);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_time_rel(md_system *s, int dn, int c, double t_off)
{
    const md_config &cf = s->cfg;
    k_time_rel<<<1, 1, 0, s->stream>>>(s->ds, dn, c, t_off, cf.dt, cf.shear_rate * cf.box[1], cf.box[0], s->geom.le,
                                       (float)(cf.skin < s->skin_p ? cf.skin : s->skin_p), s->margin, s->ctl);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_cond_rebuild(md_system *s, cudaGraphConditionalHandle h)
{
    k_cond_rebuild<<<1, 1, 0, s->stream>>>(s->ctl, h);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_set_loop(md_system *s, int64_t n)
{
    k_set_loop<<<1, 1, 0, s->stream>>>(s->ds, n);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}

cudaError_t launch_zero_forces(md_system *s, unsigned levels)
{
    const int nf = s->n_plt > 0 ? 3 : 1;
    for (int l = 0; l < nf; ++l)
        if (levels & (1u << l)) {
            k_zero_f4<<<blocks_for(s->n), MSM_TPB, 0, s->stream>>>(s->f[l], s->n);
            MSM_COUNT(s, 1);
        }
    return cudaGetLastError();
}
