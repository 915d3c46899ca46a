// K2: Verlet-skin neighbour lists (Table 1, "neighbor lists construction").
//
// One thread per list row scans the cells within reach of its particle and
// appends every partner that passes the binary32 list predicate
//     r2 = (dx*dx + dy*dy) + dz*dz < (cut + skin)^2        (no FMA)
// computed from the minimum-image separation of min_image_f32(); a CPU
// evaluation of the same operation sequence yields the identical pair set.
//
// Half lists keep each unordered pair once, in the row of the particle that
// comes first in the grid's cell-sorted order; a row therefore only scans
// cells whose index is not below its own, half of the neighbourhood.
//
// Lists are built row-major ELL (entry k of row r at r*cap + k): a row's
// entries are contiguous, so a warp that streams the concatenated rows of 32
// consecutive particles reads them nearly coalesced; the plasma list is then
// repacked so that they are (below).  Row counts beyond the capacity are
// recorded (overflow bit + longest row) and never written.
//
//   MD_LIST_FLUID  rows: every particle (cell-sorted); later plasma/wall
//                  partners, plasma-plasma and plasma-wall pairs (Eq. 1);
//                  stored as warp streams (each warp's 32 rows back to back
//                  from its first row's slot, entry = j | lane << 27)
//   MD_LIST_IFACE  rows: platelet particles; partners: every plasma or wall
//                  particle (Eq. 3)
//   MD_LIST_LJ     rows: platelet particles in platelet sub-grid order; later
//                  platelet particles, excluding same-platelet pairs closer
//                  than lj_excl at rest (Eq. 2)
//   MD_LIST_MORSE  rows: receptor sites in receptor sub-grid order; later
//                  receptors of another platelet (Eq. 4)
#include "msm_internal.cuh"

namespace {

struct build_args {
    int64_t n;
    int64_t rows;
    const int32_t *row_idx;     // null: row r is particle r
    const float4 *x32;
    const int32_t *tag;
    const float4 *X0;           // rest positions by id (LJ kind)
    md_grid g;
    const int32_t *members;     // null: main grid
    md_geom geom;
    const md_dstate *ds;
    float R, cut2, excl2;
    int32_t *nl, *nc;
    int cap;
    int32_t *ctl;
    const int32_t *near;        // LJ / Morse kinds: platelets with a neighbour platelet in reach
    int near_bit;
    const float4 *bound;        // platelet bounding spheres (row-level test when P is small)
    int P;
    const int2 *cell_pid;       // LJ / Morse sub-grids: lowest and highest platelet id per cell
};

template <int KIND>
__global__ void __launch_bounds__(MSM_TPB) k_build(build_args a, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    constexpr bool HALF = KIND != MD_LIST_IFACE;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = r < a.rows;
    int cnt = 0;
    if (active) {
        const int32_t i = a.row_idx ? a.row_idx[r] : (int32_t)r;
        const float4 xi = a.x32[i];
        const int ci = class_of(xi);
        const float delta = a.ds->le_offset_f;
        if (KIND != MD_LIST_FLUID || ci != CLS_PLT) {
            int32_t ti = 0;
            float4 x0i = make_float4(0.f, 0.f, 0.f, 0.f);
            if (KIND == MD_LIST_LJ || KIND == MD_LIST_MORSE) ti = a.tag[i] & ~MD_RECEPTOR_BIT;
            // no other platelet within reach of this one's bounding sphere: no
            // partner can pass (same-platelet pairs need a rest distance of at
            // least lj_excl, which the caller rules out before using `near`)
            if ((KIND == MD_LIST_LJ || KIND == MD_LIST_MORSE) && a.near) {
                bool reach = (a.near[ti] & a.near_bit) != 0;
                if (reach && a.P <= 64) {   // this particle itself within reach of another sphere?
                    reach = false;
                    for (int q = 0; q < a.P && !reach; ++q) {
                        if (q == ti) continue;
                        const float4 bq = a.bound[q];
                        float dx = xi.x - bq.x, dy = xi.y - bq.y, dz = xi.z - bq.z;
                        dx -= a.geom.L[0] * rintf(dx / a.geom.L[0]);
                        dz -= a.geom.L[2] * rintf(dz / a.geom.L[2]);
                        if (!a.geom.walls) {
                            const float dy0 = dy;
                            dy -= a.geom.L[1] * rintf(dy / a.geom.L[1]);
                            if (a.geom.le && dy != dy0) dx = 0.0f;
                        }
                        const float lim = bq.w + a.R + 0.5f;
                        reach = dx * dx + dy * dy + dz * dz < lim * lim;
                    }
                }
                if (!reach) {
                    if (active) a.nc[r] = 0;
                    goto done;
                }
            }
            if (KIND == MD_LIST_LJ) x0i = a.X0[id_of(xi)];
            const int64_t rows = a.rows;
            // LJ / Morse without same-platelet pairs: cells holding only this
            // platelet's particles hold no partner
            const int2 *cp = (KIND == MD_LIST_LJ || KIND == MD_LIST_MORSE) && a.near ? a.cell_pid : nullptr;
            auto skip = [&](int c) {
                if (!cp) return false;
                const int2 q = cp[c];
                return q.x == ti && q.y == ti;
            };
            for_candidates<HALF>(a.g, a.geom, delta, xi, a.R, a.members, (int32_t)r, [&](int32_t s, int32_t j) {
                const float4 xj = a.x32[j];
                const int cj = class_of(xj);
                if (KIND == MD_LIST_FLUID) {
                    if (cj == CLS_PLT || (ci == CLS_WALL && cj == CLS_WALL)) return;
                } else if (KIND == MD_LIST_IFACE) {
                    if (cj == CLS_PLT) return;
                }
                float dx, dy, dz, vs;
                min_image_f32(a.geom, delta, xi, xj, dx, dy, dz, vs);
                if (!(r2_f32(dx, dy, dz) < a.cut2)) return;
                if (KIND == MD_LIST_LJ || KIND == MD_LIST_MORSE) {
                    const bool same = (a.tag[j] & ~MD_RECEPTOR_BIT) == ti;
                    if (KIND == MD_LIST_MORSE && same) return;
                    if (KIND == MD_LIST_LJ && same) {
                        const float4 x0j = a.X0[id_of(xj)];
                        const float ex = __fsub_rn(x0i.x, x0j.x), ey = __fsub_rn(x0i.y, x0j.y),
                                    ez = __fsub_rn(x0i.z, x0j.z);
                        if (r2_f32(ex, ey, ez) < a.excl2) return;
                    }
                }
                if (cnt < a.cap) a.nl[r * a.cap + cnt] = j;
                ++cnt;
            }, skip);
        }
    }
done:
    // every lane of the warp reaches the row bookkeeping (shuffle needs all)
    if (active) a.nc[r] = cnt;
    const int m = __reduce_max_sync(0xffffffffu, active ? cnt : 0);
    if ((threadIdx.x & 31) == 0 && m > 0) {
        atomicMax(&a.ctl[CTL_MAXROW + KIND], m);
        if (m > a.cap) atomicOr(&a.ctl[CTL_OVERFLOW], 1 << KIND);
    }
    if (KIND == MD_LIST_FLUID) {
        // Warp-stream layout for the force pass: the warp's 32 rows, written
        // one per slot of cap entries, are packed back to back from the first
        // row's slot, each entry carrying its row's lane.  In place: flat entry
        // f of row L (prefix P_L <= L cap) moves from L cap + f - P_L to f,
        // never above its source, and each round of 32 reads before it writes.
        const int lane = threadIdx.x & 31;
        const int64_t r0 = r - lane;
        const int c = active ? min(cnt, a.cap) : 0;
        int pre = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += t;
        }
        const int total = __shfl_sync(0xffffffffu, pre, 31);
        pre -= c;
        int32_t *slot = a.nl + r0 * a.cap;
        __syncwarp();      // the rows' entries, written by each lane, visible to the warp
        for (int base = 0; base < total; base += 32) {
            const int f = base + lane;
            int row = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int p = __shfl_sync(0xffffffffu, pre, row + step);
                if (p <= f) row += step;
            }
            const int k = f - __shfl_sync(0xffffffffu, pre, row);
            const int32_t e = f < total ? (slot[row * a.cap + k] | (row << MSM_STREAM_SHIFT)) : 0;
            __syncwarp();
            if (f < total) slot[f] = e;
            __syncwarp();
        }
    }
}

// AI-MTS drift strides.  cmask[p] collects the step ratios (bit k - 1) of
// the platelets that share an LJ or receptor list pair with p -- a superset
// of the pairs that can act before the next build -- and stride[p] = K /
// lcm(k_p, those ratios): every term that involves p (its own at multiples of
// K / k_p, a pair with q at multiples of K / max(k_p, k_q)) is due at
// multiples of stride[p] only.
__global__ void __launch_bounds__(256) k_zero_u64(unsigned long long *p, int n, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0ull;
}

__global__ void __launch_bounds__(MSM_TPB) k_contact_levels(int64_t rows, const int32_t *__restrict__ row_idx,
                                                            const int32_t *__restrict__ nl,
                                                            const int32_t *__restrict__ nc, int cap,
                                                            const int32_t *__restrict__ tag,
                                                            const int32_t *__restrict__ plt_k,
                                                            unsigned long long *cmask, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int c = min(nc[r], cap);
    if (c <= 0) return;
    const int32_t p = tag[row_idx[r]] & ~MD_RECEPTOR_BIT;
    const unsigned long long bit_p = 1ull << (plt_k[p] - 1);
    unsigned long long mine = 0ull;
    int32_t last = -1;
    for (int e = 0; e < c; ++e) {
        const int32_t q = tag[nl[r * (int64_t)cap + e]] & ~MD_RECEPTOR_BIT;
        if (q == p) continue;
        mine |= 1ull << (plt_k[q] - 1);
        if (q != last) {           // partners of one platelet tend to come in runs
            atomicOr(&cmask[q], bit_p);
            last = q;
        }
    }
    if (mine) atomicOr(&cmask[p], mine);
}

__global__ void __launch_bounds__(256) k_strides(int P, int K, const int32_t *__restrict__ plt_k,
                                                 const unsigned long long *__restrict__ cmask, int32_t *stride,
                                                 const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int L = plt_k[p];
    for (unsigned long long m = cmask[p]; m; m &= m - 1) {
        const int k = __ffsll((long long)m);     // the ratio of bit k - 1
        int a = L, b = k;
        while (b) { const int t = a % b; a = b; b = t; }
        L = L / a * k;
    }
    stride[p] = K / L;      // every ratio divides K, so L does
}

__global__ void __launch_bounds__(MSM_TPB) k_row_strides(int64_t rows, const int32_t *__restrict__ row_idx,
                                                         const int32_t *__restrict__ tag,
                                                         const int32_t *__restrict__ stride, int32_t *row_stride,
                                                         const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) row_stride[r] = stride[tag[row_idx[r]] & ~MD_RECEPTOR_BIT];
}

// Bounding sphere of every platelet at the build, over blocks (p, chunk):
// pass 1 sums the member offsets from the first member (minimum image) into
// bound[p].xyz, pass 2 the largest squared distance from the centre of mass
// into bound[p].w (float bits; k_plt_near turns both into centre and radius).
__global__ void __launch_bounds__(256) k_plt_com(const int32_t *__restrict__ off, const int32_t *__restrict__ ids,
                                                 const int32_t *__restrict__ pos_of_id, const float4 *__restrict__ x32,
                                                 md_geom geom, const md_dstate *ds, float4 *bound, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int p = blockIdx.x, b = off[p], e = off[p + 1];
    const float4 ref = x32[pos_of_id[ids[b]]];
    const float delta = ds->le_offset_f;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int m = b + blockIdx.y * blockDim.x + threadIdx.x; m < e; m += gridDim.y * blockDim.x) {
        float dx, dy, dz, vs;
        min_image_f32(geom, delta, x32[pos_of_id[ids[m]]], ref, dx, dy, dz, vs);
        sx += dx; sy += dy; sz += dz;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&bound[p].x, sx);
        atomicAdd(&bound[p].y, sy);
        atomicAdd(&bound[p].z, sz);
    }
}

__global__ void __launch_bounds__(256) k_plt_radius(const int32_t *__restrict__ off, const int32_t *__restrict__ ids,
                                                    const int32_t *__restrict__ pos_of_id,
                                                    const float4 *__restrict__ x32, md_geom geom, const md_dstate *ds,
                                                    float4 *bound, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int p = blockIdx.x, b = off[p], e = off[p + 1];
    const float4 ref = x32[pos_of_id[ids[b]]];
    const float delta = ds->le_offset_f;
    const float inv_n = 1.0f / (float)(e - b);
    const float cx = bound[p].x * inv_n, cy = bound[p].y * inv_n, cz = bound[p].z * inv_n;
    float r2 = 0.f;
    for (int m = b + blockIdx.y * blockDim.x + threadIdx.x; m < e; m += gridDim.y * blockDim.x) {
        float dx, dy, dz, vs;
        min_image_f32(geom, delta, x32[pos_of_id[ids[m]]], ref, dx, dy, dz, vs);
        dx -= cx; dy -= cy; dz -= cz;
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
    r2 = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(r2)));   // r2 >= 0
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned *)&bound[p].w, __float_as_uint(r2));
}

// near[p] bit 0 (1): some other platelet's bounding sphere comes within the
// LJ (Morse) list reach of p's.  Under Lees-Edwards the x separation of a
// pair across the y boundary is taken as zero (its image offset varies).
__global__ void k_plt_near(const int32_t *__restrict__ off, const int32_t *__restrict__ ids,
                           const int32_t *__restrict__ pos_of_id, const float4 *__restrict__ x32, float4 *bound, int P,
                           md_geom geom, float reach_lj, float reach_m, int32_t *near, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    // sums and squared radii -> centre of mass and radius
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const float4 ref = x32[pos_of_id[ids[off[p]]]];
        const float4 a = bound[p];
        const float inv_n = 1.0f / (float)(off[p + 1] - off[p]);
        bound[p] = make_float4(ref.x + a.x * inv_n, ref.y + a.y * inv_n, ref.z + a.z * inv_n,
                               sqrtf(__uint_as_float(__float_as_uint(a.w))));
    }
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const float4 bp = bound[p];
        int bits = 0;
        for (int q = 0; q < P && bits != 3; ++q) {
            if (q == p) continue;
            const float4 bq = bound[q];
            float dx = bp.x - bq.x, dy = bp.y - bq.y, dz = bp.z - bq.z;
            dz -= geom.L[2] * rintf(dz / geom.L[2]);
            bool crossed = false;
            if (!geom.walls) {
                const float dy0 = dy;
                dy -= geom.L[1] * rintf(dy / geom.L[1]);
                crossed = dy != dy0;
            }
            dx -= geom.L[0] * rintf(dx / geom.L[0]);
            if (geom.le && crossed) dx = 0.0f;
            const float d = sqrtf(dx * dx + dy * dy + dz * dz) - bp.w - bq.w;
            if (d < reach_lj + 0.5f) bits |= 1;
            if (d < reach_m + 0.5f) bits |= 2;
        }
        near[p] = bits;
    }
}

// Lowest and highest platelet id among the members of every sub-grid cell
// (empty cells: (INT_MAX, -1)).
__global__ void k_cell_pid(int64_t ncell, const int32_t *__restrict__ start, const int32_t *__restrict__ members,
                           const int32_t *__restrict__ tag, int2 *out, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int lo = 0x7fffffff, hi = -1;
    for (int32_t s = start[c]; s < start[c + 1]; ++s) {
        const int p = tag[members[s]] & ~MD_RECEPTOR_BIT;
        lo = min(lo, p);
        hi = max(hi, p);
    }
    out[c] = make_int2(lo, hi);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)(n > 0 ? (n + MSM_TPB - 1) / MSM_TPB : 1); }

}  // namespace

cudaError_t launch_build_lists(md_system *s, const int32_t *gate)
{
    const float margin = 1.0f + 1e-5f;
    build_args a;
    a.n = s->n;
    a.x32 = s->x32;
    a.tag = s->tag_s;
    a.X0 = s->X0;
    a.geom = s->geom;
    a.ds = s->ds;
    a.ctl = s->ctl;
    a.excl2 = s->excl2;
    a.near = nullptr;
    a.near_bit = 0;
    a.bound = nullptr;
    a.P = 0;
    a.cell_pid = nullptr;

    // plasma / wall list over the main grid
    a.rows = s->n;
    a.row_idx = nullptr;
    a.g = s->gmain;
    a.members = nullptr;
    a.R = (float)(s->cfg.rc + s->cfg.skin) * margin;
    a.cut2 = s->cut2[MD_LIST_FLUID];
    a.nl = s->nl[MD_LIST_FLUID];
    a.nc = s->nc[MD_LIST_FLUID];
    a.cap = s->cap[MD_LIST_FLUID];
    k_build<MD_LIST_FLUID><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a, gate);

    if (s->n_plt > 0) {
        // interface: platelet rows (platelet sub-grid order) against the main grid
        a.rows = s->n_plt;
        a.row_idx = s->plt_sorted;
        a.R = (float)(s->cfg.rc + 0.5 * (s->cfg.skin + s->skin_p)) * margin;
        a.cut2 = s->cut2[MD_LIST_IFACE];
        a.nl = s->nl[MD_LIST_IFACE];
        a.nc = s->nc[MD_LIST_IFACE];
        a.cap = s->cap[MD_LIST_IFACE];
        k_build<MD_LIST_IFACE><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a, gate);

        // platelets far from every other platelet get empty LJ / Morse rows
        // without a scan (only when no same-platelet pair can feel LJ)
        const bool prefilter = s->cfg.lj_excl > 1e20;
        if (prefilter) {
            const int P = s->cfg.n_platelets;
            const int64_t per = s->n_plt / P / 256 + 1;
            const int chunks = (int)(per < 256 ? per : 256);
            cudaError_t e = cudaMemsetAsync(s->plt_bound, 0, sizeof(float4) * P, s->stream);
            if (e != cudaSuccess) return e;
            k_plt_com<<<dim3(P, chunks), 256, 0, s->stream>>>(s->plt_off, s->plt_ids, s->pos_of_id, s->x32, s->geom,
                                                               s->ds, s->plt_bound, gate);
            k_plt_radius<<<dim3(P, chunks), 256, 0, s->stream>>>(s->plt_off, s->plt_ids, s->pos_of_id, s->x32,
                                                                  s->geom, s->ds, s->plt_bound, gate);
            k_plt_near<<<1, 256, 0, s->stream>>>(s->plt_off, s->plt_ids, s->pos_of_id, s->x32, s->plt_bound, P,
                                                 s->geom, (float)(s->cfg.lj_rc + s->skin_p),
                                                 (float)(s->cfg.morse_rc + s->skin_p), s->plt_near, gate);
        }
        a.near = prefilter ? s->plt_near : nullptr;
        a.near_bit = 1;
        a.bound = s->plt_bound;
        a.P = s->cfg.n_platelets;
        if (prefilter)
            k_cell_pid<<<blocks_for(s->gplt.ncell), MSM_TPB, 0, s->stream>>>(s->gplt.ncell, s->gplt.start, s->plt_sorted,
                                                                            s->tag_s, s->cell_pid, gate);
        a.cell_pid = s->cell_pid;
        a.g = s->gplt;
        a.members = s->plt_sorted;
        a.R = (float)(s->cfg.lj_rc + s->skin_p) * margin;
        a.cut2 = s->cut2[MD_LIST_LJ];
        a.nl = s->nl[MD_LIST_LJ];
        a.nc = s->nc[MD_LIST_LJ];
        a.cap = s->cap[MD_LIST_LJ];
        k_build<MD_LIST_LJ><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a, gate);

        if (s->n_rec > 0) {
            a.rows = s->n_rec;
            a.row_idx = s->rec_sorted;
            a.g = s->grec;
            a.members = s->rec_sorted;
            a.R = (float)(s->cfg.morse_rc + s->skin_p) * margin;
            a.near_bit = 2;
            if (prefilter)
                k_cell_pid<<<blocks_for(s->grec.ncell), MSM_TPB, 0, s->stream>>>(s->grec.ncell, s->grec.start,
                                                                                s->rec_sorted, s->tag_s, s->cell_pid,
                                                                                gate);
            a.cut2 = s->cut2[MD_LIST_MORSE];
            a.nl = s->nl[MD_LIST_MORSE];
            a.nc = s->nc[MD_LIST_MORSE];
            a.cap = s->cap[MD_LIST_MORSE];
            k_build<MD_LIST_MORSE><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a, gate);
        }
    }
    if (s->n_plt > 0 && s->have_levels) {
        cudaError_t e = launch_strides(s, gate);
        if (e != cudaSuccess) return e;
    }
    MSM_COUNT(s, 1 + (s->n_plt > 0 ? 2 + (s->n_rec > 0 ? 1 : 0) + (s->cfg.lj_excl > 1e20 ? 4 + (s->n_rec > 0 ? 1 : 0) : 0) : 0));
    return cudaGetLastError();
}

cudaError_t launch_strides(md_system *s, const int32_t *gate)
{
    const int P = s->cfg.n_platelets;
    if (s->n_plt <= 0 || P <= 0 || !s->plt_stride) return cudaSuccess;
    k_zero_u64<<<(P + 255) / 256, 256, 0, s->stream>>>(s->plt_cmask, P, gate);
    k_contact_levels<<<blocks_for(s->n_plt), MSM_TPB, 0, s->stream>>>(
        s->n_plt, s->plt_sorted, s->nl[MD_LIST_LJ], s->nc[MD_LIST_LJ], s->cap[MD_LIST_LJ], s->tag_s, s->plt_k,
        s->plt_cmask, gate);
    int n = 3;
    if (s->n_rec > 0) {
        k_contact_levels<<<blocks_for(s->n_rec), MSM_TPB, 0, s->stream>>>(
            s->n_rec, s->rec_sorted, s->nl[MD_LIST_MORSE], s->nc[MD_LIST_MORSE], s->cap[MD_LIST_MORSE], s->tag_s,
            s->plt_k, s->plt_cmask, gate);
        ++n;
    }
    k_strides<<<(P + 255) / 256, 256, 0, s->stream>>>(P, s->plt_K, s->plt_k, s->plt_cmask, s->plt_stride, gate);
    k_row_strides<<<blocks_for(s->n_plt), MSM_TPB, 0, s->stream>>>(s->n_plt, s->plt_sorted, s->tag_s, s->plt_stride,
                                                                  s->plt_row_stride, gate);
    MSM_COUNT(s, n + 1);
    return cudaGetLastError();
}

