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
// Lists are row-major ELL (entry k of row r at r*cap + k): a row's entries
// are contiguous, so a warp that streams the concatenated rows of 32
// consecutive particles reads them nearly coalesced.  Row counts beyond the
// capacity are recorded (overflow bit + longest row) and never written.
//
//   MD_LIST_FLUID  rows: every particle (cell-sorted); later plasma/wall
//                  partners, plasma-plasma and plasma-wall pairs (Eq. 1)
//   MD_LIST_IFACE  rows: platelet particles; partners: every plasma or wall
//                  particle (Eq. 3)
//   MD_LIST_LJ     rows: platelet particles in platelet sub-grid order; later
//                  platelet particles, excluding same-platelet pairs closer
//                  than lj_excl at rest (Eq. 2)
//   MD_LIST_MORSE  rows: receptor sites in receptor sub-grid order; later
//                  receptors of another platelet (Eq. 4)
#include "msm_internal.cuh"

namespace {

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
// [-2, n+1] and to at most n cells, so that a non-finite or escaped position
// (reported by the integrator's unstable flag) still gives a bounded scan.
__device__ __forceinline__ void cell_span(float x, float lo0, float R, float inv_h, int n, int &lo, int &hi)
{
    lo = __float2int_rd((x - lo0 - R) * inv_h);
    hi = __float2int_rd((x - lo0 + R) * inv_h);
    lo = min(max(lo, -2), n + 1);
    hi = min(max(hi, -2), n + 1);
    if (hi - lo + 1 > n) hi = lo + n - 1;
}

// Visit (member position s, particle index) of every member of the cells
// within reach R of xi; Lees-Edwards rows that cross the y boundary are
// shifted by the image offset.  half: skip cells with a lower index than
// xi's own cell.
template <bool HALF, class F>
__device__ __forceinline__ void for_candidates(const md_grid &g, const md_geom &geom, float delta, float4 xi,
                                               float R, const int32_t *__restrict__ members, int32_t r, F fn)
{
    const int own = cell_index32(g, cell_coord(g, 0, xi.x), cell_coord(g, 1, xi.y), cell_coord(g, 2, xi.z));
    int zlo, zhi, ylo, yhi;
    cell_span(xi.z, g.lo[2], R, g.inv_h[2], g.nc[2], zlo, zhi);
    cell_span(xi.y, g.lo[1], R, g.inv_h[1], g.nc[1], ylo, yhi);
    if (geom.walls) {
        ylo = max(ylo, 0);
        yhi = min(yhi, g.nc[1] - 1);
    }
    for (int cz = zlo; cz <= zhi; ++cz) {
        const int wz = wrapc(cz, g.nc[2]);
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
            const int rowc = cell_index32(g, 0, wy, wz);
            if (HALF && rowc + g.nc[0] - 1 < own) continue;   // whole row below own cell
            int xlo, xhi;
            cell_span(xi.x + sx, g.lo[0], R, g.inv_h[0], g.nc[0], xlo, xhi);
            for (int cx = xlo; cx <= xhi; ++cx) {
                const int c = rowc + wrapc(cx, g.nc[0]);
                if (HALF && c < own) continue;
                int32_t b = g.start[c];
                const int32_t e = g.start[c + 1];
                if (HALF && b <= r) b = r + 1;    // own cell: later members only
                for (int32_t s = b; s < e; ++s) fn(s, members ? members[s] : s);
            }
        }
    }
}

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
            if (KIND == MD_LIST_LJ) x0i = a.X0[id_of(xi)];
            const int64_t rows = a.rows;
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
            });
        }
    }
    // every lane of the warp reaches the row bookkeeping (shuffle needs all)
    if (active) a.nc[r] = cnt;
    const int m = __reduce_max_sync(0xffffffffu, active ? cnt : 0);
    if ((threadIdx.x & 31) == 0 && m > 0) {
        atomicMax(&a.ctl[CTL_MAXROW + KIND], m);
        if (m > a.cap) atomicOr(&a.ctl[CTL_OVERFLOW], 1 << KIND);
    }
}

// ---------------------------------------------------------------------------
// Plasma list, one warp per home cell.  The warp stages the positions of the
// home cell and of its neighbour cells with a higher index (the forward half
// of the stencil) in shared memory, then walks its home particles one at a
// time: the 32 lanes test 32 staged candidates at once and the hits are
// compacted into the row with a warp ballot.
// ---------------------------------------------------------------------------
constexpr int BC_WARPS = 4;
constexpr int BC_CAND = 256;
constexpr int BC_HOME = 64;

struct bc_smem {
    float4 cx[BC_WARPS][BC_CAND];
    int32_t cj[BC_WARPS][BC_CAND];
    int32_t cnt[BC_WARPS][BC_HOME];
};

// Distinct periodic neighbours of coordinate c along an edge of n cells.
__device__ __forceinline__ int stencil_axis(int c, int n, bool periodic, int out[3])
{
    if (!periodic) {
        int m = 0;
        for (int d = -1; d <= 1; ++d)
            if (c + d >= 0 && c + d < n) out[m++] = c + d;
        return m;
    }
    if (n >= 3) {
        out[0] = c == 0 ? n - 1 : c - 1;
        out[1] = c;
        out[2] = c == n - 1 ? 0 : c + 1;
        return 3;
    }
    for (int d = 0; d < n; ++d) out[d] = d;
    return n;
}

__global__ void __launch_bounds__(BC_WARPS * 32) k_build_fluid_cells(build_args a, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    __shared__ bc_smem sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const md_grid &g = a.g;
    const int c = blockIdx.x * BC_WARPS + warp;
    if (c >= g.ncell) return;                     // warp-uniform; no block barrier is used
    const int hb = g.start[c], he = g.start[c + 1];
    if (hb == he) return;
    const unsigned lt = (1u << lane) - 1u;
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    const float delta = a.ds->le_offset_f;
    const int64_t rows = a.rows;
    int zs[3], ys[3], xs3[3];
    const int nzs = stencil_axis(cz, nz, true, zs);
    const int nys = stencil_axis(cy, ny, !a.geom.walls, ys);
    const int nxs = stencil_axis(cx, nx, true, xs3);

    for (int h0 = hb; h0 < he; h0 += BC_HOME) {
        const int h1 = min(he, h0 + BC_HOME);
        for (int t = lane; t < h1 - h0; t += 32) sm.cnt[warp][t] = 0;
        __syncwarp();
        int nst = 0;
        auto process = [&]() {
            __syncwarp();
            for (int i = h0; i < h1; ++i) {
                const float4 xi = a.x32[i];
                const int ci = class_of(xi);
                if (ci == CLS_PLT) continue;
                int cnt = sm.cnt[warp][i - h0];
                for (int t0 = 0; t0 < nst; t0 += 32) {
                    const int t = t0 + lane;
                    bool hit = false;
                    int32_t j = 0;
                    if (t < nst) {
                        j = sm.cj[warp][t];
                        const float4 xj = sm.cx[warp][t];
                        const int cj = class_of(xj);
                        if (j > i && cj != CLS_PLT && !(ci == CLS_WALL && cj == CLS_WALL)) {
                            float dx, dy, dz, vs;
                            min_image_f32(a.geom, delta, xi, xj, dx, dy, dz, vs);
                            hit = r2_f32(dx, dy, dz) < a.cut2;
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, hit);
                    if (hit) {
                        const int k = cnt + __popc(m & lt);
                        if (k < a.cap) a.nl[(int64_t)i * a.cap + k] = j;
                    }
                    cnt += __popc(m);
                }
                if (lane == 0) sm.cnt[warp][i - h0] = cnt;
                __syncwarp();
            }
            nst = 0;
        };
        auto stage = [&](int cc) {
            const int cb = g.start[cc], ce = g.start[cc + 1];
            for (int p = cb; p < ce;) {
                const int room = BC_CAND - nst;
                if (room == 0) { process(); continue; }
                const int m = min(ce - p, room);
                __syncwarp();
                for (int t = lane; t < m; t += 32) {
                    sm.cx[warp][nst + t] = a.x32[p + t];
                    sm.cj[warp][nst + t] = p + t;
                }
                nst += m;
                p += m;
            }
        };
        for (int iz = 0; iz < nzs; ++iz) {
            for (int iy = 0; iy < nys; ++iy) {
                const int wy = ys[iy];
                const int rowc = (zs[iz] * ny + wy) * nx;
                const bool crossing = a.geom.le && ((cy == 0 && wy == ny - 1 && ny > 1) ||
                                                    (cy == ny - 1 && wy == 0 && ny > 1));
                if (!crossing) {
                    for (int ix = 0; ix < nxs; ++ix) {
                        const int cc = rowc + xs3[ix];
                        if (cc >= c) stage(cc);
                    }
                } else {
                    // images across the Lees-Edwards boundary sit delta away in x
                    const float sx = (cy == ny - 1) ? -delta : delta;
                    const float x0 = g.lo[0] + cx * g.h[0];
                    int xlo = __float2int_rd((x0 + sx - g.lo[0] - a.R) * g.inv_h[0]);
                    int xhi = __float2int_rd((x0 + g.h[0] + sx - g.lo[0] + a.R) * g.inv_h[0]);
                    if (xhi - xlo + 1 > nx) xhi = xlo + nx - 1;
                    for (int xx = xlo; xx <= xhi; ++xx) {
                        const int cc = rowc + wrapc(xx, nx);
                        if (cc >= c) stage(cc);
                    }
                }
            }
        }
        process();
        for (int t = lane; t < h1 - h0; t += 32) a.nc[h0 + t] = sm.cnt[warp][t];
        int mx = 0;
        for (int t = lane; t < h1 - h0; t += 32) mx = max(mx, sm.cnt[warp][t]);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0 && mx > 0) {
            atomicMax(&a.ctl[CTL_MAXROW + MD_LIST_FLUID], mx);
            if (mx > a.cap) atomicOr(&a.ctl[CTL_OVERFLOW], 1 << MD_LIST_FLUID);
        }
        __syncwarp();
    }
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
    k_build_fluid_cells<<<(unsigned)((a.g.ncell + BC_WARPS - 1) / BC_WARPS), BC_WARPS * 32, 0, s->stream>>>(a, gate);

    if (s->n_plt > 0) {
        // interface: platelet rows (platelet sub-grid order) against the main grid
        a.rows = s->n_plt;
        a.row_idx = s->plt_sorted;
        a.cut2 = s->cut2[MD_LIST_IFACE];
        a.nl = s->nl[MD_LIST_IFACE];
        a.nc = s->nc[MD_LIST_IFACE];
        a.cap = s->cap[MD_LIST_IFACE];
        k_build<MD_LIST_IFACE><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a, gate);

        a.g = s->gplt;
        a.members = s->plt_sorted;
        a.R = (float)(s->cfg.lj_rc + s->cfg.skin) * margin;
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
            a.R = (float)(s->cfg.morse_rc + s->cfg.skin) * margin;
            a.cut2 = s->cut2[MD_LIST_MORSE];
            a.nl = s->nl[MD_LIST_MORSE];
            a.nc = s->nc[MD_LIST_MORSE];
            a.cap = s->cap[MD_LIST_MORSE];
            k_build<MD_LIST_MORSE><<<blocks_for(a.rows), MSM_TPB, 0, s->stream>>>(a, gate);
        }
    }
    MSM_COUNT(s, 1 + (s->n_plt > 0 ? 2 + (s->n_rec > 0 ? 1 : 0) : 0));
    return cudaGetLastError();
}
