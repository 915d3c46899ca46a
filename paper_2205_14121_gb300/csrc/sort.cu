// K1: cell binning, counting sort and reorder of the particle arrays (the
// "neighbor lists construction" step of Table 1), plus the platelet and
// receptor sub-grids used by the longer-ranged lists.
//
// Every kernel here takes a `gate` pointer: when it is non-null and *gate is
// zero the kernel returns at once, so the whole rebuild chain can be enqueued
// every step and only does work when the displacement check tripped.
#include "msm_internal.cuh"

namespace {

constexpr int SCAN_TPB = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_TPB * SCAN_ITEMS;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (blockDim = 1024).
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *total)
{
    __shared__ int32_t wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t incl = warp_incl_scan(v);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int32_t t = warp_incl_scan(wsum[lane]);
        wsum[lane] = t;
    }
    __syncthreads();
    const int32_t excl = incl - v + (w > 0 ? wsum[w - 1] : 0);
    if (total) *total = wsum[31];
    __syncthreads();
    return excl;
}

__global__ void k_scan_local(const int32_t *in, int32_t *out, int64_t count, int32_t *sums,
                             const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t a[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        a[k] = (base + k < count) ? in[base + k] : 0;
        s += a[k];
    }
    int32_t tot;
    int32_t run = block_excl_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < count) out[base + k] = run;
        run += a[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of the block sums by one block; writes the grand total.
__global__ void k_scan_sums(int32_t *sums, int64_t nblocks, int32_t *total_out, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t per = (nblocks + SCAN_TPB - 1) / SCAN_TPB;
    const int64_t b0 = (int64_t)threadIdx.x * per;
    int32_t s = 0;
    for (int64_t k = 0; k < per; ++k)
        if (b0 + k < nblocks) s += sums[b0 + k];
    int32_t tot;
    int32_t run = block_excl_scan(s, &tot);
    for (int64_t k = 0; k < per; ++k) {
        if (b0 + k < nblocks) {
            const int32_t t = sums[b0 + k];
            sums[b0 + k] = run;
            run += t;
        }
    }
    if (threadIdx.x == 0 && total_out) *total_out = tot;
}

__global__ void k_scan_add(int32_t *out, int64_t count, const int32_t *sums, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int32_t add = sums[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += SCAN_TPB) {
        const int64_t i = base + k;
        if (i < count) out[i] += add;
    }
}

__global__ void k_zero_i32(int32_t *p, int64_t count, int32_t *ctl, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) p[i] = 0;
    if (ctl && blockIdx.x == 0 && threadIdx.x < 8) {
        // subset counters and per-build row maxima
        if (threadIdx.x == 0) ctl[CTL_NPLT] = 0;
        if (threadIdx.x == 1) ctl[CTL_NREC] = 0;
        if (threadIdx.x >= 4) ctl[CTL_MAXROW + threadIdx.x - 4] = 0;
    }
}

__global__ void k_bin(const float4 *__restrict__ x32, int64_t n, md_grid g, int32_t *__restrict__ cellid,
                      int32_t *__restrict__ slot, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = x32[i];
    const int64_t c = cell_index(g, cell_coord(g, 0, p.x), cell_coord(g, 1, p.y), cell_coord(g, 2, p.z));
    cellid[i] = (int32_t)c;
    slot[i] = atomicAdd(&g.count[c], 1);
}

__global__ void k_scatter(int64_t n, const int32_t *__restrict__ cellid, const int32_t *__restrict__ slot,
                          const int32_t *__restrict__ start, int32_t *__restrict__ perm, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[start[cellid[i]] + slot[i]] = (int32_t)i;
}

struct gather_args {
    int64_t n;
    const int32_t *perm;
    const double *xs, *ys, *zs;
    const float4 *x32, *v;
    const float4 *f[3];
    const int32_t *tag;
    double *alt64;
    float4 *altx, *altv, *altf[3];
    int32_t *alt_tag;
    int nf;
    unsigned carry;
};

__global__ void k_gather(gather_args a, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const int32_t i = a.perm[k];
    a.alt64[k] = a.xs[i];
    a.alt64[a.n + k] = a.ys[i];
    a.alt64[2 * a.n + k] = a.zs[i];
    a.altx[k] = a.x32[i];
    a.altv[k] = a.v[i];
    a.alt_tag[k] = a.tag[i];
    for (int l = 0; l < a.nf; ++l)
        if (a.carry & (1u << l)) a.altf[l][k] = a.f[l][i];
}

struct copyback_args {
    int64_t n;
    double *xs, *ys, *zs;
    float4 *x32, *v, *xb;
    float4 *f[3];
    int32_t *tag, *pos_of_id;
    const double *alt64;
    const float4 *altx, *altv, *altf[3];
    const int32_t *alt_tag;
    int nf;
    unsigned carry;
};

__global__ void k_copyback(copyback_args a, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    a.xs[k] = a.alt64[k];
    a.ys[k] = a.alt64[a.n + k];
    a.zs[k] = a.alt64[2 * a.n + k];
    const float4 x = a.altx[k];
    a.x32[k] = x;
    a.xb[k] = x;
    a.v[k] = a.altv[k];
    a.tag[k] = a.alt_tag[k];
    for (int l = 0; l < a.nf; ++l)
        if (a.carry & (1u << l)) a.f[l][k] = a.altf[l][k];
    a.pos_of_id[id_of(x)] = (int32_t)k;
}

__global__ void k_remap_bonds(int64_t nb, const int32_t *__restrict__ bond_id, const int32_t *__restrict__ pos_of_id,
                              int32_t *__restrict__ bond_ij, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= 2 * nb) return;
    bond_ij[b] = pos_of_id[bond_id[b]];
}

// ids -> current storage slots for `count` entries (angle ends)
__global__ void k_remap_ids(int64_t count, const int32_t *__restrict__ ids, const int32_t *__restrict__ pos_of_id,
                            int32_t *__restrict__ slots, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    slots[q] = pos_of_id[ids[q]];
}

__global__ void k_compact_subsets(int64_t n, const int32_t *__restrict__ tag, int32_t *plt_idx, int32_t *rec_idx,
                                  int32_t *ctl, int64_t n_plt, int64_t n_rec, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t t = tag[k];
    if (t < 0) return;
    const int32_t p = atomicAdd(&ctl[CTL_NPLT], 1);
    if (p < n_plt) plt_idx[p] = (int32_t)k;
    if (t & MD_RECEPTOR_BIT) {
        const int32_t r = atomicAdd(&ctl[CTL_NREC], 1);
        if (r < n_rec) rec_idx[r] = (int32_t)k;
    }
}

__global__ void k_bin_subset(const int32_t *__restrict__ idx, int64_t m, const float4 *__restrict__ x32, md_grid g,
                             int32_t *__restrict__ cellid, int32_t *__restrict__ slot, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const float4 p = x32[idx[r]];
    const int64_t c = cell_index(g, cell_coord(g, 0, p.x), cell_coord(g, 1, p.y), cell_coord(g, 2, p.z));
    cellid[r] = (int32_t)c;
    slot[r] = atomicAdd(&g.count[c], 1);
}

__global__ void k_scatter_subset(const int32_t *__restrict__ idx, int64_t m, const int32_t *__restrict__ cellid,
                                 const int32_t *__restrict__ slot, const int32_t *__restrict__ start,
                                 int32_t *__restrict__ sorted, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    sorted[start[cellid[r]] + slot[r]] = idx[r];
}

__global__ void k_finish_build(int32_t *ctl, md_dstate *ds, const int32_t *gate)
{
    if (gate_closed(gate)) return;
    ds->n_builds += 1;
    ds->le_build_f = ds->le_offset_f;
    ctl[CTL_REBUILD] = 0;
    ctl[CTL_NFAST] = 0;      // every particle at its build position
}

inline unsigned blocks_for(int64_t n, int tpb = MSM_TPB)
{
    return (unsigned)((n + tpb - 1) / tpb > 0 ? (n + tpb - 1) / tpb : 1);
}

}  // namespace

// Exclusive scan out[k] = sum in[0..k) (count up to 64M; in may equal out),
// grand total -> *total_out.
cudaError_t launch_scan(md_system *s, const int32_t *in, int32_t *out, int64_t count, int32_t *total_out,
                        const int32_t *gate)
{
    const int64_t nblk = (count + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nblk > s->scan_cap) return cudaErrorInvalidValue;
    if (count <= 0) return cudaSuccess;
    k_scan_local<<<(unsigned)nblk, SCAN_TPB, 0, s->stream>>>(in, out, count, s->scan_sums, gate);
    k_scan_sums<<<1, SCAN_TPB, 0, s->stream>>>(s->scan_sums, nblk, total_out, gate);
    k_scan_add<<<(unsigned)nblk, SCAN_TPB, 0, s->stream>>>(out, count, s->scan_sums, gate);
    MSM_COUNT(s, 3);
    return cudaGetLastError();
}

// The whole rebuild chain: bin + sort + reorder + sub-grids + every list.
cudaError_t launch_rebuild(md_system *s, const int32_t *gate, unsigned carry)
{
    const int64_t n = s->n;
    cudaStream_t st = s->stream;
    md_grid &g = s->gmain;
    k_zero_i32<<<blocks_for(g.ncell, 1024) > 4096 ? 4096 : blocks_for(g.ncell, 1024), 1024, 0, st>>>(
        g.count, g.ncell, s->ctl, gate);
    k_bin<<<blocks_for(n), MSM_TPB, 0, st>>>(s->x32, n, g, s->cellid, s->slot, gate);
    cudaError_t e = launch_scan(s, g.count, g.start, g.ncell, g.start + g.ncell, gate);
    if (e != cudaSuccess) return e;
    k_scatter<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->cellid, s->slot, g.start, s->perm, gate);

    const int nf = s->n_plt > 0 ? 3 : 1;
    gather_args ga;
    ga.n = n; ga.perm = s->perm; ga.xs = s->xs; ga.ys = s->ys; ga.zs = s->zs;
    ga.x32 = s->x32; ga.v = s->v; ga.tag = s->tag_s;
    ga.alt64 = s->alt64; ga.altx = s->altx; ga.altv = s->altv; ga.alt_tag = s->alt_tag;
    for (int l = 0; l < 3; ++l) { ga.f[l] = s->f[l]; ga.altf[l] = s->altf[l]; }
    ga.nf = nf;
    ga.carry = carry;
    k_gather<<<blocks_for(n), MSM_TPB, 0, st>>>(ga, gate);
    copyback_args ca;
    ca.n = n; ca.xs = s->xs; ca.ys = s->ys; ca.zs = s->zs; ca.x32 = s->x32; ca.v = s->v; ca.xb = s->xb;
    ca.tag = s->tag_s; ca.pos_of_id = s->pos_of_id;
    ca.alt64 = s->alt64; ca.altx = s->altx; ca.altv = s->altv; ca.alt_tag = s->alt_tag;
    for (int l = 0; l < 3; ++l) { ca.f[l] = s->f[l]; ca.altf[l] = s->altf[l]; }
    ca.nf = nf;
    ca.carry = carry;
    k_copyback<<<blocks_for(n), MSM_TPB, 0, st>>>(ca, gate);
    if (s->nb > 0)
        k_remap_bonds<<<blocks_for(2 * s->nb), MSM_TPB, 0, st>>>(s->nb, s->bond_id, s->pos_of_id, s->bond_ij, gate);
    if (s->na > 0)   // the same id -> slot map for the 3 na angle ends
        k_remap_ids<<<blocks_for(3 * s->na), MSM_TPB, 0, st>>>(3 * s->na, s->angle_id, s->pos_of_id, s->angle_ijk,
                                                              gate);

    if (s->n_plt > 0) {
        k_compact_subsets<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->tag_s, s->plt_idx, s->rec_idx, s->ctl,
                                                            s->n_plt, s->n_rec, gate);
        // platelet sub-grid
        md_grid &gp = s->gplt;
        k_zero_i32<<<blocks_for(gp.ncell, 1024) > 4096 ? 4096 : blocks_for(gp.ncell, 1024), 1024, 0, st>>>(
            gp.count, gp.ncell, nullptr, gate);
        k_bin_subset<<<blocks_for(s->n_plt), MSM_TPB, 0, st>>>(s->plt_idx, s->n_plt, s->x32, gp, s->plt_cell,
                                                              s->plt_slot, gate);
        e = launch_scan(s, gp.count, gp.start, gp.ncell, gp.start + gp.ncell, gate);
        if (e != cudaSuccess) return e;
        k_scatter_subset<<<blocks_for(s->n_plt), MSM_TPB, 0, st>>>(s->plt_idx, s->n_plt, s->plt_cell, s->plt_slot,
                                                                  gp.start, s->plt_sorted, gate);
        if (s->n_rec > 0) {
            md_grid &gr = s->grec;
            k_zero_i32<<<blocks_for(gr.ncell, 1024) > 4096 ? 4096 : blocks_for(gr.ncell, 1024), 1024, 0, st>>>(
                gr.count, gr.ncell, nullptr, gate);
            k_bin_subset<<<blocks_for(s->n_rec), MSM_TPB, 0, st>>>(s->rec_idx, s->n_rec, s->x32, gr, s->rec_cell,
                                                                  s->rec_slot, gate);
            e = launch_scan(s, gr.count, gr.start, gr.ncell, gr.start + gr.ncell, gate);
            if (e != cudaSuccess) return e;
            k_scatter_subset<<<blocks_for(s->n_rec), MSM_TPB, 0, st>>>(s->rec_idx, s->n_rec, s->rec_cell,
                                                                      s->rec_slot, gr.start, s->rec_sorted, gate);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_build_lists(s, gate);
    if (e != cudaSuccess) return e;
    k_finish_build<<<1, 1, 0, st>>>(s->ctl, s->ds, gate);
    // zero, bin, scatter, gather, copyback, finish (+ remap) (+ subset passes)
    MSM_COUNT(s, 6 + (s->nb > 0 ? 1 : 0) + (s->na > 0 ? 1 : 0) + (s->n_plt > 0 ? 4 + (s->n_rec > 0 ? 3 : 0) : 0));
    return cudaGetLastError();
}
