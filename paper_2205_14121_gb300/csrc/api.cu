// The C ABI of libmsm (include/msm.h): system set-up over a caller-owned
// device workspace, state import/export, and the multi-level time loop of
// Table 1 driving the kernels of sort.cu, neighbor.cu, forces.cu,
// integrate.cu and reduce.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <vector>

#include "msm_internal.cuh"

namespace {

const char *g_static_err = "no error";

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct carver {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(int64_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (size_t)(count > 0 ? count : 1);
        return p;
    }
};

bool setup_grid(const md_config &c, double cut, md_grid &g, std::string &err)
{
    const bool walls = c.flags & MD_CFG_WALLS;
    double lo[3] = {0.0, walls ? -c.wall : 0.0, 0.0};
    double hi[3] = {c.box[0], walls ? c.box[1] + c.wall : c.box[1], c.box[2]};
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        const double ext = hi[d] - lo[d];
        // fewer than three cells along a periodic edge is fine: the candidate
        // scan clamps its cell range to the grid, visiting each cell once
        int nc = (int)floor(ext / cut);
        if (nc < 1) nc = 1;
        if (nc > (1 << 20)) {
            err = "grid too fine";
            return false;
        }
        g.nc[d] = nc;
        g.lo[d] = (float)lo[d];
        g.h[d] = (float)(ext / nc);
        g.inv_h[d] = (float)(nc / ext);
        ncell *= nc;
    }
    g.ncell = ncell;
    return true;
}

int default_cap(int v, int d) { return v > 0 ? v : d; }

bool plan(const md_config &c, md_system &s, carver &cv, std::string &err)
{
    // the plasma list packs a partner index into 27 bits
    if (c.n <= 0 || c.n > MSM_STREAM_JMASK + 1) { err = "n out of range (1 .. 2^27)"; return false; }
    if (c.n_plt_particles < 0 || c.n_plt_particles > c.n || c.n_receptors < 0 ||
        c.n_receptors > c.n_plt_particles || c.n_bonds < 0) {
        err = "inconsistent particle counts"; return false;
    }
    if (!(c.dt > 0) || !(c.rc > 0) || !(c.skin >= 0) || !(c.box[0] > 0) || !(c.box[1] > 0) || !(c.box[2] > 0)) {
        err = "dt, rc, skin and box must be positive"; return false;
    }
    if ((c.flags & MD_CFG_WALLS) && (c.flags & MD_CFG_LEES_EDWARDS)) {
        err = "walls and Lees-Edwards images are exclusive"; return false;
    }
    s.cfg = c;
    s.n = c.n;
    s.n_plt = c.n_plt_particles;
    s.n_rec = c.n_receptors;
    s.nb = c.n_bonds;
    // a half row holds up to the full neighbour count (a particle early in the
    // cell order): 27.6 on average at rho = 3 within 1.3, beyond 64 in the
    // far tail of the density fluctuations of a few million particles
    s.cap[MD_LIST_FLUID] = default_cap(c.cap_fluid, 96);
    s.cap[MD_LIST_IFACE] = default_cap(c.cap_iface, 96);
    s.cap[MD_LIST_LJ] = default_cap(c.cap_lj, 1024);   // shells in contact: hundreds of partners
    s.cap[MD_LIST_MORSE] = default_cap(c.cap_morse, 256);
    // list cells at least half the list reach wide: the candidate scan visits
    // contiguous row ranges trimmed to the reach sphere
    if (!setup_grid(c, 0.5 * (c.rc + c.skin), s.gmain, err)) return false;
    if ((c.flags & MD_CFG_LEES_EDWARDS) && s.gmain.nc[1] < 6) {
        err = "Lees-Edwards images need Ly of at least three list reaches (rc + skin)";
        return false;
    }
    const bool plt = s.n_plt > 0;
    if (!(c.skin_plt >= 0)) { err = "skin_plt must not be negative"; return false; }
    s.skin_p = c.skin_plt > 0 ? c.skin_plt : c.skin;
    if (plt) {
        if (!setup_grid(c, 0.5 * (c.lj_rc + s.skin_p), s.gplt, err)) return false;
        if (s.n_rec > 0 && !setup_grid(c, 0.5 * (c.morse_rc + s.skin_p), s.grec, err)) return false;
    }
    const int64_t n = s.n;
    s.xs = cv.take<double>(n);
    s.ys = cv.take<double>(n);
    s.zs = cv.take<double>(n);
    s.x32 = cv.take<float4>(n);
    s.v = cv.take<float4>(n);
    const int nf = plt ? 3 : 1;
    for (int l = 0; l < 3; ++l) {
        s.f[l] = l < nf ? cv.take<float4>(n) : nullptr;
        s.altf[l] = l < nf ? cv.take<float4>(n) : nullptr;
    }
    s.xb = cv.take<float4>(n);
    s.fast_max = n / 64 > 4096 ? n / 64 : 4096;
    s.fast_idx = cv.take<int32_t>(s.fast_max);
    s.fast_flag = cv.take<uint32_t>(n);
    for (int l = 0; l < 3; ++l)
        s.fdet[l] = (l == 0 || c.n_plt_particles > 0) ? cv.take<unsigned long long>(3 * n) : nullptr;
    s.tag_s = cv.take<int32_t>(n);
    s.cellid = cv.take<int32_t>(n);
    s.slot = cv.take<int32_t>(n);
    s.perm = cv.take<int32_t>(n);
    s.pos_of_id = cv.take<int32_t>(n);
    s.alt64 = cv.take<double>(3 * n);
    s.altv = cv.take<float4>(n);
    s.altx = cv.take<float4>(n);
    s.alt_tag = cv.take<int32_t>(n);
    s.tag_id = cv.take<int32_t>(n);
    s.X0 = plt ? cv.take<float4>(n) : nullptr;
    s.gmain.start = cv.take<int32_t>(s.gmain.ncell + 1);
    s.gmain.count = cv.take<int32_t>(s.gmain.ncell);
    int64_t max_cells = s.gmain.ncell;
    if (plt) {
        s.gplt.start = cv.take<int32_t>(s.gplt.ncell + 1);
        s.gplt.count = cv.take<int32_t>(s.gplt.ncell);
        max_cells = s.gplt.ncell > max_cells ? s.gplt.ncell : max_cells;
        s.plt_idx = cv.take<int32_t>(s.n_plt);
        s.plt_sorted = cv.take<int32_t>(s.n_plt);
        s.plt_cell = cv.take<int32_t>(s.n_plt);
        s.plt_slot = cv.take<int32_t>(s.n_plt);
        if (s.n_rec > 0) {
            s.grec.start = cv.take<int32_t>(s.grec.ncell + 1);
            s.grec.count = cv.take<int32_t>(s.grec.ncell);
            max_cells = s.grec.ncell > max_cells ? s.grec.ncell : max_cells;
            s.rec_idx = cv.take<int32_t>(s.n_rec);
            s.rec_sorted = cv.take<int32_t>(s.n_rec);
            s.rec_cell = cv.take<int32_t>(s.n_rec);
            s.rec_slot = cv.take<int32_t>(s.n_rec);
        }
    }
    s.scan_cap = max_cells / 4096 + 2;
    if (s.scan_cap > 1024 * 64) { err = "too many cells for the scan"; return false; }
    s.scan_sums = cv.take<int32_t>(s.scan_cap);
    const int64_t rows[4] = {n, s.n_plt, s.n_plt, s.n_rec};
    for (int k = 0; k < 4; ++k) {
        if (rows[k] > 0 && (k == 0 || plt)) {
            s.nl[k] = cv.take<int32_t>(rows[k] * (int64_t)s.cap[k]);
            s.nc[k] = cv.take<int32_t>(rows[k]);
        } else {
            s.nl[k] = nullptr;
            s.nc[k] = nullptr;
        }
    }
    if (s.nb > 0) {
        s.bond_id = cv.take<int32_t>(2 * s.nb);
        s.bond_ij = cv.take<int32_t>(2 * s.nb);
        s.bond_r0 = cv.take<float>(s.nb);
    }
    if (c.n_angles < 0 || (c.n_angles > 0 && !plt)) { err = "angle triplets need platelet particles"; return false; }
    s.na = c.n_angles;
    if (s.na > 0) {
        s.angle_id = cv.take<int32_t>(3 * s.na);
        s.angle_ijk = cv.take<int32_t>(3 * s.na);
        s.angle_t0 = cv.take<float>(s.na);
    }
    if (plt) {
        const int64_t P = c.n_platelets > 0 ? c.n_platelets : 1;
        s.plt_off = cv.take<int32_t>(P + 1);
        s.plt_ids = cv.take<int32_t>(s.n_plt);
        s.bond_off = cv.take<int32_t>(P + 1);
        if (s.nb > 0) s.bond_blk = cv.take<int2>((s.nb + MSM_TPB - 1) / MSM_TPB);
        if (s.na > 0) s.angle_blk = cv.take<int2>((s.na + MSM_TPB - 1) / MSM_TPB);
        s.plt_cmask = cv.take<unsigned long long>(P);
        s.plt_stride = cv.take<int32_t>(P);
        s.plt_row_stride = cv.take<int32_t>(s.n_plt);
        s.plt_contacts = cv.take<int32_t>(P);
        s.feat = cv.take<double>(12 * P);
        s.ring = cv.take<float>(P * (int64_t)s.ring_T * 12);
        s.plt_k = cv.take<int32_t>(P);
        s.plt_bound = cv.take<float4>(P);
        s.feat_sums = cv.take<double>(25 * P + (P + 1) / 2);
        s.plt_near = cv.take<int32_t>(P);
        s.cell_pid = cv.take<int2>(s.gplt.ncell > s.grec.ncell ? s.gplt.ncell : s.grec.ncell);
    }
    s.red_blocks = (int)((n + MSM_TPB - 1) / MSM_TPB);
    if (s.red_blocks > RED_BLOCKS_MAX) s.red_blocks = RED_BLOCKS_MAX;
    s.red_part = cv.take<double>((int64_t)s.red_blocks * RED_WORDS);
    s.red_out = cv.take<double>(RED_WORDS);
    s.prof_part = cv.take<double>((int64_t)(PROF_BLOCKS + 1) * 2 * PROF_BINS_MAX);
    s.vir_acc = cv.take<double>(9);
    s.ctl = cv.take<int32_t>(CTL_WORDS);
    s.ds = cv.take<md_dstate>(1);
    return true;
}

unsigned blocks_for(int64_t n) { return (unsigned)(n > 0 ? (n + MSM_TPB - 1) / MSM_TPB : 1); }

// ---------------------------------------------------------------------------
// import / export kernels (id order <-> sorted storage)
// ---------------------------------------------------------------------------
__global__ void k_import_x(int64_t n, const double *__restrict__ aos, double *xs, double *ys, double *zs,
                           float4 *x32, float4 *xb)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double x = aos[3 * k], y = aos[3 * k + 1], z = aos[3 * k + 2];
    xs[k] = x; ys[k] = y; zs[k] = z;
    const float4 p = make_float4((float)x, (float)y, (float)z, __int_as_float((int)k));
    x32[k] = p;
    xb[k] = p;
}

__global__ void k_import_v(int64_t n, const double *__restrict__ aos, const int32_t *__restrict__ tag, float4 *v,
                           int32_t *tag_s, int32_t *pos_of_id, float4 *x32, float4 *xb)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float w = __int_as_float((int)pack_w((uint32_t)k, tag[k]));
    x32[k].w = w;
    xb[k].w = w;
    v[k] = make_float4((float)aos[3 * k], (float)aos[3 * k + 1], (float)aos[3 * k + 2], __int_as_float(tag[k]));
    tag_s[k] = tag[k];
    pos_of_id[k] = (int32_t)k;
}

// Clear the rows idx[0..n) of a float4 buffer.
__global__ void k_zero_rows(const int32_t *__restrict__ idx, int64_t n, float4 *buf)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) buf[idx[r]] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_import_f4(int64_t n, const double *__restrict__ aos, float4 *out, float w)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[k] = make_float4((float)aos[3 * k], (float)aos[3 * k + 1], (float)aos[3 * k + 2], w);
}

__global__ void k_import_forces(int64_t n, const float *__restrict__ aos, float4 *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[k] = make_float4(aos[3 * k], aos[3 * k + 1], aos[3 * k + 2], 0.0f);
}

__global__ void k_export_x(int64_t n, const double *xs, const double *ys, const double *zs, const float4 *x32,
                           double *aos)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t id = id_of(x32[k]);
    aos[3 * id] = xs[k]; aos[3 * id + 1] = ys[k]; aos[3 * id + 2] = zs[k];
}

__global__ void k_export_f4(int64_t n, const float4 *src, const float4 *x32, double *aos)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t id = id_of(x32[k]);
    const float4 p = src[k];
    aos[3 * id] = p.x; aos[3 * id + 1] = p.y; aos[3 * id + 2] = p.z;
}

__global__ void k_export_x32(int64_t n, const float4 *x32, float *aos)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 p = x32[k];
    const int64_t id = id_of(p);
    aos[3 * id] = p.x; aos[3 * id + 1] = p.y; aos[3 * id + 2] = p.z;
}

__global__ void k_export_forces(int64_t n, const float4 *f0, const float4 *f1, const float4 *f2, const float4 *x32,
                                const int32_t *tag, float g, double *aos)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t id = id_of(x32[k]);
    double fx = 0, fy = 0, fz = 0;
    if (f0) { const float4 p = f0[k]; fx += p.x; fy += p.y; fz += p.z; if (tag[k] != MD_TAG_WALL) fx += g; }
    if (f1) { const float4 p = f1[k]; fx += p.x; fy += p.y; fz += p.z; }
    if (f2) { const float4 p = f2[k]; fx += p.x; fy += p.y; fz += p.z; }
    aos[3 * id] = fx; aos[3 * id + 1] = fy; aos[3 * id + 2] = fz;
}

// Forces of a deterministic md_forces, exactly: the levels' fixed-point sums
// added as integers, then scaled by 2^-32 (exact in FP64 below 2^21).
__global__ void k_export_fixed(int64_t n, const unsigned long long *q0, const unsigned long long *q1,
                               const unsigned long long *q2, const float4 *x32, const int32_t *tag, float g,
                               double *aos)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t id = id_of(x32[k]);
    const double u = 1.0 / 4294967296.0;
    for (int d = 0; d < 3; ++d) {
        unsigned long long t = 0;
        if (q0) t += q0[3 * k + d];
        if (q1) t += q1[3 * k + d];
        if (q2) t += q2[3 * k + d];
        double v = (double)(long long)t * u;
        if (d == 0 && q0 && tag[k] != MD_TAG_WALL) v += g;
        aos[3 * id + d] = v;
    }
}

__global__ void k_set_word(int32_t *p, int32_t v) { *p = v; }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
int check(md_system *s, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return MD_OK;
    return cuda_fail(s, e, where);
}

#define CK(expr, where)                                   \
    do {                                                  \
        int _rc = check(s, (expr), where);                \
        if (_rc != MD_OK) return _rc;                     \
    } while (0)

int sync_ctl(md_system *s)
{
    CK(cudaMemcpyAsync(s->h_ctl, s->ctl, sizeof(int32_t) * CTL_WORDS, cudaMemcpyDeviceToHost, s->stream), "ctl copy");
    CK(cudaMemcpyAsync(s->h_ds, s->ds, sizeof(md_dstate), cudaMemcpyDeviceToHost, s->stream), "dstate copy");
    CK(cudaStreamSynchronize(s->stream), "stream sync");
    return MD_OK;
}

int check_flags(md_system *s)
{
    int rc = sync_ctl(s);
    if (rc) return rc;
    if (s->h_ctl[CTL_OVERFLOW]) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "neighbour list overflow (kind mask 0x%x; longest rows %d/%d/%d/%d, capacities %d/%d/%d/%d)",
                 s->h_ctl[CTL_OVERFLOW], s->h_ctl[CTL_MAXROW], s->h_ctl[CTL_MAXROW + 1], s->h_ctl[CTL_MAXROW + 2],
                 s->h_ctl[CTL_MAXROW + 3], s->cap[0], s->cap[1], s->cap[2], s->cap[3]);
        return set_error(s, MD_ENBR_OVERFLOW, buf);
    }
    if (s->h_ctl[CTL_UNSTABLE]) return set_error(s, MD_EUNSTABLE, "NaN/Inf state or a particle escaped the walls");
    return MD_OK;
}

double host_le_offset(const md_system *s, double t)
{
    if (!s->geom.le) return 0.0;
    double d = fmod(s->cfg.shear_rate * s->cfg.box[1] * t, s->cfg.box[0]);
    if (d < 0.0) d += s->cfg.box[0];
    return d;
}

int request_rebuild(md_system *s)
{
    s->det_levels = 0;   // the re-sort moves the particles: no exact forces to export
    k_set_word<<<1, 1, 0, s->stream>>>(s->ctl + CTL_REBUILD, 1);
    CK(cudaGetLastError(), "rebuild request");
    CK(launch_rebuild(s, s->ctl + CTL_REBUILD), "rebuild");
    s->lists_stale = false;
    return MD_OK;
}

int ensure_lists(md_system *s)
{
    if (!s->lists_stale) return MD_OK;
    return request_rebuild(s);
}

int eval_forces(md_system *s, unsigned levels, bool virial, bool det = false)
{
    CK(launch_zero_forces(s, levels), "zero forces");
    if (virial) CK(cudaMemsetAsync(s->vir_acc, 0, 9 * sizeof(double), s->stream), "virial reset");
    float4 *out[3] = {s->f[0], s->f[1], s->f[2]};
    s->det_levels = 0;
    if (!det) {
        CK(launch_forces(s, levels, out, virial), "forces");
        return MD_OK;
    }
    // one level at a time into its fixed-point sums, then its FP32 buffer
    for (int l = 0; l < 3; ++l) {
        const unsigned bit = 1u << l;
        if (!(levels & bit) || !s->fdet[l]) continue;
        CK(cudaMemsetAsync(s->fdet[l], 0, sizeof(unsigned long long) * 3 * s->n, s->stream), "zero fixed sums");
        CK(launch_forces(s, bit, out, virial, true, s->fdet[l]), "forces (deterministic)");
        CK(launch_fixed_to_f4(s, s->fdet[l], s->f[l]), "fixed to float");
    }
    s->det_levels = levels;
    return MD_OK;
}

// Lists first, always: forces restored from a checkpoint are current while
// the lists of the new particle order are not.
int ensure_forces(md_system *s)
{
    const unsigned all = s->n_plt > 0 ? MD_LEVEL_ALL : MD_LEVEL_FLUID;
    int rc = ensure_lists(s);
    if (rc) return rc;
    if (!s->forces_stale && (s->forces_levels & all) == all) return MD_OK;
    rc = eval_forces(s, all, false, s->det_step);
    if (rc) return rc;
    s->forces_stale = false;
    s->forces_levels = all;
    return MD_OK;
}

// Context of a graph capture of the outer step (null: direct launches).
struct capture_ctx {
    cudaGraphConditionalHandle loop;
    std::vector<cudaGraph_t> if_bodies;
    std::vector<unsigned> if_carry;
};

// The rebuild chain: gated kernels when launched directly; under capture, a
// kernel that copies the rebuild flag into a conditional handle and an IF
// node whose body (captured later) is the ungated chain.
int enqueue_rebuild(md_system *s, capture_ctx *cap, unsigned carry)
{
    if (!cap) {
        prof_begin(s, MD_PROF_BUILD);
        CK(launch_rebuild(s, s->ctl + CTL_REBUILD, carry), "rebuild");
        prof_end(s);
        return MD_OK;
    }
    cudaStreamCaptureStatus st;
    cudaGraph_t capg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(s->stream, &st, nullptr, &capg, &deps, nullptr, &ndeps), "capture info");
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, capg, 0, cudaGraphCondAssignDefault), "conditional handle");
    CK(launch_cond_rebuild(s, h), "rebuild condition");
    CK(cudaStreamGetCaptureInfo(s->stream, &st, nullptr, &capg, &deps, nullptr, &ndeps), "capture info");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, capg, deps, nullptr, ndeps, &p), "IF node");
    cap->if_bodies.push_back(p.conditional.phGraph_out[0]);
    cap->if_carry.push_back(carry);
    CK(cudaStreamUpdateCaptureDependencies(s->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
       "capture dependencies");
    return MD_OK;
}

int enqueue_forces(md_system *s, unsigned levels)
{
    float4 *out[3] = {s->f[0], s->f[1], s->f[2]};
    static const int cls[3] = {MD_PROF_FLUID, MD_PROF_IFACE, MD_PROF_PLT};
    for (int l = 0; l < 3; ++l) {
        const unsigned bit = 1u << l;
        if (!(levels & bit) || (l > 0 && s->n_plt == 0)) continue;
        if (s->det_step) {
            // MD_SCHED_DETERMINISTIC: the level's fixed-point sums (pair and
            // bond terms with the lower id first), then its FP32 buffer
            CK(cudaMemsetAsync(s->fdet[l], 0, sizeof(unsigned long long) * 3 * s->n, s->stream), "zero fixed sums");
            prof_begin(s, cls[l]);
            CK(launch_forces(s, bit, out, false, false, s->fdet[l]), "forces (deterministic)");
            prof_end(s);
            if (l < 2) {
                prof_begin(s, MD_PROF_OTHER);
                CK(launch_fast_pairs(s, bit, out, false, s->fdet[l]), "fast pairs (deterministic)");
                prof_end(s);
            }
            CK(launch_fixed_to_f4(s, s->fdet[l], s->f[l]), "fixed to float");
            continue;
        }
        prof_begin(s, cls[l]);
        CK(launch_forces(s, bit, out, false, false), "forces");
        prof_end(s);
        if (l < 2) {   // the fast-particle pass of a DPD level, timed apart
            prof_begin(s, MD_PROF_OTHER);
            CK(launch_fast_pairs(s, bit, out, false), "fast pairs");
            prof_end(s);
        }
    }
    return MD_OK;
}

int enqueue_kd(md_system *s, const float h[3], int kick_which, double dt, int drift_which, unsigned zero,
               bool plt_rows, int stride_q = -1)
{
    prof_begin(s, MD_PROF_INTEG);
    CK(launch_kick_drift(s, h, kick_which, dt, drift_which, zero, plt_rows, stride_q), "kick-drift");
    prof_end(s);
    return MD_OK;
}

int enqueue_time(md_system *s, int dn, int c, double t_off)
{
    prof_begin(s, MD_PROF_OTHER);
    CK(launch_time_rel(s, dn, c, t_off), "time");
    prof_end(s);
    return MD_OK;
}

#define RC(expr)                    \
    do {                            \
        int _rc = (expr);           \
        if (_rc != MD_OK) return _rc; \
    } while (0)

// One outer step of Table 1 (read symmetrically).  STS: velocity-Verlet with
// every force at dt_f; the kick fuses the previous step's closing half-kick
// unless `first`.  RESPA: k_m interface substeps of k_p platelet substeps;
// plasma feels no inner force, so it drifts once per interface substep while
// platelets drift every platelet substep.  Step-dependent values come from
// the device time state, so the same sequence can be captured once and
// replayed.
// Per-platelet measurements of the state at the end of the step appended to
// the feature ring (inside the step, so a replayed graph records every step).
// In AI-MTS the platelet buffer holds impulses: the platelet-level forces
// are evaluated afresh into a sort buffer (free between rebuilds).
int enqueue_record(md_system *s, int mode)
{
    prof_begin(s, MD_PROF_OTHER);
    const float4 *fp = nullptr;
    if (mode == MD_MODE_AI) {
        k_zero_rows<<<blocks_for(s->n_plt), MSM_TPB, 0, s->stream>>>(s->plt_sorted, s->n_plt, s->altf[2]);
        CK(cudaGetLastError(), "zero scratch forces");
        MSM_COUNT(s, 1);
        float4 *out[3] = {nullptr, nullptr, s->altf[2]};
        CK(launch_forces(s, MD_LEVEL_PLT, out, false), "record forces");
        fp = s->altf[2];
    }
    // the stored velocities still miss the closing half kick(s) that the
    // next step's opening kick applies: the fluid level, and in STS all levels
    const float h = (float)(0.5 * s->cfg.dt);
    const float hk[3] = {h, mode == MD_MODE_STS ? h : 0.f, mode == MD_MODE_STS ? h : 0.f};
    CK(launch_features(s, s->feat, fp, hk), "features");
    CK(launch_feature_ring(s, s->feat), "feature ring");
    prof_end(s);
    return MD_OK;
}

int enqueue_outer_step(md_system *s, int mode, int k_m, int k_p, bool first, capture_ctx *cap, bool record)
{
    const md_config &c = s->cfg;
    const bool plt = s->n_plt > 0;
    prof_begin(s, MD_PROF_OTHER);
    CK(launch_outer_begin(s, cap ? cap->loop : 0, cap != nullptr), "outer begin");
    prof_end(s);
    if (mode == MD_MODE_STS) {
        const float hk = (float)(first ? 0.5 * c.dt : c.dt);
        const float h[3] = {hk, plt ? hk : 0.f, plt ? hk : 0.f};
        RC(enqueue_time(s, 1, 0, c.dt));
        RC(enqueue_kd(s, h, DRIFT_ALL, c.dt, DRIFT_ALL, plt ? MD_LEVEL_ALL : MD_LEVEL_FLUID, false));
        RC(enqueue_rebuild(s, cap, 0u));   // every level was cleared by the kick-drift
        RC(enqueue_forces(s, plt ? MD_LEVEL_ALL : MD_LEVEL_FLUID));
        if (record) RC(enqueue_record(s, mode));
        return MD_OK;
    }
    const double dtf = c.dt, dtm = dtf / k_m, dtp = dtm / k_p;
    for (int ci = 0; ci < k_m; ++ci) {
        const bool last_c = ci + 1 == k_m;
        const int dn = last_c ? 1 : 0;
        const int c_end = last_c ? 0 : ci + 1;
        const double tc = ci * dtm;
        RC(enqueue_time(s, dn, c_end, tc + dtm));
        // A: fluid kick (first substep; fused with the previous outer step's
        //    closing half-kick) + opening interface half-kick (after the first
        //    substep fused with the previous substep's closing one: no force
        //    is evaluated between them); plasma drift
        float h[3] = {0.f, 0.f, 0.f};
        if (ci == 0) h[0] = (float)(first ? 0.5 * dtf : dtf);
        h[1] = plt ? (float)(ci == 0 ? 0.5 * dtm : dtm) : 0.f;
        const unsigned zero = (plt ? MD_LEVEL_IFACE : 0u) | (ci == 0 ? MD_LEVEL_FLUID : 0u);
        RC(enqueue_kd(s, h, DRIFT_ALL, dtm, plt ? DRIFT_FLUID : DRIFT_ALL, zero, false));
        if (plt && mode == MD_MODE_AI) {
            // B (AI-MTS): every platelet particle drifts on the fine grid of
            //    K = lcm(k) substeps of dt_m / K; the platelet buffer holds
            //    impulses, so substep q kicks by 1/2 (q = 0) or 1 (fused
            //    closing + opening) of the terms due at its start, and the
            //    terms due at its end are evaluated after the drift.
            const int K = s->plt_K;
            const double dts = dtm / K;
            for (int q = 0; q < K; ++q) {
                RC(enqueue_time(s, dn, c_end, tc + (q + 1) * dts));
                const float hq[3] = {0.f, 0.f, q == 0 ? 0.5f : 1.0f};
                RC(enqueue_kd(s, hq, DRIFT_PLT, dts, DRIFT_PLT, MD_LEVEL_PLT, true, q));
                s->due_on = true;
                s->due_q = q + 1;
                s->due_dtm = dtm;
                const int rc = enqueue_forces(s, MD_LEVEL_PLT);
                s->due_on = false;
                if (rc != MD_OK) return rc;
            }
            const float hc[3] = {0.f, 0.f, 0.5f};
            RC(enqueue_kd(s, hc, DRIFT_PLT, 0.0, -1, 0u, true));
        } else if (plt) {
            // B: platelet substeps; the kick of substep q fuses the closing
            //    half-kick of q-1 with its own opening half-kick
            for (int q = 0; q < k_p; ++q) {
                RC(enqueue_time(s, dn, c_end, tc + (q + 1) * dtp));
                const float hq[3] = {0.f, 0.f, (float)(q == 0 ? 0.5 * dtp : dtp)};
                RC(enqueue_kd(s, hq, DRIFT_PLT, dtp, DRIFT_PLT, MD_LEVEL_PLT, true));
                RC(enqueue_forces(s, MD_LEVEL_PLT));
            }
            const float hc[3] = {0.f, 0.f, (float)(0.5 * dtp)};
            RC(enqueue_kd(s, hc, DRIFT_PLT, 0.0, -1, 0u, true));
        }
        // the fluid level is cleared at the first substep and the interface
        // level at every one: only the platelet level holds values here
        RC(enqueue_rebuild(s, cap, plt ? MD_LEVEL_PLT : 0u));
        if (plt) {
            RC(enqueue_forces(s, MD_LEVEL_IFACE));
            // the closing interface half-kick; before the next interface
            // substep it is fused into that substep's opening kick, before the
            // fluid forces (velocity dependent: Eq. 1's dissipative term) it
            // is not
            if (last_c) {
                const float hm[3] = {0.f, (float)(0.5 * dtm), 0.f};
                RC(enqueue_kd(s, hm, DRIFT_ALL, 0.0, -1, 0u, false));
            }
        }
    }
    RC(enqueue_forces(s, MD_LEVEL_FLUID));
    if (record) RC(enqueue_record(s, mode));
    return MD_OK;
}

int closing_kick(md_system *s, float hf, float hm, float hp)
{
    const float h[3] = {hf, s->n_plt > 0 ? hm : 0.f, s->n_plt > 0 ? hp : 0.f};
    RC(enqueue_kd(s, h, DRIFT_ALL, 0.0, -1, 0u, false));
    return MD_OK;
}

void drop_graph(md_system *s)
{
    if (s->step_exec) cudaGraphExecDestroy(s->step_exec);
    if (s->step_graph) cudaGraphDestroy(s->step_graph);
    s->step_exec = nullptr;
    s->step_graph = nullptr;
    for (int k = 0; k < 4; ++k) s->graph_key[k] = -1;
}

// Capture WHILE(steps_left) { outer step } once per schedule shape.
int build_step_graph(md_system *s, int mode, int k_m, int k_p, bool record)
{
    const int key[4] = {mode | (record ? 256 : 0) | (s->det_step ? 512 : 0), k_m, k_p, (int)s->cfg_k_m};
    bool same = s->step_exec != nullptr;
    for (int k = 0; k < 4; ++k) same = same && s->graph_key[k] == key[k];
    if (same) return MD_OK;
    drop_graph(s);
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0), "graph create");
    capture_ctx cap;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cap.loop, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = cap.loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(s, e, "WHILE node");
    }
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    cudaStream_t saved = s->stream;
    const bool prof = s->prof_on;
    s->prof_on = false;
    s->stream = cs;
    const int64_t l0 = s->nlaunch;
    int rc = MD_OK;
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = enqueue_outer_step(s, mode, k_m, k_p, false, &cap, record);
        cudaGraph_t out = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &out);
        if (rc == MD_OK && e2 != cudaSuccess) rc = cuda_fail(s, e2, "end capture");
    } else {
        rc = cuda_fail(s, e, "begin capture");
    }
    const int64_t l1 = s->nlaunch;
    for (size_t k = 0; rc == MD_OK && k < cap.if_bodies.size(); ++k) {
        e = cudaStreamBeginCaptureToGraph(cs, cap.if_bodies[k], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { rc = cuda_fail(s, e, "begin capture (rebuild)"); break; }
        cudaError_t e1 = launch_rebuild(s, nullptr, cap.if_carry[k]);
        cudaGraph_t out = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &out);
        if (e1 != cudaSuccess) rc = cuda_fail(s, e1, "rebuild capture");
        else if (e2 != cudaSuccess) rc = cuda_fail(s, e2, "end capture (rebuild)");
    }
    const int64_t l2 = s->nlaunch;
    s->stream = saved;
    s->prof_on = prof;
    s->nlaunch = l0;
    cudaStreamDestroy(cs);
    if (rc == MD_OK) {
        e = cudaGraphInstantiate(&s->step_exec, g, 0);
        if (e != cudaSuccess) rc = cuda_fail(s, e, "graph instantiate");
    }
    if (rc != MD_OK) {
        cudaGraphDestroy(g);
        s->step_exec = nullptr;
        cudaGetLastError();
        return rc;
    }
    s->step_graph = g;
    for (int k = 0; k < 4; ++k) s->graph_key[k] = key[k];
    s->graph_body_launches = l1 - l0;
    s->graph_chain_launches = cap.if_bodies.empty() ? 0 : (l2 - l1) / (int64_t)cap.if_bodies.size();
    return MD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// shared error helpers
// ---------------------------------------------------------------------------
int set_error(md_system *s, int code, const char *msg)
{
    if (s) s->err = msg;
    return code;
}

int cuda_fail(md_system *s, cudaError_t e, const char *where)
{
    char buf[256];
    snprintf(buf, sizeof buf, "CUDA error in %s: %s", where, cudaGetErrorString(e));
    return set_error(s, MD_ECUDA, buf);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int md_config_defaults(md_config *c)
{
    if (!c) return MD_EINVAL;
    const int64_t n = c->n;
    const double bx = c->box[0], by = c->box[1], bz = c->box[2];
    memset(c, 0, sizeof *c);
    c->n = n;
    c->box[0] = bx; c->box[1] = by; c->box[2] = bz;
    c->wall = 1.0;
    c->dt = 0.01;
    c->skin = 0.3;
    c->skin_plt = 0.0;   // the plasma skin
    c->rc = 1.0; c->a_ff = 25.0; c->a_fw = 25.0; c->a_fp = 50.0; c->gamma = 4.5; c->sigma = 3.0;
    c->lj_eps = 1.0; c->lj_sigma = 0.8; c->lj_rc = 2.0; c->lj_excl = 1e30;   // no LJ within one platelet
    c->morse_D = 2.0; c->morse_alpha = 2.0; c->morse_r0 = 1.0; c->morse_rc = 5.0; c->f_A = 0.0;
    c->k_bond = 100.0;
    c->k_angle = 5.0;
    c->seed = 20220528ull;
    return MD_OK;
}

int md_workspace_size(const md_config *cfg, size_t *bytes)
{
    if (!cfg || !bytes) return MD_EINVAL;
    md_system tmp;
    carver cv{nullptr};
    std::string err;
    if (!plan(*cfg, tmp, cv, err)) return MD_EINVAL;
    *bytes = cv.off + 256;
    return MD_OK;
}

int md_init(const md_config *cfg, const md_buffers *bufs, void *cuda_stream, md_system **out)
{
    if (!cfg || !bufs || !out) return MD_EINVAL;
    *out = nullptr;
    md_system *s = new (std::nothrow) md_system();
    if (!s) return MD_ENOMEM;
    carver probe{nullptr};
    std::string err;
    if (!plan(*cfg, *s, probe, err)) {
        g_static_err = "md_init: invalid configuration";
        delete s;
        return MD_EINVAL;
    }
    if (!bufs->workspace || bufs->workspace_bytes < probe.off + 256) {
        g_static_err = "md_init: workspace smaller than md_workspace_size()";
        delete s;
        return MD_ENOMEM;
    }
    char *base = (char *)(((uintptr_t)bufs->workspace + 255) & ~(uintptr_t)255);
    carver cv{base};
    plan(*cfg, *s, cv, err);
    s->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&s->device);
    const md_config &c = s->cfg;
    s->geom.walls = (c.flags & MD_CFG_WALLS) ? 1 : 0;
    s->geom.le = (c.flags & MD_CFG_LEES_EDWARDS) ? 1 : 0;
    for (int d = 0; d < 3; ++d) {
        s->geom.L[d] = (float)c.box[d];
        s->geom.hL[d] = 0.5f * s->geom.L[d];
    }
    s->geom.shear_v = (float)(c.shear_rate * c.box[1]);
    // a plasma-platelet pair: plasma within skin/2, the platelet particle
    // within skin_plt/2 of their build positions
    const double cuts[4] = {c.rc + c.skin, c.rc + 0.5 * (c.skin + s->skin_p), c.lj_rc + s->skin_p,
                            c.morse_rc + s->skin_p};
    for (int k = 0; k < 4; ++k) s->cut2[k] = (float)(cuts[k] * cuts[k]);
    s->excl2 = (float)(c.lj_excl * c.lj_excl);
    cudaError_t e = cudaHostAlloc((void **)&s->h_ctl, sizeof(int32_t) * CTL_WORDS, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_ds, sizeof(md_dstate), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        g_static_err = "md_init: pinned host allocation failed";
        if (s->h_ctl) cudaFreeHost(s->h_ctl);
        delete s;
        return MD_ECUDA;
    }
    e = cudaMemsetAsync(s->ctl, 0, sizeof(int32_t) * CTL_WORDS, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ds, 0, sizeof(md_dstate), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->vir_acc, 0, 9 * sizeof(double), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        g_static_err = "md_init: device initialisation failed";
        cudaFreeHost(s->h_ctl);
        cudaFreeHost(s->h_ds);
        delete s;
        return MD_ECUDA;
    }
    *out = s;
    return MD_OK;
}

void md_destroy(md_system *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    drop_graph(s);
    for (auto &r : s->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    if (s->h_ctl) cudaFreeHost(s->h_ctl);
    if (s->h_ds) cudaFreeHost(s->h_ds);
    delete s;
}

const char *md_last_error(const md_system *s)
{
    if (!s) return g_static_err;
    return s->err.empty() ? "no error" : s->err.c_str();
}

static int load_xv(md_system *s, const double *x, const double *v, int64_t step0);

int md_set_particles(md_system *s, const double *x, const double *v, const int32_t *tag, const double *X0,
                     int64_t step0)
{
    if (!s || !x || !v || !tag) return set_error(s, MD_EINVAL, "md_set_particles: null argument");
    const int64_t n = s->n;
    // the same particle set as before (a new state of it): the tags were
    // validated and the platelet member lists built then
    const bool same = s->have_particles && s->h_tag.size() == (size_t)n &&
                      memcmp(s->h_tag.data(), tag, sizeof(int32_t) * (size_t)n) == 0;
    // host-side validation of the tag counts
    int64_t np = 0, nr = 0, npl = 0;
    for (int64_t k = 0; k < (same ? 0 : n); ++k) {
        const int32_t t = tag[k];
        if (t < MD_TAG_WALL) return set_error(s, MD_EINVAL, "md_set_particles: invalid tag");
        if (t >= 0) {
            ++np;
            if (t & MD_RECEPTOR_BIT) ++nr;
            const int64_t p = t & ~MD_RECEPTOR_BIT;
            if (p + 1 > npl) npl = p + 1;
        }
        if (t == MD_TAG_WALL && !s->geom.walls) return set_error(s, MD_EINVAL, "wall particles without walls");
    }
    if (!same && (np != s->n_plt || nr != s->n_rec))
        return set_error(s, MD_EINVAL, "md_set_particles: platelet/receptor counts differ from the configuration");
    if (!same && npl > (s->n_plt > 0 ? s->cfg.n_platelets : 0))
        return set_error(s, MD_EINVAL, "md_set_particles: platelet id beyond cfg.n_platelets");
    cudaStream_t st = s->stream;
    if (!same) s->h_tag.assign(tag, tag + n);
    if (s->n_plt > 0 && !same) {
        // member lists per platelet (ids ascending)
        const int P = s->cfg.n_platelets;
        std::vector<int32_t> off((size_t)P + 1, 0), ids((size_t)s->n_plt);
        for (int64_t k = 0; k < n; ++k)
            if (tag[k] >= 0) off[(size_t)(tag[k] & ~MD_RECEPTOR_BIT) + 1]++;
        for (int p = 0; p < P; ++p) off[(size_t)p + 1] += off[(size_t)p];
        std::vector<int32_t> fill(off.begin(), off.end() - 1);
        for (int64_t k = 0; k < n; ++k)
            if (tag[k] >= 0) ids[(size_t)fill[(size_t)(tag[k] & ~MD_RECEPTOR_BIT)]++] = (int32_t)k;
        for (int p = 0; p < P; ++p)
            if (off[(size_t)p + 1] == off[(size_t)p])
                return set_error(s, MD_EINVAL, "md_set_particles: a platelet id has no particles");
        CK(cudaMemcpyAsync(s->plt_off, off.data(), sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice, st), "plt off");
        CK(cudaMemcpyAsync(s->plt_ids, ids.data(), sizeof(int32_t) * s->n_plt, cudaMemcpyHostToDevice, st), "ids");
        CK(cudaStreamSynchronize(st), "sync");
        if (s->nb == 0) {
            std::vector<int32_t> z((size_t)P + 1, 0);
            CK(cudaMemcpyAsync(s->bond_off, z.data(), sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice, st), "bo");
            CK(cudaStreamSynchronize(st), "sync");
        }
    }
    if (!same) CK(cudaMemcpyAsync(s->tag_id, tag, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st), "upload tag");
    if (s->X0) {
        CK(cudaMemcpyAsync(s->alt64, X0 ? X0 : x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st), "upload X0");
        k_import_f4<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->alt64, s->X0, 0.0f);
        CK(cudaGetLastError(), "import X0");
    }
    s->have_particles = true;
    return load_xv(s, x, v, step0);
}

// Upload of positions and velocities (id order) with the tags kept on the
// device; storage back in id order, time index step0, lists and forces stale.
static int load_xv(md_system *s, const double *x, const double *v, int64_t step0)
{
    const int64_t n = s->n;
    s->det_levels = 0;
    cudaStream_t st = s->stream;
    CK(cudaMemcpyAsync(s->alt64, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st), "upload x");
    k_import_x<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->alt64, s->xs, s->ys, s->zs, s->x32, s->xb);
    CK(cudaGetLastError(), "import x");
    CK(cudaMemcpyAsync(s->alt64, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st), "upload v");
    k_import_v<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->alt64, s->tag_id, s->v, s->tag_s, s->pos_of_id, s->x32,
                                                   s->xb);
    CK(cudaGetLastError(), "import v");
    for (int l = 0; l < 3; ++l)
        if (s->f[l]) CK(cudaMemsetAsync(s->f[l], 0, sizeof(float4) * n, st), "zero f");
    CK(cudaMemsetAsync(s->fast_flag, 0, sizeof(uint32_t) * n, st), "zero fast flags");
    md_dstate *h = s->h_ds;
    memset(h, 0, sizeof *h);
    h->step = step0;
    h->base = step0;
    h->done = step0;
    h->time = (double)step0 * s->cfg.dt;
    h->le_offset = host_le_offset(s, h->time);
    h->le_offset_f = (float)h->le_offset;
    h->le_build_f = h->le_offset_f;
    h->fast_stamp = 1;          // fast_flag starts at 0: no particle listed
    CK(cudaMemcpyAsync(s->ds, h, sizeof(md_dstate), cudaMemcpyHostToDevice, st), "upload dstate");
    CK(cudaMemsetAsync(s->ctl, 0, sizeof(int32_t) * CTL_WORDS, st), "reset ctl");
    // empty rows until the first build (the workspace holds stale contents)
    const int64_t rows_k[4] = {s->n, s->n_plt, s->n_plt, s->n_rec};
    for (int k = 0; k < 4; ++k)
        if (s->nc[k] && rows_k[k] > 0) CK(cudaMemsetAsync(s->nc[k], 0, sizeof(int32_t) * rows_k[k], st), "reset rows");
    CK(cudaStreamSynchronize(st), "set_particles sync");
    s->host_step = step0;
    s->host_sub = 0;
    s->lists_stale = true;
    s->forces_stale = true;
    s->forces_levels = 0;
    return MD_OK;
}

// md_set_xv after the placement: counters, rebuild check, forces cleared,
// the check's verdict read back.
static int finish_set_xv(md_system *s, int64_t step0)
{
    const int64_t n = s->n;
    cudaStream_t st = s->stream;
    CK(cudaMemsetAsync(s->ctl + CTL_UNSTABLE, 0, sizeof(int32_t), st), "reset unstable");
    CK(launch_set_time(s, step0, 0, (double)step0 * s->cfg.dt), "time");
    CK(launch_check_placed(s, step0), "check");
    for (int l = 0; l < 3; ++l)
        if (s->f[l]) CK(cudaMemsetAsync(s->f[l], 0, sizeof(float4) * n, st), "zero f");
    CK(cudaMemcpyAsync(s->h_ctl, s->ctl, sizeof(int32_t) * CTL_WORDS, cudaMemcpyDeviceToHost, st), "read ctl");
    CK(cudaStreamSynchronize(st), "set_xv sync");
    s->host_step = step0;
    s->host_sub = 0;
    s->lists_stale = s->h_ctl[CTL_REBUILD] != 0;
    s->forces_stale = true;
    s->forces_levels = 0;
    if (s->h_ctl[CTL_UNSTABLE]) return set_error(s, MD_EUNSTABLE, "md_set_xv: non-finite or escaped position");
    return MD_OK;
}

int md_set_xv(md_system *s, const double *x, const double *v, int64_t step0)
{
    if (!s || !x || !v) return set_error(s, MD_EINVAL, "md_set_xv: null argument");
    if (!s->have_particles) return set_error(s, MD_EINVAL, "md_set_xv: md_set_particles was never called");
    if (s->lists_stale) return load_xv(s, x, v, step0);
    // lists built: the new state goes into the current storage order and
    // keeps them if the kick-drift's rebuild check passes on it
    const int64_t n = s->n;
    s->det_levels = 0;
    cudaStream_t st = s->stream;
    // page-locked host arrays: both uploads back to back on a side stream
    // (after the work already on st), the positions placed while the
    // velocities are still arriving, staged in the deterministic-mode buffer
    // of the fluid level (3n words, free here: this call voids the
    // deterministic results anyway).  Pageable arrays: one stream (their
    // copies go through the driver's staging and gain nothing from it).
    cudaPointerAttributes ax, av;
    const bool pinned = cudaPointerGetAttributes(&ax, x) == cudaSuccess &&
                        cudaPointerGetAttributes(&av, v) == cudaSuccess && ax.type == cudaMemoryTypeHost &&
                        av.type == cudaMemoryTypeHost;
    cudaGetLastError();   // an unregistered pointer may leave an error behind on older runtimes
    if (!pinned) {
        CK(cudaMemcpyAsync(s->alt64, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st), "upload x");
        CK(launch_place_state(s, s->alt64, false), "place x");
        CK(cudaMemcpyAsync(s->alt64, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st), "upload v");
        CK(launch_place_state(s, s->alt64, true), "place v");
        return finish_set_xv(s, step0);
    }
    struct side_t {
        cudaStream_t cs = nullptr;
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        ~side_t()
        {
            if (cs) cudaStreamSynchronize(cs);   // no copy outlives the call, on any path
            for (auto e : ev)
                if (e) cudaEventDestroy(e);
            if (cs) cudaStreamDestroy(cs);
        }
    } side;
    CK(cudaStreamCreateWithFlags(&side.cs, cudaStreamNonBlocking), "upload stream");
    for (auto &e : side.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "upload events");
    double *vstage = reinterpret_cast<double *>(s->fdet[0]);
    CK(cudaEventRecord(side.ev[0], st), "fork");
    CK(cudaStreamWaitEvent(side.cs, side.ev[0], 0), "fork wait");
    CK(cudaMemcpyAsync(s->alt64, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, side.cs), "upload x");
    CK(cudaEventRecord(side.ev[1], side.cs), "x uploaded");
    CK(cudaMemcpyAsync(vstage, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, side.cs), "upload v");
    CK(cudaEventRecord(side.ev[2], side.cs), "v uploaded");
    CK(cudaStreamWaitEvent(st, side.ev[1], 0), "x wait");
    CK(launch_place_state(s, s->alt64, false), "place x");
    CK(cudaStreamWaitEvent(st, side.ev[2], 0), "v wait");
    CK(launch_place_state(s, vstage, true), "place v");
    return finish_set_xv(s, step0);
}

// First and last platelet of every block of MSM_TPB terms of an array
// grouped by platelet (platelet p's terms at [off[p], off[p+1])).
static std::vector<int2> block_platelets(const std::vector<int32_t> &off, int64_t n)
{
    const int64_t nblk = (n + MSM_TPB - 1) / MSM_TPB;
    std::vector<int2> blk((size_t)nblk);
    int p = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        const int64_t t0 = b * MSM_TPB, t1 = std::min(t0 + MSM_TPB, n) - 1;
        while (off[(size_t)p + 1] <= t0) ++p;
        int q = p;
        while (off[(size_t)q + 1] <= t1) ++q;
        blk[(size_t)b] = make_int2(p, q);
    }
    return blk;
}

int md_set_bonds(md_system *s, const int32_t *ij, const double *r0, int64_t nb)
{
    if (!s) return MD_EINVAL;
    if (nb != s->nb) return set_error(s, MD_EINVAL, "md_set_bonds: count differs from the configuration");
    if (nb == 0) return MD_OK;
    if (!ij || !r0) return set_error(s, MD_EINVAL, "md_set_bonds: null argument");
    if ((int64_t)s->h_tag.size() != s->n) return set_error(s, MD_EINVAL, "md_set_bonds: set particles first");
    const int P = s->cfg.n_platelets;
    std::vector<int32_t> off((size_t)(P > 0 ? P : 0) + 1, 0);
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t i = ij[2 * b], j = ij[2 * b + 1];
        if (i < 0 || i >= s->n || j < 0 || j >= s->n)
            return set_error(s, MD_EINVAL, "md_set_bonds: particle id out of range");
        const int32_t ti = s->h_tag[(size_t)i], tj = s->h_tag[(size_t)j];
        if (ti < 0 || tj < 0 || (ti & ~MD_RECEPTOR_BIT) != (tj & ~MD_RECEPTOR_BIT))
            return set_error(s, MD_EINVAL, "md_set_bonds: a bond must join two particles of one platelet");
        off[(size_t)(ti & ~MD_RECEPTOR_BIT) + 1]++;
    }
    for (int p = 0; p < P; ++p) off[(size_t)p + 1] += off[(size_t)p];
    // store the bonds grouped by platelet (the bond kernel is order-independent)
    std::vector<int32_t> ijs((size_t)(2 * nb));
    std::vector<float> r0f((size_t)nb);
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t p = s->h_tag[(size_t)ij[2 * b]] & ~MD_RECEPTOR_BIT;
        const int32_t q = fill[(size_t)p]++;
        ijs[(size_t)(2 * q)] = ij[2 * b];
        ijs[(size_t)(2 * q + 1)] = ij[2 * b + 1];
        r0f[(size_t)q] = (float)r0[b];
    }
    CK(cudaMemcpyAsync(s->bond_id, ijs.data(), sizeof(int32_t) * 2 * nb, cudaMemcpyHostToDevice, s->stream),
       "upload bonds");
    CK(cudaMemcpyAsync(s->bond_r0, r0f.data(), sizeof(float) * nb, cudaMemcpyHostToDevice, s->stream), "upload r0");
    CK(cudaMemcpyAsync(s->bond_off, off.data(), sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice, s->stream),
       "upload bond offsets");
    std::vector<int2> blk = block_platelets(off, nb);
    CK(cudaMemcpyAsync(s->bond_blk, blk.data(), sizeof(int2) * blk.size(), cudaMemcpyHostToDevice, s->stream),
       "upload bond blocks");
    CK(cudaStreamSynchronize(s->stream), "set_bonds sync");
    s->have_bonds = true;
    s->lists_stale = true;   // the remap of bond ends happens in the rebuild
    s->forces_stale = true;
    return MD_OK;
}

int md_set_angles(md_system *s, const int32_t *ijk, const double *theta0, int64_t na)
{
    if (!s) return MD_EINVAL;
    if (na != s->na) return set_error(s, MD_EINVAL, "md_set_angles: count differs from the configuration");
    if (na == 0) return MD_OK;
    if (!ijk || !theta0) return set_error(s, MD_EINVAL, "md_set_angles: null argument");
    if ((int64_t)s->h_tag.size() != s->n) return set_error(s, MD_EINVAL, "md_set_angles: set particles first");
    const int P = s->cfg.n_platelets;
    std::vector<int32_t> plt_of((size_t)na), off((size_t)P + 1, 0);
    for (int64_t q = 0; q < na; ++q) {
        int32_t pl = -1;
        for (int e = 0; e < 3; ++e) {
            const int32_t i = ijk[3 * q + e];
            if (i < 0 || i >= s->n) return set_error(s, MD_EINVAL, "md_set_angles: particle id out of range");
            const int32_t t = s->h_tag[(size_t)i];
            if (t < 0) return set_error(s, MD_EINVAL, "md_set_angles: a triplet must lie on one platelet");
            if (pl >= 0 && (t & ~MD_RECEPTOR_BIT) != pl)
                return set_error(s, MD_EINVAL, "md_set_angles: a triplet must lie on one platelet");
            pl = t & ~MD_RECEPTOR_BIT;
        }
        if (!(theta0[q] >= 0.0 && theta0[q] <= 3.14159265358979323846))
            return set_error(s, MD_EINVAL, "md_set_angles: rest angle outside [0, pi]");
        plt_of[(size_t)q] = pl;
        off[(size_t)pl + 1]++;
    }
    for (int p = 0; p < P; ++p) off[(size_t)p + 1] += off[(size_t)p];
    // stored grouped by platelet (the angle kernel is order-independent)
    std::vector<int32_t> ids((size_t)(3 * na)), fill(off.begin(), off.end() - 1);
    std::vector<float> t0((size_t)na);
    for (int64_t q = 0; q < na; ++q) {
        const int32_t r = fill[(size_t)plt_of[(size_t)q]]++;
        for (int e = 0; e < 3; ++e) ids[(size_t)(3 * r + e)] = ijk[3 * q + e];
        t0[(size_t)r] = (float)theta0[q];
    }
    CK(cudaMemcpyAsync(s->angle_id, ids.data(), sizeof(int32_t) * 3 * na, cudaMemcpyHostToDevice, s->stream),
       "angles");
    CK(cudaMemcpyAsync(s->angle_t0, t0.data(), sizeof(float) * na, cudaMemcpyHostToDevice, s->stream), "theta0");
    std::vector<int2> blk = block_platelets(off, na);
    CK(cudaMemcpyAsync(s->angle_blk, blk.data(), sizeof(int2) * blk.size(), cudaMemcpyHostToDevice, s->stream),
       "upload angle blocks");
    CK(cudaStreamSynchronize(s->stream), "set_angles sync");
    s->have_angles = true;
    s->lists_stale = true;   // the remap of the triplets happens in the rebuild
    s->forces_stale = true;
    return MD_OK;
}

int md_set_platelet_levels(md_system *s, const int32_t *k)
{
    if (!s || !k) return set_error(s, MD_EINVAL, "md_set_platelet_levels: null argument");
    if (s->n_plt == 0 || !s->plt_k) return set_error(s, MD_EINVAL, "md_set_platelet_levels: no platelets");
    const int P = s->cfg.n_platelets;
    int64_t K = 1;
    for (int p = 0; p < P; ++p) {
        if (k[p] < 1 || k[p] > MD_AI_K_LCM_MAX)
            return set_error(s, MD_EINVAL, "md_set_platelet_levels: k out of range");
        int64_t a = K, b = k[p];
        while (b) { const int64_t t = a % b; a = b; b = t; }
        K = K / a * k[p];
        if (K > MD_AI_K_LCM_MAX) return set_error(s, MD_EINVAL, "md_set_platelet_levels: lcm(k) too large");
    }
    CK(cudaMemcpyAsync(s->plt_k, k, sizeof(int32_t) * P, cudaMemcpyHostToDevice, s->stream), "upload k");
    CK(cudaStreamSynchronize(s->stream), "levels sync");
    s->h_plt_k.assign(k, k + P);
    s->plt_K = (int)K;
    s->have_levels = true;
    if (!s->lists_stale) {     // else the next build sets the strides
        CK(launch_strides(s, nullptr), "drift strides");
        CK(cudaStreamSynchronize(s->stream), "strides sync");
    }
    return MD_OK;
}

int md_neighbor_build(md_system *s, uint32_t list_mask, int force)
{
    if (!s || !s->have_particles) return set_error(s, MD_EINVAL, "md_neighbor_build: no particles");
    if (list_mask & ~0xFu) return set_error(s, MD_EINVAL, "md_neighbor_build: bad list mask");
    s->det_levels = 0;
    if (force || s->lists_stale) {
        int rc = request_rebuild(s);
        if (rc) return rc;
    } else {
        CK(launch_rebuild(s, s->ctl + CTL_REBUILD), "rebuild");
    }
    return check_flags(s);
}

int md_forces(md_system *s, uint32_t level_mask, uint32_t flags)
{
    if (!s || !s->have_particles) return set_error(s, MD_EINVAL, "md_forces: no particles");
    if ((level_mask & ~MD_LEVEL_ALL) || !level_mask) return set_error(s, MD_EINVAL, "md_forces: bad level mask");
    if (s->nb > 0 && !s->have_bonds) return set_error(s, MD_EINVAL, "md_forces: bonds not set");
    if (s->na > 0 && !s->have_angles) return set_error(s, MD_EINVAL, "md_forces: angles not set");
    int rc = ensure_lists(s);
    if (rc) return rc;
    if (s->n_plt == 0) level_mask &= MD_LEVEL_FLUID;
    if (flags & ~(MD_FORCE_VIRIAL | MD_FORCE_DETERMINISTIC)) return set_error(s, MD_EINVAL, "md_forces: bad flags");
    rc = eval_forces(s, level_mask, (flags & MD_FORCE_VIRIAL) != 0, (flags & MD_FORCE_DETERMINISTIC) != 0);
    if (rc) return rc;
    s->forces_levels = level_mask;
    s->forces_stale = level_mask != (s->n_plt > 0 ? MD_LEVEL_ALL : MD_LEVEL_FLUID);
    return check_flags(s);
}

int md_read_forces(md_system *s, uint32_t level_mask, double *f)
{
    if (!s || !f) return MD_EINVAL;
    const int rc = ensure_forces(s);
    if (rc) return rc;
    const int64_t n = s->n;
    if (s->det_levels && !(level_mask & ~s->det_levels)) {
        // the last md_forces was deterministic and covers the levels: exact sums
        k_export_fixed<<<blocks_for(n), MSM_TPB, 0, s->stream>>>(
            n, (level_mask & MD_LEVEL_FLUID) ? s->fdet[0] : nullptr, (level_mask & MD_LEVEL_IFACE) ? s->fdet[1] : nullptr,
            (level_mask & MD_LEVEL_PLT) ? s->fdet[2] : nullptr, s->x32, s->tag_s, (float)s->cfg.body_force, s->alt64);
    } else {
        const float4 *f0 = (level_mask & MD_LEVEL_FLUID) ? s->f[0] : nullptr;
        const float4 *f1 = (level_mask & MD_LEVEL_IFACE) ? s->f[1] : nullptr;
        const float4 *f2 = (level_mask & MD_LEVEL_PLT) ? s->f[2] : nullptr;
        k_export_forces<<<blocks_for(n), MSM_TPB, 0, s->stream>>>(n, f0, f1, f2, s->x32, s->tag_s,
                                                                   (float)s->cfg.body_force, s->alt64);
    }
    CK(cudaGetLastError(), "export forces");
    CK(cudaMemcpyAsync(f, s->alt64, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream), "download forces");
    CK(cudaStreamSynchronize(s->stream), "read_forces sync");
    return MD_OK;
}

int md_read_particles(md_system *s, double *x, double *v, float *x32)
{
    if (!s) return MD_EINVAL;
    const int64_t n = s->n;
    cudaStream_t st = s->stream;
    if (x) {
        k_export_x<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->xs, s->ys, s->zs, s->x32, s->alt64);
        CK(cudaGetLastError(), "export x");
        CK(cudaMemcpyAsync(x, s->alt64, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st), "download x");
        CK(cudaStreamSynchronize(st), "sync");
    }
    if (v) {
        k_export_f4<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->v, s->x32, s->alt64);
        CK(cudaGetLastError(), "export v");
        CK(cudaMemcpyAsync(v, s->alt64, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st), "download v");
        CK(cudaStreamSynchronize(st), "sync");
    }
    if (x32) {
        k_export_x32<<<blocks_for(n), MSM_TPB, 0, st>>>(n, s->x32, (float *)s->alt64);
        CK(cudaGetLastError(), "export x32");
        CK(cudaMemcpyAsync(x32, s->alt64, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st), "download x32");
        CK(cudaStreamSynchronize(st), "sync");
    }
    return MD_OK;
}

int md_mts_step(md_system *s, int64_t n_outer, const md_mts_schedule *sched)
{
    if (!s || !sched || n_outer < 0) return set_error(s, MD_EINVAL, "md_mts_step: bad argument");
    if (!s->have_particles) return set_error(s, MD_EINVAL, "md_mts_step: no particles");
    if (s->nb > 0 && !s->have_bonds) return set_error(s, MD_EINVAL, "md_mts_step: bonds not set");
    if (s->na > 0 && !s->have_angles) return set_error(s, MD_EINVAL, "md_mts_step: angles not set");
    if (n_outer == 0) return MD_OK;
    s->det_levels = 0;
    const int mode = sched->mode;
    const bool record = (sched->flags & MD_SCHED_RECORD) != 0;
    if (record && s->n_plt == 0) return set_error(s, MD_EINVAL, "md_mts_step: recording needs platelets");
    const bool det = (sched->flags & MD_SCHED_DETERMINISTIC) != 0;
    if (det && mode == MD_MODE_AI)
        return set_error(s, MD_EINVAL, "md_mts_step: deterministic steps cover STS and RESPA, not AI-MTS");
    // the forces at hand (computed, or restored from a checkpoint) are part of
    // the state and are kept; the mode applies to every later evaluation
    s->det_step = det;
    int k_m = sched->k_m > 0 ? sched->k_m : 1;
    int k_p = sched->k_p > 0 ? sched->k_p : 1;
    if (mode == MD_MODE_STS) { k_m = 1; k_p = 1; }
    else if (mode == MD_MODE_AI) {
        if (s->n_plt == 0) return set_error(s, MD_EINVAL, "md_mts_step: AI-MTS needs platelets");
        if (!s->have_levels) return set_error(s, MD_EINVAL, "md_mts_step: platelet levels not set");
        k_p = s->plt_K;   // the fine grid; part of the captured graph's shape
    } else if (mode != MD_MODE_RESPA) return set_error(s, MD_EINVAL, "md_mts_step: unsupported mode");
    if (s->cfg_k_m != k_m) {
        // the interface noise amplitude depends on dt_m: recompute those forces
        s->cfg_k_m = k_m;
        s->forces_stale = true;
    }
    s->margin = (mode == MD_MODE_STS) ? 0.0f : 0.05f;
    int rc = ensure_forces(s);
    if (rc) return rc;
    const md_config &c = s->cfg;
    if (mode == MD_MODE_AI) {
        // the platelet buffer switches to impulses: every term due (qe = K)
        CK(cudaMemsetAsync(s->f[2], 0, sizeof(float4) * s->n, s->stream), "zero platelet level");
        s->due_on = true;
        s->due_q = s->plt_K;
        s->due_dtm = c.dt / k_m;
        rc = enqueue_forces(s, MD_LEVEL_PLT);
        s->due_on = false;
        if (rc) return rc;
    }
    rc = enqueue_outer_step(s, mode, k_m, k_p, true, nullptr, record);
    if (rc) return rc;
    const int64_t rest = n_outer - 1;
    if (rest > 0) {
        bool use_graph = !s->prof_on && !s->graph_failed && !(sched->flags & MD_SCHED_DIRECT);
        if (use_graph && build_step_graph(s, mode, k_m, k_p, record) != MD_OK) {
            s->graph_failed = true;   // keep going with direct launches
            use_graph = false;
        }
        if (use_graph) {
            rc = sync_ctl(s);
            if (rc) return rc;
            const int64_t builds0 = s->h_ds->n_builds;
            CK(launch_set_loop(s, rest), "loop count");
            CK(cudaGraphLaunch(s->step_exec, s->stream), "graph launch");
            rc = sync_ctl(s);
            if (rc) return rc;
            s->nlaunch += rest * s->graph_body_launches + (s->h_ds->n_builds - builds0) * s->graph_chain_launches;
        } else {
            for (int64_t it = 0; it < rest; ++it) {
                rc = enqueue_outer_step(s, mode, k_m, k_p, false, nullptr, record);
                if (rc) return rc;
            }
        }
    }
    if (mode == MD_MODE_STS) {
        const float hh = (float)(0.5 * c.dt);
        rc = closing_kick(s, hh, hh, hh);
    } else {
        rc = closing_kick(s, (float)(0.5 * c.dt), 0.f, 0.f);
    }
    if (rc) return rc;
    if (mode == MD_MODE_AI) {
        // the platelet buffer held impulses: plain platelet forces of the final state
        CK(cudaMemsetAsync(s->f[2], 0, sizeof(float4) * s->n, s->stream), "zero platelet level");
        rc = enqueue_forces(s, MD_LEVEL_PLT);
        if (rc) return rc;
    }
    s->host_step += n_outer;
    return check_flags(s);
}

int md_flow_profile(md_system *s, int32_t nbins, double *out)
{
    if (!s || !out || nbins < 1 || nbins > PROF_BINS_MAX)
        return set_error(s, MD_EINVAL, "md_flow_profile: nbins must be in [1, 256]");
    CK(launch_flow_profile(s, nbins), "flow profile");
    std::vector<double> r((size_t)(2 * nbins));
    CK(cudaMemcpyAsync(r.data(), s->prof_part + (int64_t)PROF_BLOCKS * 2 * PROF_BINS_MAX, sizeof(double) * 2 * nbins,
                       cudaMemcpyDeviceToHost, s->stream), "download profile");
    CK(cudaStreamSynchronize(s->stream), "sync");
    const md_config &c = s->cfg;
    const double slab = c.box[0] * c.box[2] * c.box[1] / nbins;
    for (int b = 0; b < nbins; ++b) {
        out[b] = r[(size_t)(nbins + b)] > 0.0 ? r[(size_t)b] / r[(size_t)(nbins + b)] : 0.0;
        out[nbins + b] = r[(size_t)(nbins + b)] / slab;
    }
    return MD_OK;
}

int md_observables(md_system *s, md_observables_t *o)
{
    if (!s || !o) return MD_EINVAL;
    CK(launch_kinetics(s), "kinetics");
    double red[RED_WORDS], vir[9];
    CK(cudaMemcpyAsync(red, s->red_out, sizeof red, cudaMemcpyDeviceToHost, s->stream), "download kinetics");
    CK(cudaMemcpyAsync(vir, s->vir_acc, sizeof vir, cudaMemcpyDeviceToHost, s->stream), "download virial");
    int rc = sync_ctl(s);
    if (rc) return rc;
    memset(o, 0, sizeof *o);
    o->step = s->h_ds->step;
    o->time = s->h_ds->time;
    for (int k = 0; k < 3; ++k) o->momentum[k] = red[k];
    o->kinetic = red[3];
    const double kt[9] = {red[4], red[7], red[8], red[7], red[5], red[9], red[8], red[9], red[6]};
    memcpy(o->kin_tensor, kt, sizeof kt);
    memcpy(o->virial_c, vir, sizeof vir);
    const double nm = red[10];
    const double ndof = s->geom.walls ? 3.0 * nm : 3.0 * nm - 3.0;
    o->temperature = ndof > 0 ? (kt[0] + kt[4] + kt[8]) / ndof : 0.0;
    const double V = s->cfg.box[0] * s->cfg.box[1] * s->cfg.box[2];
    o->pressure = (kt[0] + kt[4] + kt[8] + vir[0] + vir[4] + vir[8]) / (3.0 * V);
    o->n_builds = s->h_ds->n_builds;
    for (int k = 0; k < 4; ++k) o->max_rows[k] = s->h_ctl[CTL_MAXROW + k];
    return MD_OK;
}

int md_platelet_features(md_system *s, double *out)
{
    if (!s || !out) return MD_EINVAL;
    if (s->n_plt == 0) return set_error(s, MD_EINVAL, "md_platelet_features: no platelets");
    int rc = ensure_forces(s);
    if (rc) return rc;
    CK(launch_features(s, s->feat), "features");
    CK(cudaMemcpyAsync(out, s->feat, sizeof(double) * 12 * s->cfg.n_platelets, cudaMemcpyDeviceToHost, s->stream),
       "download features");
    CK(cudaStreamSynchronize(s->stream), "sync");
    return MD_OK;
}

int md_record_features(md_system *s)
{
    if (!s) return MD_EINVAL;
    if (s->n_plt == 0) return set_error(s, MD_EINVAL, "md_record_features: no platelets");
    int rc = ensure_forces(s);
    if (rc) return rc;
    CK(launch_features(s, s->feat), "features");
    CK(launch_feature_ring(s, s->feat), "feature ring");
    return MD_OK;
}

int md_read_feature_ring(md_system *s, float *out, int64_t *count)
{
    if (!s || !count) return MD_EINVAL;
    if (s->n_plt == 0) return set_error(s, MD_EINVAL, "md_read_feature_ring: no platelets");
    if (!out) {         // the record count alone
        int rc = sync_ctl(s);
        if (rc) return rc;
        *count = s->h_ds->ring_count;
        return MD_OK;
    }
    const int P = s->cfg.n_platelets, T = s->ring_T;
    std::vector<float> raw((size_t)P * T * 12);
    CK(cudaMemcpyAsync(raw.data(), s->ring, sizeof(float) * raw.size(), cudaMemcpyDeviceToHost, s->stream), "ring");
    int rc = sync_ctl(s);
    if (rc) return rc;
    const int64_t ring_count = s->h_ds->ring_count;
    // chronological order: the oldest retained record first
    const int64_t n = ring_count < T ? ring_count : T;
    const int64_t first = ring_count - n;
    for (int p = 0; p < P; ++p)
        for (int64_t t = 0; t < n; ++t) {
            const int64_t slot = (first + t) % T;
            memcpy(out + ((int64_t)p * T + t) * 12, raw.data() + ((int64_t)p * T + slot) * 12, 12 * sizeof(float));
        }
    *count = ring_count;
    return MD_OK;
}

int md_neighbor_pairs(md_system *s, int32_t kind, int32_t *pairs, int64_t cap, int64_t *count)
{
    if (!s || !count || kind < 0 || kind > 3) return MD_EINVAL;
    int rc = ensure_lists(s);
    if (rc) return rc;
    rc = check_flags(s);
    if (rc) return rc;
    const int64_t rows_k[4] = {s->n, s->n_plt, s->n_plt, s->n_rec};
    const int32_t *row_idx_k[4] = {nullptr, s->plt_sorted, s->plt_sorted, s->rec_sorted};
    const int64_t rows = rows_k[kind];
    *count = 0;
    if (rows == 0 || !s->nl[kind]) return MD_OK;
    const int cp = s->cap[kind];
    if (!pairs) {   // the count alone: the row counts (every pair is stored once)
        std::vector<int32_t> nc((size_t)rows);
        CK(cudaMemcpyAsync(nc.data(), s->nc[kind], sizeof(int32_t) * rows, cudaMemcpyDeviceToHost, s->stream), "nc");
        CK(cudaStreamSynchronize(s->stream), "sync");
        int64_t total = 0;
        for (int64_t r = 0; r < rows; ++r) total += nc[(size_t)r] < cp ? nc[(size_t)r] : cp;
        *count = total;
        return MD_OK;
    }
    std::vector<int32_t> nc((size_t)rows), nl((size_t)(rows * cp)), ridx;
    std::vector<float> x32h((size_t)(4 * s->n));
    cudaStream_t st = s->stream;
    CK(cudaMemcpyAsync(nc.data(), s->nc[kind], sizeof(int32_t) * rows, cudaMemcpyDeviceToHost, st), "nc");
    CK(cudaMemcpyAsync(nl.data(), s->nl[kind], sizeof(int32_t) * rows * cp, cudaMemcpyDeviceToHost, st), "nl");
    CK(cudaMemcpyAsync(x32h.data(), s->x32, sizeof(float4) * s->n, cudaMemcpyDeviceToHost, st), "x32");
    if (row_idx_k[kind]) {
        ridx.resize((size_t)rows);
        CK(cudaMemcpyAsync(ridx.data(), row_idx_k[kind], sizeof(int32_t) * rows, cudaMemcpyDeviceToHost, st), "rows");
    }
    CK(cudaStreamSynchronize(st), "sync");
    auto id_of_h = [&](int64_t k) {
        int32_t id;
        memcpy(&id, &x32h[(size_t)(4 * k + 3)], sizeof id);
        id &= (int32_t)MSM_ID_MASK;
        return id;
    };
    int64_t total = 0;
    if (kind == MD_LIST_FLUID) {
        // warp-stream layout: rows 32w .. 32w + 31 store their entries back
        // to back from row 32w's slot, each entry j | (row - 32w) << 27
        for (int64_t r0 = 0; r0 < rows; r0 += 32) {
            int64_t tot = 0;
            for (int64_t r = r0; r < rows && r < r0 + 32; ++r) tot += nc[(size_t)r] < cp ? nc[(size_t)r] : cp;
            for (int64_t f = 0; f < tot; ++f) {
                const uint32_t e = (uint32_t)nl[(size_t)(r0 * cp + f)];
                const int32_t idi = id_of_h(r0 + (e >> MSM_STREAM_SHIFT));
                const int32_t idj = id_of_h((int64_t)(e & MSM_STREAM_JMASK));
                if (pairs && total < cap) {
                    pairs[2 * total] = idi < idj ? idi : idj;
                    pairs[2 * total + 1] = idi < idj ? idj : idi;
                }
                ++total;
            }
        }
        *count = total;
        return MD_OK;
    }
    for (int64_t r = 0; r < rows; ++r) {
        const int64_t i = ridx.empty() ? r : ridx[(size_t)r];
        const int32_t idi = id_of_h(i);
        const int cnt = nc[(size_t)r] < cp ? nc[(size_t)r] : cp;
        for (int k = 0; k < cnt; ++k) {
            const int32_t idj = id_of_h(nl[(size_t)(r * cp + k)]);
            if (pairs && total < cap) {
                pairs[2 * total] = idi < idj ? idi : idj;
                pairs[2 * total + 1] = idi < idj ? idj : idi;
            }
            ++total;
        }
    }
    *count = total;
    return MD_OK;
}

// checkpoint blob: header, x64[3n] FP64, v[3n] FP32, forces nf x [3n] FP32
struct blob_header {
    uint64_t magic;
    int64_t n, step;
    int32_t sub, nf;
    double time;
};
static const uint64_t BLOB_MAGIC = 0x4d534d5354415445ull;

int md_get_state(md_system *s, void *blob, size_t *nbytes)
{
    if (!s || !nbytes) return MD_EINVAL;
    const int64_t n = s->n;
    const int nf = s->n_plt > 0 ? 3 : 1;
    const size_t need = sizeof(blob_header) + sizeof(double) * 3 * n + sizeof(float) * 3 * n * (1 + nf);
    if (!blob) { *nbytes = need; return MD_OK; }
    if (*nbytes < need) return set_error(s, MD_EINVAL, "md_get_state: blob too small");
    int rc = ensure_forces(s);
    if (rc) return rc;
    rc = sync_ctl(s);
    if (rc) return rc;
    blob_header h = {BLOB_MAGIC, n, s->host_step, s->host_sub, nf, s->h_ds->time};
    char *p = (char *)blob;
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    rc = md_read_particles(s, (double *)p, nullptr, nullptr);
    if (rc) return rc;
    p += sizeof(double) * 3 * n;
    std::vector<double> tmp((size_t)(3 * n));
    rc = md_read_particles(s, nullptr, tmp.data(), nullptr);
    if (rc) return rc;
    for (int64_t k = 0; k < 3 * n; ++k) ((float *)p)[k] = (float)tmp[(size_t)k];
    p += sizeof(float) * 3 * n;
    for (int l = 0; l < nf; ++l) {
        k_export_f4<<<blocks_for(n), MSM_TPB, 0, s->stream>>>(n, s->f[l], s->x32, s->alt64);
        CK(cudaGetLastError(), "export f");
        CK(cudaMemcpyAsync(tmp.data(), s->alt64, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream), "f");
        CK(cudaStreamSynchronize(s->stream), "sync");
        for (int64_t k = 0; k < 3 * n; ++k) ((float *)p)[k] = (float)tmp[(size_t)k];
        p += sizeof(float) * 3 * n;
    }
    *nbytes = need;
    return MD_OK;
}

int md_set_state(md_system *s, const void *blob, size_t nbytes)
{
    if (!s || !blob || nbytes < sizeof(blob_header)) return MD_EINVAL;
    s->det_levels = 0;
    blob_header h;
    memcpy(&h, blob, sizeof h);
    const int64_t n = s->n;
    const int nf = s->n_plt > 0 ? 3 : 1;
    if (h.magic != BLOB_MAGIC || h.n != n || h.nf != nf) return set_error(s, MD_EINVAL, "md_set_state: bad blob");
    const size_t need = sizeof(blob_header) + sizeof(double) * 3 * n + sizeof(float) * 3 * n * (1 + nf);
    if (nbytes < need) return set_error(s, MD_EINVAL, "md_set_state: blob too small");
    // tags stay as they are: read them back in id order
    std::vector<int32_t> tag((size_t)n);
    std::vector<int32_t> tag_sorted((size_t)n);
    std::vector<float> x32h((size_t)(4 * n));
    CK(cudaMemcpyAsync(tag_sorted.data(), s->tag_s, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->stream), "tags");
    CK(cudaMemcpyAsync(x32h.data(), s->x32, sizeof(float4) * n, cudaMemcpyDeviceToHost, s->stream), "ids");
    CK(cudaStreamSynchronize(s->stream), "sync");
    for (int64_t k = 0; k < n; ++k) {
        int32_t id;
        memcpy(&id, &x32h[(size_t)(4 * k + 3)], sizeof id);
        id &= (int32_t)MSM_ID_MASK;
        tag[(size_t)id] = tag_sorted[(size_t)k];
    }
    std::vector<double> X0;
    if (s->X0) {
        X0.resize((size_t)(3 * n));
        std::vector<float> x0f((size_t)(4 * n));
        CK(cudaMemcpyAsync(x0f.data(), s->X0, sizeof(float4) * n, cudaMemcpyDeviceToHost, s->stream), "X0");
        CK(cudaStreamSynchronize(s->stream), "sync");
        for (int64_t k = 0; k < n; ++k)
            for (int d = 0; d < 3; ++d) X0[(size_t)(3 * k + d)] = x0f[(size_t)(4 * k + d)];
    }
    const char *p = (const char *)blob + sizeof h;
    const double *x = (const double *)p;
    p += sizeof(double) * 3 * n;
    std::vector<double> v((size_t)(3 * n));
    for (int64_t k = 0; k < 3 * n; ++k) v[(size_t)k] = ((const float *)p)[k];
    p += sizeof(float) * 3 * n;
    int rc = md_set_particles(s, x, v.data(), tag.data(), s->X0 ? X0.data() : nullptr, h.step);
    if (rc) return rc;
    for (int l = 0; l < nf; ++l) {
        CK(cudaMemcpyAsync(s->alt64, p, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s->stream), "upload f");
        k_import_forces<<<blocks_for(n), MSM_TPB, 0, s->stream>>>(n, (const float *)s->alt64, s->f[l]);
        CK(cudaGetLastError(), "import f");
        p += sizeof(float) * 3 * n;
    }
    CK(cudaStreamSynchronize(s->stream), "sync");
    s->forces_stale = false;
    s->forces_levels = s->n_plt > 0 ? MD_LEVEL_ALL : MD_LEVEL_FLUID;
    return MD_OK;
}

}  // extern "C"
