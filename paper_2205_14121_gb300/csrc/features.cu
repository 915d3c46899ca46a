// K8: per-platelet measurements (Sec. 3.3: angular velocity, kinetic state,
// flow speed at the centre of mass) reduced in FP64 (raw sums over blocks of
// every platelet, then one block per platelet for the moments):
//
//  0-2  centre-of-mass velocity V
//  3-5  angular velocity w = I^-1 L (L, I about the centre of mass)
//  6-8  principal values (ascending) of S = -1/2 sum_i (r_i F_i^T + F_i r_i^T)
//  9    largest bond strain |r - r0| / r0
//  10   receptor contacts with other platelets closer than 1.5 r0 (Morse r0)
//  11   mean speed of the plasma within 2 of the centre of mass
//
// Positions enter through their FP32 copies (minimum image about the first
// member), velocities and forces as stored; every sum is FP64.
#include "msm_internal.cuh"

namespace {

constexpr int FT_TPB = 256;

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < FT_TPB / 32; ++k) s += sh[k];
    return s;
}

__device__ __forceinline__ double block_max(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = sh[0];
    for (int k = 1; k < FT_TPB / 32; ++k) s = fmax(s, sh[k]);
    return s;
}

// Eigenvalues of a symmetric 3x3 matrix (trigonometric closed form, Smith
// 1961), ascending.  In FP32 (FP64 transcendental functions are long
// sequences on the scarce FP64 pipe): the matrix is shifted by its mean
// eigenvalue and scaled by the spread p before the closed form, so the
// result keeps FP32 relative accuracy in p.
__device__ void sym3_eigvals(const double ad[6], double out[3])
{
    // a: xx, yy, zz, xy, xz, yz
    const double qd = (ad[0] + ad[1] + ad[2]) / 3.0;
    const float a0 = (float)(ad[0] - qd), a1 = (float)(ad[1] - qd), a2 = (float)(ad[2] - qd);
    const float a3 = (float)ad[3], a4 = (float)ad[4], a5 = (float)ad[5];
    const float p1 = a3 * a3 + a4 * a4 + a5 * a5;
    const float p2 = a0 * a0 + a1 * a1 + a2 * a2 + 2.0f * p1;
    if (!(p2 > 0.0f)) {
        out[0] = out[1] = out[2] = qd;
        return;
    }
    if (p1 <= 1e-30f * p2) {
        float e[3] = {a0, a1, a2};
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j)
                if (e[j] < e[i]) { const float t = e[i]; e[i] = e[j]; e[j] = t; }
        out[0] = qd + e[0]; out[1] = qd + e[1]; out[2] = qd + e[2];
        return;
    }
    const float p = sqrtf(p2 / 6.0f), ip = 1.0f / p;
    const float b0 = a0 * ip, b1 = a1 * ip, b2 = a2 * ip, b3 = a3 * ip, b4 = a4 * ip, b5 = a5 * ip;
    const float detb = b0 * (b1 * b2 - b5 * b5) - b3 * (b3 * b2 - b5 * b4) + b4 * (b3 * b5 - b1 * b4);
    const float rr = fminf(fmaxf(0.5f * detb, -1.0f), 1.0f);
    const float phi = acosf(rr) / 3.0f;
    const float e1 = 2.0f * p * cosf(phi);
    const float e3 = 2.0f * p * cosf(phi + 2.09439510f);
    const float e2 = -e1 - e3;
    out[0] = qd + e3; out[1] = qd + e2; out[2] = qd + e1;
}

struct feat_args {
    int P;
    const int32_t *plt_off, *plt_ids;      // members of platelet p: ids plt_ids[plt_off[p] .. plt_off[p+1])
    const int32_t *bond_off;               // bonds of platelet p: [bond_off[p], bond_off[p+1]) (platelet order)
    const int32_t *bond_ij;
    const float *bond_r0;
    const int32_t *pos_of_id;
    const float4 *x32, *v, *f0, *f1, *f2;
    const int32_t *tag;
    const int32_t *contacts;               // per platelet, from k_contacts
    md_grid g;
    md_geom geom;
    double L[3];
    float g_body;
    double flow_r2, skin;
    float hk[3];                           // half kicks still pending per level (0: none)
    double *out;                           // [P][12]
};

// Velocity at the recorded time: the stored one plus the half kicks that a
// step recording from inside itself has not applied yet (none otherwise).
__device__ __forceinline__ float4 vel_at(const feat_args &a, int k)
{
    float4 v = a.v[k];
    if ((a.hk[0] == 0.f && a.hk[1] == 0.f && a.hk[2] == 0.f) || a.tag[k] == MD_TAG_WALL) return v;
    const float4 *fl[3] = {a.f0, a.f1, a.f2};
    for (int l = 0; l < 3; ++l) {
        if (a.hk[l] == 0.f || !fl[l]) continue;
        const float4 q = fl[l][k];
        v.x += a.hk[l] * q.x; v.y += a.hk[l] * q.y; v.z += a.hk[l] * q.z;
    }
    v.x += a.hk[0] * a.g_body;
    return v;
}

// Minimum image of a separation along one axis (|d| < 1.5 L), no division.
__device__ __forceinline__ double img64(double d, double L, bool periodic)
{
    if (!periodic) return d;
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

// Raw FP64 sums per platelet, about its first member r_ref (the centre of
// mass is not known until every block has added its members):
//   0 n | 1-3 sum r | 4-6 sum v | 7-9 sum r x v | 10-15 sum r_a r_b (xx yy zz
//   xy xz yz) | 16-18 sum F | 19-24 sum (r_a F_b + F_a r_b) / 2
constexpr int FS_N = 25;

// Blocks (p, chunk): members and bonds of platelet p strided over the chunks
// of the y grid dimension; block sums go to the platelet's accumulators by
// FP64 atomics, the largest bond strain by an integer max on float bits.
// FP32 pair accumulator (hi, lo): Knuth's TwoSum keeps the rounding error
// of every addition, the fma residual that of every product.
struct ffacc {
    float hi, lo;
    __device__ void add(float x)
    {
        const float s = __fadd_rn(hi, x);
        const float bb = __fsub_rn(s, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
        hi = s;
    }
    __device__ void add_prod(float p, float q)
    {
        const float m = __fmul_rn(p, q);
        add(m);
        lo = __fadd_rn(lo, fmaf(p, q, -m));
    }
};

// Separation along one axis in FP32 (the correctly rounded difference of two
// FP32 coordinates) with the periodic image.
__device__ __forceinline__ float img32(float d, float L, bool periodic)
{
    if (periodic) {
        if (d > 0.5f * L) d -= L;
        else if (d < -0.5f * L) d += L;
    }
    return d;
}

__global__ void __launch_bounds__(FT_TPB) k_feat_sums(feat_args a, double *sums, unsigned *strain)
{
    // FP64 is scarce on this part: a thread sums its few members' position
    // and velocity terms in FP32 (each term rounded once, |r| < half the
    // box) and the force moments, whose terms cancel, in FP32 pairs with
    // exact products; warps and blocks reduce in FP32 pairs, platelets in FP64
    __shared__ float2 sh[FT_TPB / 32][FS_N];
    const int p = blockIdx.x;
    const int b = a.plt_off[p], e = a.plt_off[p + 1];
    const bool py = !a.geom.walls;
    const float4 ref = a.x32[a.pos_of_id[a.plt_ids[b]]];
    const float Lf[3] = {(float)a.L[0], (float)a.L[1], (float)a.L[2]};
    float ta[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) ta[q] = 0.0f;
    ffacc tb[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) tb[q] = ffacc{0.0f, 0.0f};
    const int stride = gridDim.y * FT_TPB;
    for (int m = b + blockIdx.y * FT_TPB + threadIdx.x; m < e; m += stride) {
        const int k = a.pos_of_id[a.plt_ids[m]];
        const float4 xk = a.x32[k];
        const float4 vk = vel_at(a, k);
        const float rx = img32(xk.x - ref.x, Lf[0], true);
        const float ry = img32(xk.y - ref.y, Lf[1], py);
        const float rz = img32(xk.z - ref.z, Lf[2], true);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        if (a.f0) { const float4 q = a.f0[k]; fx += q.x; fy += q.y; fz += q.z; fx += a.g_body; }
        if (a.f1) { const float4 q = a.f1[k]; fx += q.x; fy += q.y; fz += q.z; }
        if (a.f2) { const float4 q = a.f2[k]; fx += q.x; fy += q.y; fz += q.z; }
        ta[0] += 1.0f;
        ta[1] += rx; ta[2] += ry; ta[3] += rz;
        ta[4] += vk.x; ta[5] += vk.y; ta[6] += vk.z;
        ta[7] += ry * vk.z - rz * vk.y; ta[8] += rz * vk.x - rx * vk.z; ta[9] += rx * vk.y - ry * vk.x;
        ta[10] += rx * rx; ta[11] += ry * ry; ta[12] += rz * rz; ta[13] += rx * ry; ta[14] += rx * rz; ta[15] += ry * rz;
        tb[0].add(fx); tb[1].add(fy); tb[2].add(fz);
        tb[3].add_prod(rx, fx); tb[4].add_prod(ry, fy); tb[5].add_prod(rz, fz);
        // (r_a F_b + F_a r_b) / 2, halved at the end
        tb[6].add_prod(rx, fy); tb[6].add_prod(fx, ry);
        tb[7].add_prod(rx, fz); tb[7].add_prod(fx, rz);
        tb[8].add_prod(ry, fz); tb[8].add_prod(fy, rz);
    }
    float smax = 0.f;
    for (int bb = a.bond_off[p] + blockIdx.y * FT_TPB + threadIdx.x; bb < a.bond_off[p + 1]; bb += stride) {
        const float4 xi = a.x32[a.bond_ij[2 * bb]], xj = a.x32[a.bond_ij[2 * bb + 1]];
        // the largest strain needs no FP64 arithmetic: the exact separation rounded to FP32
        const float dx = img32(xi.x - xj.x, Lf[0], true);
        const float dy = img32(xi.y - xj.y, Lf[1], py);
        const float dz = img32(xi.z - xj.z, Lf[2], true);
        const float r0 = a.bond_r0[bb];
        smax = fmaxf(smax, fabsf(sqrtf(dx * dx + dy * dy + dz * dz) - r0) / r0);
    }
    smax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(smax)));   // smax >= 0
    if ((threadIdx.x & 31) == 0 && smax > 0.f) atomicMax(&strain[p], __float_as_uint(smax));
    // warp sums and then the block's warps in FP32 pairs, one FP64 value
    // and atomic per block and word
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < FS_N; ++w) {
        ffacc v = w < 16 ? ffacc{ta[w < 16 ? w : 0], 0.0f} : tb[w >= 16 ? w - 16 : 0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, v.hi, o);
            const float ol = __shfl_xor_sync(0xffffffffu, v.lo, o);
            v.add(oh);
            v.lo = __fadd_rn(v.lo, ol);
        }
        if (lane == 0) sh[wid][w] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (threadIdx.x < FS_N) {
        ffacc v = {0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < FT_TPB / 32; ++q) {
            const float2 t = sh[q][threadIdx.x];
            v.add(t.x);
            v.lo = __fadd_rn(v.lo, t.y);
        }
        const double d = ((double)v.hi + (double)v.lo) * (threadIdx.x >= 22 ? 0.5 : 1.0);
        atomicAdd(&sums[(int64_t)p * FS_N + threadIdx.x], d);
    }
}

// One block per platelet: moments about the centre of mass from the raw
// sums, the flow speed around it, the 12 measurements.
__global__ void __launch_bounds__(FT_TPB) k_feat_final(feat_args a, const double *sums, const unsigned *strain)
{
    __shared__ double sh[FT_TPB / 32];
    const int p = blockIdx.x;
    const double *S = sums + (int64_t)p * FS_N;
    const bool py = !a.geom.walls;
    const double n = S[0];
    const double rc[3] = {S[1] / n, S[2] / n, S[3] / n}, vc[3] = {S[4] / n, S[5] / n, S[6] / n};
    const float4 ref = a.x32[a.pos_of_id[a.plt_ids[a.plt_off[p]]]];
    // plasma speed near the centre of mass (cells of the last list build:
    // particles have moved by less than skin/2 since)
    const double cx = ref.x + rc[0], cy = ref.y + rc[1], cz = ref.z + rc[2];
    const md_grid &g = a.g;
    const double rr = sqrt(a.flow_r2) + a.skin;
    const int reach[3] = {(int)ceil(rr / g.h[0]), (int)ceil(rr / g.h[1]), (int)ceil(rr / g.h[2])};
    const int c0[3] = {(int)floor((cx - g.lo[0]) / g.h[0]), (int)floor((cy - g.lo[1]) / g.h[1]),
                       (int)floor((cz - g.lo[2]) / g.h[2])};
    const int span[3] = {min(2 * reach[0] + 1, g.nc[0]), min(2 * reach[1] + 1, g.nc[1]), min(2 * reach[2] + 1, g.nc[2])};
    const int ncand = span[0] * span[1] * span[2];
    // the sphere test runs in FP32 (FP64 instructions are scarce on this
    // part); only candidates whose FP32 d^2 lies within `band` of the radius,
    // far more than the FP32 rounding of the coordinates can move it, repeat
    // it in FP64
    const float cf[3] = {(float)cx, (float)cy, (float)cz};
    const float Lf[3] = {(float)a.L[0], (float)a.L[1], (float)a.L[2]};
    const float r2f = (float)a.flow_r2;
    const float band = 1e-5f * (fmaxf(Lf[0], fmaxf(Lf[1], Lf[2])) + 1.0f) * (1.0f + r2f);
    double fs = 0.0, fn = 0.0;
    for (int q = threadIdx.x; q < ncand; q += FT_TPB) {
        const int ox = q % span[0], oy = (q / span[0]) % span[1], oz = q / (span[0] * span[1]);
        int ix = c0[0] - reach[0] + ox, iy = c0[1] - reach[1] + oy, iz = c0[2] - reach[2] + oz;
        ix = ((ix % g.nc[0]) + g.nc[0]) % g.nc[0];
        iz = ((iz % g.nc[2]) + g.nc[2]) % g.nc[2];
        if (py) iy = ((iy % g.nc[1]) + g.nc[1]) % g.nc[1];
        else if (iy < 0 || iy >= g.nc[1]) continue;
        const int64_t c = ((int64_t)iz * g.nc[1] + iy) * g.nc[0] + ix;
        for (int32_t k = g.start[c]; k < g.start[c + 1]; ++k) {
            const float4 xk = a.x32[k];
            if (class_of(xk) != CLS_FLUID) continue;
            const float ex = img32(xk.x - cf[0], Lf[0], true), ey = img32(xk.y - cf[1], Lf[1], py),
                        ez = img32(xk.z - cf[2], Lf[2], true);
            const float d2f = ex * ex + ey * ey + ez * ez;
            bool inside = d2f < r2f;
            if (fabsf(d2f - r2f) <= band) {
                const double dx = img64((double)xk.x - cx, a.L[0], true);
                const double dy = img64((double)xk.y - cy, a.L[1], py);
                const double dz = img64((double)xk.z - cz, a.L[2], true);
                inside = dx * dx + dy * dy + dz * dz < a.flow_r2;
            }
            if (inside) {
                const float4 vk = vel_at(a, k);
                fs += (double)sqrtf(vk.x * vk.x + vk.y * vk.y + vk.z * vk.z);
                fn += 1.0;
            }
        }
    }
    fs = block_sum(fs, sh);
    fn = block_sum(fn, sh);
    if (threadIdx.x == 0) {
        double *o = a.out + 12 * (int64_t)p;
        o[0] = vc[0]; o[1] = vc[1]; o[2] = vc[2];
        // about the centre of mass: L = sum r x v - n rc x vc, second moments
        // M_ab = sum r_a r_b - n rc_a rc_b, I = tr(M) 1 - M
        const double Lx = S[7] - n * (rc[1] * vc[2] - rc[2] * vc[1]);
        const double Ly = S[8] - n * (rc[2] * vc[0] - rc[0] * vc[2]);
        const double Lz = S[9] - n * (rc[0] * vc[1] - rc[1] * vc[0]);
        const double Mxx = S[10] - n * rc[0] * rc[0], Myy = S[11] - n * rc[1] * rc[1], Mzz = S[12] - n * rc[2] * rc[2];
        const double Mxy = S[13] - n * rc[0] * rc[1], Mxz = S[14] - n * rc[0] * rc[2], Myz = S[15] - n * rc[1] * rc[2];
        const double I00 = Myy + Mzz, I11 = Mxx + Mzz, I22 = Mxx + Myy, I01 = -Mxy, I02 = -Mxz, I12 = -Myz;
        const double c00 = I11 * I22 - I12 * I12, c01 = I02 * I12 - I01 * I22, c02 = I01 * I12 - I02 * I11;
        const double c11 = I00 * I22 - I02 * I02, c12 = I01 * I02 - I00 * I12, c22 = I00 * I11 - I01 * I01;
        const double det = I00 * c00 + I01 * c01 + I02 * c02;
        if (det != 0.0) {
            o[3] = (c00 * Lx + c01 * Ly + c02 * Lz) / det;
            o[4] = (c01 * Lx + c11 * Ly + c12 * Lz) / det;
            o[5] = (c02 * Lx + c12 * Ly + c22 * Lz) / det;
        } else {
            o[3] = o[4] = o[5] = 0.0;
        }
        // S = -1/2 sum (r' F^T + F r'^T), r' = r - rc
        const double F[3] = {S[16], S[17], S[18]};
        const double Sm[6] = {-(S[19] - rc[0] * F[0]), -(S[20] - rc[1] * F[1]), -(S[21] - rc[2] * F[2]),
                              -(S[22] - 0.5 * (rc[0] * F[1] + F[0] * rc[1])),
                              -(S[23] - 0.5 * (rc[0] * F[2] + F[0] * rc[2])),
                              -(S[24] - 0.5 * (rc[1] * F[2] + F[1] * rc[2]))};
        double ev[3];
        sym3_eigvals(Sm, ev);
        o[6] = ev[0]; o[7] = ev[1]; o[8] = ev[2];
        o[9] = (double)__uint_as_float(strain[p]);
        o[10] = a.contacts ? (double)a.contacts[p] : 0.0;
        o[11] = fn > 0.0 ? fs / fn : 0.0;
    }
}

// Receptor contacts: Morse-list pairs closer than r_c, counted for both platelets.
__global__ void k_contacts(int64_t rows, const int32_t *row_idx, const int32_t *nl, const int32_t *nc, int cap,
                           const float4 *x32, const int32_t *tag, md_geom geom, const md_dstate *ds, float rc2,
                           int32_t *contacts)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int32_t i = row_idx[r];
    const int cnt = min(nc[r], cap);
    const float4 xi = x32[i];
    const int pi = tag[i] & ~MD_RECEPTOR_BIT;
    for (int k = 0; k < cnt; ++k) {
        const int32_t j = nl[r * cap + k];
        float dx, dy, dz, vs;
        min_image_f32(geom, ds->le_offset_f, xi, x32[j], dx, dy, dz, vs);
        if (dx * dx + dy * dy + dz * dz < rc2) {
            atomicAdd(&contacts[pi], 1);
            atomicAdd(&contacts[tag[j] & ~MD_RECEPTOR_BIT], 1);
        }
    }
}

// One block: every record of this step goes to slot ring_count % T, then the
// counter advances (device-side, so a captured step graph records in place).
__global__ void k_feature_ring(const double *feat, int P, float *ring, int T, md_dstate *ds)
{
    const int slot = (int)(ds->ring_count % T);
    for (int q = threadIdx.x; q < P * 12; q += blockDim.x) {
        const int p = q / 12, c = q % 12;
        ring[((int64_t)p * T + slot) * 12 + c] = (float)feat[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) ds->ring_count += 1;
}

}  // namespace

cudaError_t launch_features(md_system *s, double *out_dev, const float4 *f_plt, const float *hk)
{
    const int P = s->cfg.n_platelets;
    if (P <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(s->plt_contacts, 0, sizeof(int32_t) * P, s->stream);
    if (e != cudaSuccess) return e;
    if (s->n_rec > 0) {
        const float rc = (float)(1.5 * s->cfg.morse_r0);
        k_contacts<<<(unsigned)((s->n_rec + 255) / 256), 256, 0, s->stream>>>(
            s->n_rec, s->rec_sorted, s->nl[MD_LIST_MORSE], s->nc[MD_LIST_MORSE], s->cap[MD_LIST_MORSE], s->x32,
            s->tag_s, s->geom, s->ds, rc * rc, s->plt_contacts);
        MSM_COUNT(s, 1);
    }
    feat_args a;
    a.P = P;
    a.plt_off = s->plt_off;
    a.plt_ids = s->plt_ids;
    a.bond_off = s->bond_off;
    a.bond_ij = s->bond_ij;
    a.bond_r0 = s->bond_r0;
    a.pos_of_id = s->pos_of_id;
    a.x32 = s->x32;
    a.v = s->v;
    a.f0 = s->f[0];
    a.f1 = s->f[1];
    a.f2 = f_plt ? f_plt : s->f[2];
    for (int l = 0; l < 3; ++l) a.hk[l] = hk ? hk[l] : 0.0f;
    a.tag = s->tag_s;
    a.contacts = s->plt_contacts;
    a.g = s->gmain;
    a.geom = s->geom;
    for (int d = 0; d < 3; ++d) a.L[d] = s->cfg.box[d];
    a.g_body = (float)s->cfg.body_force;
    a.flow_r2 = 4.0;
    a.skin = s->cfg.skin;
    a.out = out_dev;
    e = cudaMemsetAsync(s->feat_sums, 0, sizeof(double) * FS_N * P + sizeof(unsigned) * P, s->stream);
    if (e != cudaSuccess) return e;
    unsigned *strain = (unsigned *)(s->feat_sums + (int64_t)FS_N * P);
    const int mean_members = (int)((s->n_plt + P - 1) / P);
    const int chunks = min(256, mean_members / (2 * FT_TPB) + 1);    // blocks per platelet: two members per thread
    k_feat_sums<<<dim3(P, chunks), FT_TPB, 0, s->stream>>>(a, s->feat_sums, strain);
    k_feat_final<<<P, FT_TPB, 0, s->stream>>>(a, s->feat_sums, strain);
    MSM_COUNT(s, 2);
    return cudaGetLastError();
}

cudaError_t launch_feature_ring(md_system *s, const double *feat)
{
    const int P = s->cfg.n_platelets;
    k_feature_ring<<<1, 256, 0, s->stream>>>(feat, P, s->ring, s->ring_T, s->ds);
    MSM_COUNT(s, 1);
    return cudaGetLastError();
}
