// K8: reductions of the observables (Sec. 4.2): total momentum, kinetic
// energy and the peculiar kinetic tensor (velocity relative to the imposed
// Lees-Edwards profile, or with walls to the slab mean flow), in two passes
// (per-block partials, then one block over the partials) so the result does
// not depend on atomic order; and the y-binned plasma flow profile (Fig. 4).
#include "msm_internal.cuh"

namespace {

// word layout of the partials / result
enum { W_PX = 0, W_PY, W_PZ, W_KE, W_KXX, W_KYY, W_KZZ, W_KXY, W_KXZ, W_KYZ, W_N, W_COUNT };

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP32 pair (hi, lo) accumulators: FP64 instructions issue at a small
// fraction of the FP32 rate on this part, so the per-particle terms are summed
// in FP32 with error-free transformations (Knuth's TwoSum, and the fma
// residual of a product) and converted to FP64 once per thread.
struct ff { float hi, lo; };

__device__ __forceinline__ void ff_add(ff &a, float x)
{
    const float s = __fadd_rn(a.hi, x);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, err);
}

__device__ __forceinline__ void ff_add_prod(ff &a, float p, float q)
{
    const float m = __fmul_rn(p, q);
    ff_add(a, m);
    a.lo = __fadd_rn(a.lo, fmaf(p, q, -m));
}

__device__ __forceinline__ double ff_value(const ff &a) { return (double)a.hi + (double)a.lo; }

// accumulator slots (W_KE is formed at the end from Sum vx^2 and the yy, zz terms)
enum { A_PX = 0, A_PY, A_PZ, A_VXX, A_KXX, A_KYY, A_KZZ, A_KXY, A_KXZ, A_KYZ, A_COUNT };

__global__ void __launch_bounds__(MSM_TPB) k_kinetics(int64_t n, const float4 *__restrict__ v,
                                                     const double *__restrict__ ys, const int32_t *__restrict__ tag,
                                                     int le, double rate, double half_Ly, const double *flow,
                                                     int nbins, double *part)
{
    // walls: the local flow is the y-binned mean v_x of the mobile particles
    // (flow = [sum v_x][count] per bin), kept as an FP32 pair per bin;
    // Lees-Edwards: the imposed profile, subtracted in FP64
    __shared__ float uh[PROF_BINS_MAX], ul[PROF_BINS_MAX];
    if (flow)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
            const double u = flow[nbins + b] > 0.0 ? flow[b] / flow[nbins + b] : 0.0;
            uh[b] = (float)u;
            ul[b] = (float)(u - (double)uh[b]);
        }
    __syncthreads();
    const double scale = nbins / (2.0 * half_Ly);
    ff acc[A_COUNT];
#pragma unroll
    for (int w = 0; w < A_COUNT; ++w) acc[w] = ff{0.0f, 0.0f};
    int cnt = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        if (tag[k] == MD_TAG_WALL) continue;
        const float4 vv = v[k];
        // peculiar v_x = sx + ex (ex a correction below half an ulp of sx)
        float sx = vv.x, ex = 0.0f;
        if (le) {
            const double ux = (double)vv.x - rate * (ys[k] - half_Ly);
            sx = (float)ux;
            ex = (float)(ux - (double)sx);
        } else if (flow) {
            int b = (int)floor(ys[k] * scale);
            b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
            const float s = __fsub_rn(vv.x, uh[b]);
            const float bb = __fsub_rn(s, vv.x);
            const float err = __fadd_rn(__fsub_rn(vv.x, __fsub_rn(s, bb)), __fsub_rn(-uh[b], bb));
            sx = s;
            ex = __fsub_rn(err, ul[b]);
        }
        ff_add(acc[A_PX], vv.x); ff_add(acc[A_PY], vv.y); ff_add(acc[A_PZ], vv.z);
        ff_add_prod(acc[A_VXX], vv.x, vv.x);
        ff_add_prod(acc[A_KXX], sx, sx);
        acc[A_KXX].lo = fmaf(2.0f * sx, ex, acc[A_KXX].lo);
        ff_add_prod(acc[A_KYY], vv.y, vv.y);
        ff_add_prod(acc[A_KZZ], vv.z, vv.z);
        ff_add_prod(acc[A_KXY], sx, vv.y);
        acc[A_KXY].lo = fmaf(ex, vv.y, acc[A_KXY].lo);
        ff_add_prod(acc[A_KXZ], sx, vv.z);
        acc[A_KXZ].lo = fmaf(ex, vv.z, acc[A_KXZ].lo);
        ff_add_prod(acc[A_KYZ], vv.y, vv.z);
        ++cnt;
    }
    double out[W_COUNT];
    out[W_PX] = ff_value(acc[A_PX]); out[W_PY] = ff_value(acc[A_PY]); out[W_PZ] = ff_value(acc[A_PZ]);
    out[W_KXX] = ff_value(acc[A_KXX]); out[W_KYY] = ff_value(acc[A_KYY]); out[W_KZZ] = ff_value(acc[A_KZZ]);
    out[W_KXY] = ff_value(acc[A_KXY]); out[W_KXZ] = ff_value(acc[A_KXZ]); out[W_KYZ] = ff_value(acc[A_KYZ]);
    out[W_KE] = 0.5 * (ff_value(acc[A_VXX]) + out[W_KYY] + out[W_KZZ]);
    out[W_N] = (double)cnt;
    __shared__ double sh[MSM_TPB / 32][W_COUNT];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < W_COUNT; ++w) {
        const double s = warp_sum(out[w]);
        if (lane == 0) sh[wid][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < W_COUNT) {
        double s = 0.0;
        for (int q = 0; q < MSM_TPB / 32; ++q) s += sh[q][threadIdx.x];
        part[(int64_t)blockIdx.x * RED_WORDS + threadIdx.x] = s;
    }
}

// One warp per word: lanes stride over the block partials, then a shuffle sum.
__global__ void k_reduce_final(const double *part, int nblocks, double *out)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= W_COUNT) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += part[(int64_t)b * RED_WORDS + w];
    s = warp_sum(s);
    if (lane == 0) out[w] = s;
}

// Flow profile: v_x summed per slab of y (shared-memory bins per block, then
// one pass over the block partials per bin).  Sorted storage keeps a warp's 32
// consecutive particles in one or two slabs, so each warp sums its lanes per
// distinct slab with shuffles and adds one value per slab to shared memory.
__global__ void __launch_bounds__(MSM_TPB) k_profile(int64_t n, const float4 *__restrict__ v,
                                                    const double *__restrict__ ys, const int32_t *__restrict__ tag,
                                                    double Ly, int nbins, int mobile, double *part)
{
    __shared__ double sv[PROF_BINS_MAX], sn[PROF_BINS_MAX];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) { sv[b] = 0.0; sn[b] = 0.0; }
    __syncthreads();
    const double scale = nbins / Ly;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < n; base += nw * 32) {
        const int64_t k = base + lane;
        int b = -1;
        double vx = 0.0;
        if (k < n) {
            const int32_t t = tag[k];
            const double y = ys[k];
            // plasma, clamped to the edge slabs; or every mobile particle inside [0, Ly)
            const bool in = mobile ? (t != MD_TAG_WALL && y >= 0.0 && y < Ly) : t == MD_TAG_FLUID;
            if (in) {
                b = (int)floor(y * scale);
                b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
                vx = (double)v[k].x;
            }
        }
        unsigned pending = __ballot_sync(0xffffffffu, b >= 0);
        while (pending) {
            const int leader = __ffs(pending) - 1;
            const int bl = __shfl_sync(0xffffffffu, b, leader);
            const unsigned m = __ballot_sync(0xffffffffu, b == bl);
            const double s = warp_sum(b == bl ? vx : 0.0);
            if (lane == leader) {
                atomicAdd(&sv[bl], s);
                atomicAdd(&sn[bl], (double)__popc(m));
            }
            pending &= ~m;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        part[(int64_t)blockIdx.x * 2 * PROF_BINS_MAX + b] = sv[b];
        part[(int64_t)blockIdx.x * 2 * PROF_BINS_MAX + PROF_BINS_MAX + b] = sn[b];
    }
}

// One warp per output word (nbins sums, then nbins counts).
__global__ void k_profile_final(const double *part, int nblocks, int nbins, double *out)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= 2 * nbins) return;
    const int col = w < nbins ? w : PROF_BINS_MAX + (w - nbins);
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += part[(int64_t)b * 2 * PROF_BINS_MAX + col];
    s = warp_sum(s);
    if (lane == 0) out[w] = s;
}

}  // namespace

cudaError_t launch_flow_profile(md_system *s, int nbins, bool mobile)
{
    k_profile<<<PROF_BLOCKS, MSM_TPB, 0, s->stream>>>(s->n, s->v, s->ys, s->tag_s, s->cfg.box[1], nbins, mobile ? 1 : 0,
                                                    s->prof_part);
    k_profile_final<<<(2 * nbins + 7) / 8, 256, 0, s->stream>>>(s->prof_part, PROF_BLOCKS, nbins,
                                                                    s->prof_part + (int64_t)PROF_BLOCKS * 2 * PROF_BINS_MAX);
    MSM_COUNT(s, 2);
    return cudaGetLastError();
}

cudaError_t launch_kinetics(md_system *s)
{
    const int nb = s->red_blocks;
    const double *flow = nullptr;
    if (s->geom.walls) {
        cudaError_t e = launch_flow_profile(s, KIN_BINS, true);
        if (e != cudaSuccess) return e;
        flow = s->prof_part + (int64_t)PROF_BLOCKS * 2 * PROF_BINS_MAX;
    }
    k_kinetics<<<nb, MSM_TPB, 0, s->stream>>>(s->n, s->v, s->ys, s->tag_s, s->geom.le, s->cfg.shear_rate,
                                              0.5 * s->cfg.box[1], flow, KIN_BINS, s->red_part);
    k_reduce_final<<<1, 32 * W_COUNT, 0, s->stream>>>(s->red_part, nb, s->red_out);
    MSM_COUNT(s, 2);
    return cudaGetLastError();
}
