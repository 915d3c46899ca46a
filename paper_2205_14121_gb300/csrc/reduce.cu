// K8: FP64 reductions of the observables (Sec. 4.2): total momentum,
// kinetic energy and the peculiar kinetic tensor (velocity relative to the
// imposed Lees-Edwards profile), in two passes (per-block partials, then one
// block over the partials) so the result does not depend on atomic order;
// and the y-binned plasma flow profile (Fig. 4).
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

__global__ void __launch_bounds__(MSM_TPB) k_kinetics(int64_t n, const float4 *__restrict__ v,
                                                     const double *__restrict__ ys, const int32_t *__restrict__ tag,
                                                     int le, double rate, double half_Ly, const double *flow,
                                                     int nbins, double *part)
{
    // walls: the local flow is the y-binned mean v_x of the mobile particles
    // (flow = [sum v_x][count] per bin); Lees-Edwards: the imposed profile
    __shared__ double ub[PROF_BINS_MAX];
    if (flow)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            ub[b] = flow[nbins + b] > 0.0 ? flow[b] / flow[nbins + b] : 0.0;
    __syncthreads();
    const double scale = nbins / (2.0 * half_Ly);
    double acc[W_COUNT];
#pragma unroll
    for (int w = 0; w < W_COUNT; ++w) acc[w] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        if (tag[k] == MD_TAG_WALL) continue;
        const float4 vv = v[k];
        const double vx = vv.x, vy = vv.y, vz = vv.z;
        double ux = le ? vx - rate * (ys[k] - half_Ly) : vx;
        if (flow) {
            int b = (int)floor(ys[k] * scale);
            b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
            ux -= ub[b];
        }
        acc[W_PX] += vx; acc[W_PY] += vy; acc[W_PZ] += vz;
        acc[W_KE] += 0.5 * (vx * vx + vy * vy + vz * vz);
        acc[W_KXX] += ux * ux; acc[W_KYY] += vy * vy; acc[W_KZZ] += vz * vz;
        acc[W_KXY] += ux * vy; acc[W_KXZ] += ux * vz; acc[W_KYZ] += vy * vz;
        acc[W_N] += 1.0;
    }
    __shared__ double sh[MSM_TPB / 32][W_COUNT];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < W_COUNT; ++w) {
        const double s = warp_sum(acc[w]);
        if (lane == 0) sh[wid][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < W_COUNT) {
        double s = 0.0;
        for (int q = 0; q < MSM_TPB / 32; ++q) s += sh[q][threadIdx.x];
        part[(int64_t)blockIdx.x * RED_WORDS + threadIdx.x] = s;
    }
}

__global__ void k_reduce_final(const double *part, int nblocks, double *out)
{
    const int w = threadIdx.x;
    if (w >= RED_WORDS) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * RED_WORDS + w];
    out[w] = s;
}

// Flow profile: plasma v_x summed per slab of y in [0, Ly) (shared-memory
// bins per block, then one pass over the block partials per bin).
__global__ void __launch_bounds__(MSM_TPB) k_profile(int64_t n, const float4 *__restrict__ v,
                                                    const double *__restrict__ ys, const int32_t *__restrict__ tag,
                                                    double Ly, int nbins, int mobile, double *part)
{
    __shared__ double sv[PROF_BINS_MAX], sn[PROF_BINS_MAX];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) { sv[b] = 0.0; sn[b] = 0.0; }
    __syncthreads();
    const double scale = nbins / Ly;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        // plasma, clamped to the edge slabs; or every mobile particle inside [0, Ly)
        if (mobile ? (tag[k] == MD_TAG_WALL || ys[k] < 0.0 || ys[k] >= Ly) : tag[k] != MD_TAG_FLUID) continue;
        int b = (int)floor(ys[k] * scale);
        b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
        atomicAdd(&sv[b], (double)v[k].x);
        atomicAdd(&sn[b], 1.0);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        part[(int64_t)blockIdx.x * 2 * PROF_BINS_MAX + b] = sv[b];
        part[(int64_t)blockIdx.x * 2 * PROF_BINS_MAX + PROF_BINS_MAX + b] = sn[b];
    }
}

__global__ void k_profile_final(const double *part, int nblocks, int nbins, double *out)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= 2 * nbins) return;
    const int col = w < nbins ? w : PROF_BINS_MAX + (w - nbins);
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * 2 * PROF_BINS_MAX + col];
    out[w] = s;
}

}  // namespace

cudaError_t launch_flow_profile(md_system *s, int nbins, bool mobile)
{
    k_profile<<<PROF_BLOCKS, MSM_TPB, 0, s->stream>>>(s->n, s->v, s->ys, s->tag_s, s->cfg.box[1], nbins, mobile ? 1 : 0,
                                                    s->prof_part);
    k_profile_final<<<(2 * nbins + 127) / 128, 128, 0, s->stream>>>(s->prof_part, PROF_BLOCKS, nbins,
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
    k_reduce_final<<<1, 32, 0, s->stream>>>(s->red_part, nb, s->red_out);
    MSM_COUNT(s, 2);
    return cudaGetLastError();
}
