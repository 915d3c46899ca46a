// Diagnostics of libmsm: per-class kernel accounting with CUDA events, and a
// device evaluation of the Philox4x32-10 blocks the pair noise uses, next to
// cuRAND's generator for cross-checking.
#include <curand_kernel.h>


#include "msm_internal.cuh"

namespace {

cudaEvent_t take_event(md_system *s)
{
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

__global__ void k_philox_own(int64_t n, const uint4 *ctr, uint2 key, uint4 *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = philox4x32_10(ctr[k], key);
}

__global__ void k_philox_curand(int64_t n, const uint4 *ctr, unsigned long long seed, uint4 *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint4 c = ctr[k];
    const unsigned long long subseq = (unsigned long long)c.z | ((unsigned long long)c.w << 32);
    const unsigned long long offset = 4ull * ((unsigned long long)c.x | ((unsigned long long)c.y << 32));
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq, offset, &st);
    out[k] = curand4(&st);
}

}  // namespace

void prof_begin(md_system *s, int cls)
{
    s->prof_cls = cls;
    s->prof_mark = s->nlaunch;
    if (s->prof_on) {
        s->prof_a = take_event(s);
        if (s->prof_a) cudaEventRecord(s->prof_a, s->stream);
    }
}

void prof_end(md_system *s)
{
    const int cls = s->prof_cls;
    if (cls < 0) return;
    s->cls_launch[cls] += s->nlaunch - s->prof_mark;
    if (s->prof_on && s->prof_a) {
        cudaEvent_t b = take_event(s);
        if (b) {
            cudaEventRecord(b, s->stream);
            s->prof_pending.push_back({cls, s->prof_a, b});
        } else {
            s->ev_pool.push_back(s->prof_a);
        }
    }
    s->prof_a = nullptr;
    s->prof_cls = -1;
}

// Staging buffers of md_philox_static: counters in [0, MAX), outputs in
// [MAX, 2 MAX).  Keeps the last call's contents; calls on one device share it.
static __device__ __align__(256) uint4 philox_scratch[2 * MD_PHILOX_STATIC_MAX];

extern "C" {

int md_profile_enable(md_system *s, int enable)
{
    if (!s) return MD_EINVAL;
    s->prof_on = enable != 0;
    return MD_OK;
}

int md_profile_read(md_system *s, md_profile_t *out, int reset)
{
    if (!s || !out) return MD_EINVAL;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "profile sync");
    for (auto &r : s->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) s->cls_ms[r.cls] += ms;
        s->ev_pool.push_back(r.a);
        s->ev_pool.push_back(r.b);
    }
    s->prof_pending.clear();
    for (int c = 0; c < MD_PROF_CLASSES; ++c) {
        out->launches[c] = s->cls_launch[c];
        out->ms[c] = s->cls_ms[c];
    }
    out->total_launches = s->nlaunch;
    if (reset) {
        for (int c = 0; c < MD_PROF_CLASSES; ++c) { s->cls_launch[c] = 0; s->cls_ms[c] = 0.0; }
        s->nlaunch = 0;
    }
    return MD_OK;
}

int md_philox(const uint32_t *ctr, const uint32_t key[2], int64_t n, uint32_t *out, int use_library)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return MD_EINVAL;
    if (n == 0) return MD_OK;
    if (use_library)
        for (int64_t k = 0; k < n; ++k)
            if (ctr[4 * k + 1] >= (1u << 30)) return MD_EINVAL;  // 4*counter must fit the 64-bit offset
    uint4 *d_ctr = nullptr, *d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_ctr, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_ctr, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n + 255) / 256);
        if (use_library)
            k_philox_curand<<<blocks, 256>>>(n, d_ctr, (unsigned long long)key[0] | ((unsigned long long)key[1] << 32),
                                             d_out);
        else
            k_philox_own<<<blocks, 256>>>(n, d_ctr, make_uint2(key[0], key[1]), d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    if (d_ctr) cudaFree(d_ctr);
    if (d_out) cudaFree(d_out);
    return e == cudaSuccess ? MD_OK : MD_ECUDA;
}

int md_philox_static(const uint32_t *ctr, const uint32_t key[2], int64_t n, uint32_t *out, int use_library)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return MD_EINVAL;
    if (n > MD_PHILOX_STATIC_MAX) return MD_ETOOLARGE;
    if (n == 0) return MD_OK;
    if (use_library)
        for (int64_t k = 0; k < n; ++k)
            if (ctr[4 * k + 1] >= (1u << 30)) return MD_EINVAL;  // 4*counter must fit the 64-bit offset
    // the array's address in the current context, looked up on every call
    // (no allocation; a context rebuilt after a device reset has its own)
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, philox_scratch);
    if (e != cudaSuccess) return MD_ECUDA;
    uint4 *d_ctr = (uint4 *)p, *d_out = (uint4 *)p + MD_PHILOX_STATIC_MAX;
    e = cudaMemcpy(d_ctr, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n + 255) / 256);
        if (use_library)
            k_philox_curand<<<blocks, 256>>>(n, d_ctr, (unsigned long long)key[0] | ((unsigned long long)key[1] << 32),
                                             d_out);
        else
            k_philox_own<<<blocks, 256>>>(n, d_ctr, make_uint2(key[0], key[1]), d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MD_OK : MD_ECUDA;
}

}  // extern "C"
