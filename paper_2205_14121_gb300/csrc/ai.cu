// K9/K10: the learned step-size controller of Table 2 (Sec. 3.3) on the GPU.
//
//   raw [B][T][F] -> moving average + one-level Haar soft-threshold denoise
//   -> per-feature normalisation -> GRU encoder (2 layers, hidden H)
//   -> latent (linear) -> GRU decoder (2 layers) fed the repeated latent
//   -> reconstruction (linear); FCN heads on the latent -> k-class logits and
//   log hold.  Training: reconstruction MSE for the autoencoder, softmax
//   cross-entropy + MSE(log hold) for the heads (trained separately), BPTT,
//   Adam.
//
// Every matrix product runs on the tensor cores: BF16 operands (rounded from
// the FP32 master values when staged in shared memory), FP32 accumulation,
// mma.sync.m16n8k16.  The GRU recurrences keep one CTA per 16 batch rows for
// all T steps (no inter-CTA dependence); the input projections and weight
// gradients are batched GEMMs over all time steps.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "msm_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// BF16 tensor-core helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of a 16x16 tile stored row-major (ld in bf16 elements).
__device__ __forceinline__ void load_a(uint32_t a[4], const __nv_bfloat16 *s, int ld, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const uint32_t *p0 = reinterpret_cast<const uint32_t *>(s + g * ld + 2 * t);
    const uint32_t *p1 = reinterpret_cast<const uint32_t *>(s + (g + 8) * ld + 2 * t);
    a[0] = p0[0];
    a[1] = p1[0];
    a[2] = p0[4];
    a[3] = p1[4];
}

// B fragment of a 16(k) x 8(n) tile stored as [n][k] (k contiguous).
__device__ __forceinline__ void load_b(uint32_t b[2], const __nv_bfloat16 *s, int ld, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const uint32_t *p = reinterpret_cast<const uint32_t *>(s + g * ld + 2 * t);
    b[0] = p[0];
    b[1] = p[4];
}

// ---------------------------------------------------------------------------
// GEMM: C[M,N] (+)= alpha * opA(A)[M,K] opB(B)[K,N] (+ bias[N])
//   opA(A)[m,k] = A[m*lam + k*lak], opB(B)[k,n] = B[k*lbk + n*lbn]
// 64x64 CTA tiles, 4 warps of 32x32, K in steps of 16, split-K over
// gridDim.z with FP32 atomics when split > 1.
// ---------------------------------------------------------------------------
struct gemm_args {
    int M, N, K;
    const float *A;
    int64_t lam, lak;
    const float *B;
    int64_t lbk, lbn;
    float *C;
    int64_t ldc;
    const float *bias;     // added once (by split 0) when non-null
    float alpha;
    int accumulate;        // 1: C += ..., 0: C = ...
    int atomic;            // split-K accumulation
};

constexpr int GT = 64, GK = 16, GPAD = 8;

__global__ void __launch_bounds__(128) k_gemm(gemm_args g)
{
    __shared__ __align__(16) __nv_bfloat16 As[GT][GK + GPAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[GT][GK + GPAD];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int ksplit = gridDim.z;
    const int kchunk = ((g.K + ksplit - 1) / ksplit + GK - 1) / GK * GK;
    const int kb = blockIdx.z * kchunk, ke = min(g.K, kb + kchunk);
    float acc[2][4][4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += GK) {
        // stage A (64 x 16) and B (16 x 64 as [n][k]) as BF16
        for (int e = threadIdx.x; e < GT * GK; e += 128) {
            const int mm = e / GK, kk = e % GK;
            const int gm = m0 + mm, gk = k0 + kk;
            const float va = (gm < g.M && gk < ke) ? g.A[gm * g.lam + gk * g.lak] : 0.f;
            As[mm][kk] = __float2bfloat16_rn(va);
            const int nn = e / GK;
            const int gn = n0 + nn;
            const float vb = (gn < g.N && gk < ke) ? g.B[gk * g.lbk + gn * g.lbn] : 0.f;
            Bs[nn][kk] = __float2bfloat16_rn(vb);
        }
        __syncthreads();
        uint32_t af[2][4], bf[4][2];
        for (int i = 0; i < 2; ++i) load_a(af[i], &As[wm + 16 * i][0], GK + GPAD, lane);
        for (int j = 0; j < 4; ++j) load_b(bf[j], &Bs[wn + 8 * j][0], GK + GPAD, lane);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        __syncthreads();
    }
    const int gq = lane >> 2, tq = lane & 3;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + 16 * i + gq + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * tq + (q & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = g.alpha * acc[i][j][q];
                if (g.bias && blockIdx.z == 0) v += g.bias[n];
                float *c = g.C + m * g.ldc + n;
                if (g.atomic) atomicAdd(c, v);
                else *c = g.accumulate ? *c + v : v;
            }
}

// ---------------------------------------------------------------------------
// GRU recurrences (hidden size 64, gates r, z, n stacked along 3H = 192)
// ---------------------------------------------------------------------------
constexpr int GH = 64, G3 = 192, GR = 16;   // hidden, 3*hidden, batch rows per CTA

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

struct gru_fwd_args {
    int T, B;
    const float *Gi;        // [T][B][3H] input projections incl. b_ih (t-stride 0: time-invariant)
    int64_t gi_tstride;
    const float *Whh;       // [3H][H]
    const float *bhh;       // [3H]
    float *Hs;              // [T][B][H] hidden states
    float *cache;           // [4][T][B][H]: r, z, n, W_hn h + b_hn (null: inference)
};

__global__ void __launch_bounds__(128) k_gru_fwd(gru_fwd_args a)
{
    __shared__ __align__(16) __nv_bfloat16 Ws[G3][GH + GPAD];   // B operand [n=3H][k=H]
    __shared__ __align__(16) __nv_bfloat16 hb[GR][GH + GPAD];   // A operand
    __shared__ float hs[GR][GH];
    __shared__ float gh[GR][G3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b0 = blockIdx.x * GR;
    for (int e = threadIdx.x; e < G3 * GH; e += 128) Ws[e / GH][e % GH] = __float2bfloat16_rn(a.Whh[e]);
    for (int e = threadIdx.x; e < GR * GH; e += 128) {
        hs[e / GH][e % GH] = 0.f;
        hb[e / GH][e % GH] = __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    const int64_t TBH = (int64_t)a.T * a.B * GH;
    for (int t = 0; t < a.T; ++t) {
        // gh = h W_hh^T: warp w covers gate columns [48w, 48w+48)
        float acc[6][4];
        for (int j = 0; j < 6; ++j)
            for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
        for (int k0 = 0; k0 < GH; k0 += 16) {
            uint32_t af[4];
            load_a(af, &hb[0][k0], GH + GPAD, lane);
            for (int j = 0; j < 6; ++j) {
                uint32_t bf[2];
                load_b(bf, &Ws[48 * warp + 8 * j][k0], GH + GPAD, lane);
                mma_bf16(acc[j], af, bf);
            }
        }
        const int gq = lane >> 2, tq = lane & 3;
        for (int j = 0; j < 6; ++j)
            for (int q = 0; q < 4; ++q) gh[gq + (q >= 2 ? 8 : 0)][48 * warp + 8 * j + 2 * tq + (q & 1)] = acc[j][q];
        __syncthreads();
        for (int e = threadIdx.x; e < GR * GH; e += 128) {
            const int rr = e / GH, u = e % GH;
            const int b = b0 + rr;
            if (b >= a.B) continue;
            const float *gi = a.Gi + t * a.gi_tstride + (int64_t)b * G3;
            const float ghr = gh[rr][u] + a.bhh[u];
            const float ghz = gh[rr][GH + u] + a.bhh[GH + u];
            const float ghn = gh[rr][2 * GH + u] + a.bhh[2 * GH + u];
            const float r = sigm(gi[u] + ghr);
            const float z = sigm(gi[GH + u] + ghz);
            const float n = tanhf(gi[2 * GH + u] + r * ghn);
            const float hp = hs[rr][u];
            const float h = (1.0f - z) * n + z * hp;
            hs[rr][u] = h;
            hb[rr][u] = __float2bfloat16_rn(h);
            const int64_t o = ((int64_t)t * a.B + b) * GH + u;
            a.Hs[o] = h;
            if (a.cache) {
                a.cache[o] = r;
                a.cache[TBH + o] = z;
                a.cache[2 * TBH + o] = n;
                a.cache[3 * TBH + o] = ghn;
            }
        }
        __syncthreads();
    }
}

struct gru_bwd_args {
    int T, B;
    const float *dHs;       // [T][B][H] gradient from above, or null
    const float *dh_last;   // [B][H] gradient on h_{T-1}, or null
    const float *Hs;        // forward hidden states [T][B][H]
    const float *cache;     // [4][T][B][H]
    const float *Whh;       // [3H][H]
    float *dGi, *dGh;       // [T][B][3H]
};

__global__ void __launch_bounds__(128) k_gru_bwd(gru_bwd_args a)
{
    __shared__ __align__(16) __nv_bfloat16 Ws[GH][G3 + GPAD];   // B operand [n=H][k=3H] = W_hh^T
    __shared__ __align__(16) __nv_bfloat16 gb[GR][G3 + GPAD];   // A operand: dgh
    __shared__ float dh[GR][GH];
    __shared__ float dd[GR][GH];                                 // dh * z (direct path)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b0 = blockIdx.x * GR;
    for (int e = threadIdx.x; e < G3 * GH; e += 128) {
        const int gg = e / GH, u = e % GH;
        Ws[u][gg] = __float2bfloat16_rn(a.Whh[e]);
    }
    for (int e = threadIdx.x; e < GR * GH; e += 128) {
        const int rr = e / GH, u = e % GH;
        const int b = b0 + rr;
        dh[rr][u] = (a.dh_last && b < a.B) ? a.dh_last[(int64_t)b * GH + u] : 0.f;
    }
    __syncthreads();
    const int64_t TBH = (int64_t)a.T * a.B * GH;
    for (int t = a.T - 1; t >= 0; --t) {
        for (int e = threadIdx.x; e < GR * GH; e += 128) {
            const int rr = e / GH, u = e % GH;
            const int b = b0 + rr;
            float dgr = 0.f, dgz = 0.f, dgn = 0.f, dghn = 0.f, direct = 0.f;
            if (b < a.B) {
                const int64_t o = ((int64_t)t * a.B + b) * GH + u;
                float d = dh[rr][u] + (a.dHs ? a.dHs[o] : 0.f);
                const float r = a.cache[o], z = a.cache[TBH + o], n = a.cache[2 * TBH + o];
                const float ghn = a.cache[3 * TBH + o];
                const float hp = t > 0 ? a.Hs[o - (int64_t)a.B * GH] : 0.f;
                const float dn = d * (1.0f - z);
                const float dz = d * (hp - n);
                direct = d * z;
                const float dan = dn * (1.0f - n * n);
                const float dr = dan * ghn;
                dghn = dan * r;
                dgz = dz * z * (1.0f - z);
                dgr = dr * r * (1.0f - r);
                dgn = dan;
                float *gi = a.dGi + ((int64_t)t * a.B + b) * G3;
                float *gh = a.dGh + ((int64_t)t * a.B + b) * G3;
                gi[u] = dgr; gi[GH + u] = dgz; gi[2 * GH + u] = dgn;
                gh[u] = dgr; gh[GH + u] = dgz; gh[2 * GH + u] = dghn;
            }
            gb[rr][u] = __float2bfloat16_rn(dgr);
            gb[rr][GH + u] = __float2bfloat16_rn(dgz);
            gb[rr][2 * GH + u] = __float2bfloat16_rn(dghn);
            dd[rr][u] = direct;
        }
        __syncthreads();
        // dh_prev = dd + dgh W_hh: warp w covers hidden columns [16w, 16w+16)
        float acc[2][4];
        for (int j = 0; j < 2; ++j)
            for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
        for (int k0 = 0; k0 < G3; k0 += 16) {
            uint32_t af[4];
            load_a(af, &gb[0][k0], G3 + GPAD, lane);
            for (int j = 0; j < 2; ++j) {
                uint32_t bf[2];
                load_b(bf, &Ws[16 * warp + 8 * j][k0], G3 + GPAD, lane);
                mma_bf16(acc[j], af, bf);
            }
        }
        const int gq = lane >> 2, tq = lane & 3;
        for (int j = 0; j < 2; ++j)
            for (int q = 0; q < 4; ++q) {
                const int rr = gq + (q >= 2 ? 8 : 0), u = 16 * warp + 8 * j + 2 * tq + (q & 1);
                dh[rr][u] = dd[rr][u] + acc[j][q];
            }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// elementwise and reduction kernels
// ---------------------------------------------------------------------------
// Table 2 step 2 per (row, feature) thread: causal moving average (w = 5),
// one-level Haar transform, soft threshold lambda = median|d|/0.6745 *
// sqrt(2 ln T), inverse; then (x - mean) / std.  Writes time-major [T][B][F].
__global__ void k_denoise(const float *raw, int B, int T, int F, const float *mean, const float *stdv, float *out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B * F) return;
    const int b = q / F, c = q % F;
    float x[256];
    float d[128];
    const int Tn = T > 256 ? 256 : T;
    float run = 0.f;
    for (int t = 0; t < Tn; ++t) {
        const float v = raw[((int64_t)b * T + t) * F + c];
        run += v;
        if (t >= 5) run -= raw[((int64_t)b * T + t - 5) * F + c];
        x[t] = run / (float)(t + 1 < 5 ? t + 1 : 5);
    }
    const int h = Tn / 2;
    const float s2 = 0.70710678f;
    for (int k = 0; k < h; ++k) d[k] = fabsf((x[2 * k] - x[2 * k + 1]) * s2);
    // median of |d| (insertion sort of h values)
    for (int i = 1; i < h; ++i) {
        const float key = d[i];
        int j = i - 1;
        while (j >= 0 && d[j] > key) { d[j + 1] = d[j]; --j; }
        d[j + 1] = key;
    }
    const float med = (h % 2) ? d[h / 2] : 0.5f * (d[h / 2 - 1] + d[h / 2]);
    const float lam = med / 0.6745f * sqrtf(2.0f * logf((float)Tn));
    const float mu = mean ? mean[c] : 0.f, sd = stdv ? stdv[c] : 1.f;
    for (int k = 0; k < h; ++k) {
        const float av = (x[2 * k] + x[2 * k + 1]) * s2;
        float dv = (x[2 * k] - x[2 * k + 1]) * s2;
        const float m = fabsf(dv) - lam;
        dv = m > 0.f ? copysignf(m, dv) : 0.f;
        out[((int64_t)(2 * k) * B + b) * F + c] = ((av + dv) * s2 - mu) / sd;
        out[((int64_t)(2 * k + 1) * B + b) * F + c] = ((av - dv) * s2 - mu) / sd;
    }
}

// [B][T][F] -> [T][B][F]
__global__ void k_to_time_major(const float *x, int B, int T, int F, float *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)B * T * F) return;
    const int c = q % F, t = (q / F) % T, b = q / ((int64_t)F * T);
    out[((int64_t)t * B + b) * F + c] = x[q];
}

// mean squared reconstruction error: loss (atomic) and dY = 2 (Y - X) / count;
// per-row error (mean over T, F) into rec[B].
__global__ void k_mse(const float *Y, const float *X, int B, int T, int F, float *dY, float *loss, float *rec)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = (int64_t)B * T * F;
    float e2 = 0.f;
    if (q < cnt) {
        const float e = Y[q] - X[q];
        e2 = e * e;
        if (dY) dY[q] = 2.0f * e / (float)cnt;
        if (rec) atomicAdd(&rec[(q / F) % B], e2 / (float)(T * F));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, e2 / (float)cnt);
}

__global__ void k_relu(float *x, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) x[q] = fmaxf(x[q], 0.f);
}

__global__ void k_relu_bwd(float *d, const float *act, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n && act[q] <= 0.f) d[q] = 0.f;
}

// softmax cross-entropy over C classes + MSE of the log hold; gradients / B.
__global__ void k_heads_loss(const float *logits, int C, const float *lh, const int32_t *cls, const float *lh_t,
                             int B, float w_hold, float *dlogits, float *dlh, float *loss, float *probs)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float *z = logits + (int64_t)b * C;
    float mx = z[0];
    for (int c = 1; c < C; ++c) mx = fmaxf(mx, z[c]);
    float se = 0.f;
    for (int c = 0; c < C; ++c) se += __expf(z[c] - mx);
    float l = 0.f;
    for (int c = 0; c < C; ++c) {
        const float p = __expf(z[c] - mx) / se;
        if (probs) probs[(int64_t)b * C + c] = p;
        if (cls) {
            if (c == cls[b]) l -= logf(fmaxf(p, 1e-30f));
            if (dlogits) dlogits[(int64_t)b * C + c] = (p - (c == cls[b] ? 1.f : 0.f)) / B;
        }
    }
    if (lh_t) {
        const float e = lh[b] - lh_t[b];
        l += w_hold * e * e;
        if (dlh) dlh[b] = w_hold * 2.f * e / B;
    }
    if (loss) atomicAdd(loss, l / B);
}

// column sums: out[n] (+)= sum_m A[m*lda + n], split over rows with atomics
__global__ void k_colsum(const float *A, int M, int N, int64_t lda, float *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int chunk = (M + gridDim.y - 1) / gridDim.y;
    const int m0 = blockIdx.y * chunk, m1 = min(M, m0 + chunk);
    float s = 0.f;
    for (int m = m0; m < m1; ++m) s += A[(int64_t)m * lda + n];
    atomicAdd(&out[n], s);
}

// sum over time: out[b][j] = sum_t X[t][b][j]
__global__ void k_sum_time(const float *X, int T, int64_t BJ, float *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= BJ) return;
    float s = 0.f;
    for (int t = 0; t < T; ++t) s += X[t * BJ + q];
    out[q] = s;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

// Table 2 steps 5-6 for window b: the most probable class and its ratio,
// the trust bound (top probability, reconstruction error, largest bond strain
// of the raw window), the fallback ratio for a window that fails it, and the
// hold length exp(log hold) clipped to its range.  A NaN fails every test.
// Largest value of column col of each raw window [B][T][F] (NaN if any is NaN).
__global__ void k_window_max(const float *raw, int B, int T, int F, int col, float *out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float *w = raw + (int64_t)b * T * F + col;
    float m = -INFINITY;
    bool nan = false;
    for (int t = 0; t < T; ++t) {
        const float v = w[(int64_t)t * F];
        nan |= v != v;
        m = fmaxf(m, v);
    }
    out[b] = nan ? NAN : m;
}

struct decide_args {
    const float *probs, *lh, *rec, *smax;   // smax: per-window strain maximum (k_window_max)
    int B, C, T, F;
    float p_min, rec_max, strain_max, hold_min, hold_max;
    int strain_col, fallback_k;
    int kv[8];                             // step ratio of each class
    int32_t *out;                          // [3][B]: k, hold, reason bits
};

__global__ void k_decide(decide_args a)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    const float *pr = a.probs + (int64_t)b * a.C;
    int best = 0;
    float pmax = pr[0];
    for (int c = 1; c < a.C; ++c)
        if (pr[c] > pmax) { pmax = pr[c]; best = c; }
    int why = 0;
    if (!(pmax >= a.p_min)) why |= MD_AI_UNSURE_PROB;
    if (!(a.rec[b] <= a.rec_max)) why |= MD_AI_UNSURE_REC;
    if (a.strain_col >= 0 && !(a.smax[b] <= a.strain_max)) why |= MD_AI_UNSURE_STRAIN;
    float h = expf(a.lh[b]);
    h = h != h ? a.hold_min : fminf(fmaxf(h, a.hold_min), a.hold_max);
    a.out[b] = why ? a.fallback_k : a.kv[best];
    a.out[a.B + b] = (int32_t)h;
    a.out[2 * a.B + b] = why;
}

// The last T records of every platelet from the system's feature ring, in
// time order, as raw windows [P][T][F] (the ring holds [P][T][F] with record
// r at slot r mod T).
__global__ void k_gather_ring(const float *ring, const md_dstate *ds, int P, int T, int F, float *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)P * T * F) return;
    const int f = (int)(q % F);
    const int t = (int)((q / F) % T);
    const int64_t p = q / ((int64_t)F * T);
    const int64_t count = ds->ring_count;
    const int64_t slot = ((count - T + t) % T + T) % T;
    out[q] = ring[(p * T + slot) * F + f];
}

unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

}  // namespace

// Table 2 step 2 and Adam for the other controller variant (lstm.cu)
cudaError_t ai_launch_denoise(const float *raw, int B, int T, int F, const float *mean, const float *stdv, float *out,
                              cudaStream_t st)
{
    k_denoise<<<nblk((int64_t)B * F, 128), 128, 0, st>>>(raw, B, T, F, mean, stdv, out);
    return cudaGetLastError();
}

cudaError_t ai_launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, int64_t t,
                           cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<nblk(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

// ===========================================================================
// controller object
// ===========================================================================
struct md_ai {
    md_ai_config c;
    cudaStream_t st;
    std::string err;
    int64_t nparam;
    // offsets of the parameter blocks in the flat vector
    struct gru_off { int64_t Wih, Whh, bih, bhh; };
    gru_off enc1, enc2, dec1, dec2;
    int64_t latW, latb, outW, outb;
    int64_t kh[4][2], lh_[4][2];   // W, b of each head layer
    int hd[5];                     // head dims: latent, h0, h1, h2, (C or 1)
    // device buffers (carved from the caller's workspace)
    float *P, *G, *Am, *Av;        // params, grads, Adam moments
    float *mean, *stdv;
    float *X, *Y, *dY;             // [T][B][F]
    float *Gi, *dGi, *dGh;         // [T][B][3H]
    float *H1, *H2, *D1, *D2;      // [T][B][H]
    float *C1, *C2, *C3, *C4;      // caches [4][T][B][H]
    float *dA, *dB2;               // [T][B][H] scratch gradients
    float *Z, *dZ, *GiZ, *dGiZ;    // latent [B][L], its gradient, latent input projection [B][3H] and its grad
    float *hact[2][4];             // head activations (layer inputs) [B][max width]
    float *hgrad[2];               // [B][max width] x2 scratch
    float *logits, *lh, *probs, *dlog, *dlh, *rec, *loss, *tmp;
    int32_t *cls;
    float *lht;
    int32_t *dec;                  // [3][B] decisions: k, hold, reason bits
    float *smax;                   // [B] per-window maximum of the strain column
    cudaEvent_t ring_ready = nullptr;
    int64_t adam_t = 0, adam_t_heads = 0;
    bool has_params = false, has_norm = false;
};

namespace {

void plan_ai(md_ai &m, char *base, size_t &off)
{
    auto take = [&](int64_t n) -> float * {
        off = (off + 255) & ~(size_t)255;
        float *p = base ? reinterpret_cast<float *>(base + off) : nullptr;
        off += sizeof(float) * (size_t)(n > 0 ? n : 1);
        return p;
    };
    const md_ai_config &c = m.c;
    const int64_t H = GH, H3 = G3, F = c.F, L = c.latent, T = c.T, B = c.batch_max;
    int64_t o = 0;
    auto gru = [&](int64_t nin) {
        md_ai::gru_off g;
        g.Wih = o; o += H3 * nin;
        g.Whh = o; o += H3 * H;
        g.bih = o; o += H3;
        g.bhh = o; o += H3;
        return g;
    };
    m.enc1 = gru(F);
    m.enc2 = gru(H);
    m.latW = o; o += L * H;
    m.latb = o; o += L;
    m.dec1 = gru(L);
    m.dec2 = gru(H);
    m.outW = o; o += F * H;
    m.outb = o; o += F;
    m.hd[0] = (int)L; m.hd[1] = c.head_hidden[0]; m.hd[2] = c.head_hidden[1]; m.hd[3] = c.head_hidden[2];
    for (int head = 0; head < 2; ++head) {
        const int last = head == 0 ? c.n_classes : 1;
        for (int l = 0; l < 4; ++l) {
            const int nin = m.hd[l], nout = l == 3 ? last : m.hd[l + 1];
            int64_t(*dst)[2] = head == 0 ? m.kh : m.lh_;
            dst[l][0] = o; o += (int64_t)nout * nin;
            dst[l][1] = o; o += nout;
        }
    }
    m.nparam = o;
    m.P = take(o); m.G = take(o); m.Am = take(o); m.Av = take(o);
    m.mean = take(F); m.stdv = take(F);
    m.X = take(T * B * F); m.Y = take(T * B * F); m.dY = take(T * B * F);
    m.Gi = take(T * B * H3); m.dGi = take(T * B * H3); m.dGh = take(T * B * H3);
    m.H1 = take(T * B * H); m.H2 = take(T * B * H); m.D1 = take(T * B * H); m.D2 = take(T * B * H);
    m.C1 = take(4 * T * B * H); m.C2 = take(4 * T * B * H); m.C3 = take(4 * T * B * H); m.C4 = take(4 * T * B * H);
    m.dA = take(T * B * H); m.dB2 = take(T * B * H);
    m.Z = take(B * L); m.dZ = take(B * L); m.GiZ = take(B * H3); m.dGiZ = take(B * H3);
    int wmax = c.n_classes;
    for (int l = 0; l < 4; ++l) wmax = wmax > m.hd[l] ? wmax : m.hd[l];
    for (int h = 0; h < 2; ++h) {
        for (int l = 0; l < 4; ++l) m.hact[h][l] = take(B * wmax);
        m.hgrad[h] = take(B * wmax);
    }
    m.logits = take(B * c.n_classes); m.lh = take(B); m.probs = take(B * c.n_classes);
    m.dlog = take(B * c.n_classes); m.dlh = take(B); m.rec = take(B); m.loss = take(4); m.tmp = take(B * H3);
    m.cls = reinterpret_cast<int32_t *>(take(B));
    m.lht = take(B);
    m.dec = reinterpret_cast<int32_t *>(take(3 * B));
    m.smax = take(B);
}

int ai_fail(md_ai *m, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return MD_OK;
    m->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    return MD_ECUDA;
}

#define AK(expr, where)                                  \
    do {                                                 \
        int _rc = ai_fail(m, (expr), where);             \
        if (_rc) return _rc;                             \
    } while (0)

// C[M,N] (+)= opA(A) opB(B) (+ bias); split-K for long reductions
cudaError_t gemm(md_ai *m, int M, int N, int K, const float *A, int64_t lam, int64_t lak, const float *B, int64_t lbk,
                 int64_t lbn, float *C, int64_t ldc, const float *bias, bool accumulate)
{
    gemm_args g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lam = lam; g.lak = lak;
    g.B = B; g.lbk = lbk; g.lbn = lbn;
    g.C = C; g.ldc = ldc;
    g.bias = bias;
    g.alpha = 1.f;
    g.accumulate = accumulate ? 1 : 0;
    const int tiles = ((M + GT - 1) / GT) * ((N + GT - 1) / GT);
    int split = 1;
    if (K > 4 * GK && tiles < 152) {
        split = (152 * 2) / tiles;
        const int maxs = (K + 255) / 256;
        if (split > maxs) split = maxs;
        if (split < 1) split = 1;
    }
    g.atomic = split > 1 ? 1 : 0;
    if (split > 1 && !accumulate) {   // split-K partials accumulate atomically into a zeroed C
        cudaError_t e = cudaMemset2DAsync(C, sizeof(float) * ldc, 0, sizeof(float) * N, M, m->st);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, split);
    k_gemm<<<grid, 128, 0, m->st>>>(g);
    return cudaGetLastError();
}

cudaError_t colsum(md_ai *m, const float *A, int M, int N, int64_t lda, float *out)
{
    dim3 grid((N + 127) / 128, M > 4096 ? 64 : 1);
    k_colsum<<<grid, 128, 0, m->st>>>(A, M, N, lda, out);
    return cudaGetLastError();
}

// GRU layer forward: Gi = X W_ih^T + b_ih for every step, then the recurrence.
int gru_layer_fwd(md_ai *m, const md_ai::gru_off &go, int nin, const float *Xin, bool time_invariant, int B,
                  float *Hout, float *cache)
{
    const int T = m->c.T;
    const int rows = time_invariant ? B : T * B;
    AK(gemm(m, rows, G3, nin, Xin, nin, 1, m->P + go.Wih, 1, nin, m->Gi, G3, m->P + go.bih, false), "gemm Gi");
    gru_fwd_args a;
    a.T = T; a.B = B; a.Gi = m->Gi; a.gi_tstride = time_invariant ? 0 : (int64_t)B * G3;
    a.Whh = m->P + go.Whh; a.bhh = m->P + go.bhh; a.Hs = Hout; a.cache = cache;
    k_gru_fwd<<<(B + GR - 1) / GR, 128, 0, m->st>>>(a);
    AK(cudaGetLastError(), "gru fwd");
    return MD_OK;
}

// GRU layer backward: recurrence, then weight gradients and (optional) dX.
int gru_layer_bwd(md_ai *m, const md_ai::gru_off &go, int nin, const float *Xin, bool time_invariant, int B,
                  const float *Hs, const float *cache, const float *dHs, const float *dh_last, float *dX)
{
    const int T = m->c.T;
    gru_bwd_args a;
    a.T = T; a.B = B; a.dHs = dHs; a.dh_last = dh_last; a.Hs = Hs; a.cache = cache; a.Whh = m->P + go.Whh;
    a.dGi = m->dGi; a.dGh = m->dGh;
    k_gru_bwd<<<(B + GR - 1) / GR, 128, 0, m->st>>>(a);
    AK(cudaGetLastError(), "gru bwd");
    const int TB = T * B;
    // dW_hh = sum_{t>=1} dGh[t]^T H[t-1]
    if (T > 1)
        AK(gemm(m, G3, GH, (T - 1) * B, m->dGh + (int64_t)B * G3, 1, G3, Hs, GH, 1, m->G + go.Whh, GH, nullptr, true),
           "gemm dWhh");
    AK(colsum(m, m->dGh, TB, G3, G3, m->G + go.bhh), "db_hh");
    AK(colsum(m, m->dGi, TB, G3, G3, m->G + go.bih), "db_ih");
    if (time_invariant) {
        // the input is the same every step: reduce dGi over time first
        k_sum_time<<<nblk((int64_t)B * G3), 256, 0, m->st>>>(m->dGi, T, (int64_t)B * G3, m->dGiZ);
        AK(cudaGetLastError(), "sum time");
        AK(gemm(m, G3, nin, B, m->dGiZ, 1, G3, Xin, nin, 1, m->G + go.Wih, nin, nullptr, true), "gemm dWih");
        if (dX) AK(gemm(m, B, nin, G3, m->dGiZ, G3, 1, m->P + go.Wih, nin, 1, dX, nin, nullptr, false), "gemm dX");
    } else {
        AK(gemm(m, G3, nin, TB, m->dGi, 1, G3, Xin, nin, 1, m->G + go.Wih, nin, nullptr, true), "gemm dWih");
        if (dX) AK(gemm(m, TB, nin, G3, m->dGi, G3, 1, m->P + go.Wih, nin, 1, dX, nin, nullptr, false), "gemm dX");
    }
    return MD_OK;
}

// autoencoder forward on m->X (time-major, normalised): Z, Y, per-row error
int ae_forward(md_ai *m, int B, bool train)
{
    const int T = m->c.T, F = m->c.F, L = m->c.latent;
    if (gru_layer_fwd(m, m->enc1, F, m->X, false, B, m->H1, train ? m->C1 : nullptr)) return MD_ECUDA;
    if (gru_layer_fwd(m, m->enc2, GH, m->H1, false, B, m->H2, train ? m->C2 : nullptr)) return MD_ECUDA;
    AK(gemm(m, B, L, GH, m->H2 + (int64_t)(T - 1) * B * GH, GH, 1, m->P + m->latW, 1, GH, m->Z, L, m->P + m->latb,
            false), "gemm latent");
    if (gru_layer_fwd(m, m->dec1, L, m->Z, true, B, m->D1, train ? m->C3 : nullptr)) return MD_ECUDA;
    if (gru_layer_fwd(m, m->dec2, GH, m->D1, false, B, m->D2, train ? m->C4 : nullptr)) return MD_ECUDA;
    AK(gemm(m, T * B, F, GH, m->D2, GH, 1, m->P + m->outW, 1, GH, m->Y, F, m->P + m->outb, false), "gemm out");
    AK(cudaMemsetAsync(m->loss, 0, 4 * sizeof(float), m->st), "zero loss");
    AK(cudaMemsetAsync(m->rec, 0, B * sizeof(float), m->st), "zero rec");
    const int64_t cnt = (int64_t)T * B * F;
    k_mse<<<nblk(cnt), 256, 0, m->st>>>(m->Y, m->X, B, T, F, train ? m->dY : nullptr, m->loss, m->rec);
    AK(cudaGetLastError(), "mse");
    return MD_OK;
}

int ae_backward(md_ai *m, int B)
{
    const int T = m->c.T, F = m->c.F, L = m->c.latent, TB = T * B;
    AK(gemm(m, F, GH, TB, m->dY, 1, F, m->D2, GH, 1, m->G + m->outW, GH, nullptr, true), "gemm dWout");
    AK(colsum(m, m->dY, TB, F, F, m->G + m->outb), "db out");
    AK(gemm(m, TB, GH, F, m->dY, F, 1, m->P + m->outW, GH, 1, m->dA, GH, nullptr, false), "gemm dD2");
    if (gru_layer_bwd(m, m->dec2, GH, m->D1, false, B, m->D2, m->C4, m->dA, nullptr, m->dB2)) return MD_ECUDA;
    if (gru_layer_bwd(m, m->dec1, L, m->Z, true, B, m->D1, m->C3, m->dB2, nullptr, m->dZ)) return MD_ECUDA;
    AK(gemm(m, L, GH, B, m->dZ, 1, L, m->H2 + (int64_t)(T - 1) * B * GH, GH, 1, m->G + m->latW, GH, nullptr, true),
       "gemm dWlat");
    AK(colsum(m, m->dZ, B, L, L, m->G + m->latb), "db lat");
    // dh on the last encoder state only
    AK(gemm(m, B, GH, L, m->dZ, L, 1, m->P + m->latW, GH, 1, m->tmp, GH, nullptr, false), "gemm dh last");
    if (gru_layer_bwd(m, m->enc2, GH, m->H1, false, B, m->H2, m->C2, nullptr, m->tmp, m->dA)) return MD_ECUDA;
    if (gru_layer_bwd(m, m->enc1, F, m->X, false, B, m->H1, m->C1, m->dA, nullptr, nullptr)) return MD_ECUDA;
    return MD_OK;
}

// heads on m->Z: logits, log hold (and activations for backward)
int heads_forward(md_ai *m, int B)
{
    for (int head = 0; head < 2; ++head) {
        const float *in = m->Z;
        int nin = m->hd[0];
        int64_t(*off)[2] = head == 0 ? m->kh : m->lh_;
        const int last = head == 0 ? m->c.n_classes : 1;
        for (int l = 0; l < 4; ++l) {
            const int nout = l == 3 ? last : m->hd[l + 1];
            float *out = l == 3 ? (head == 0 ? m->logits : m->lh) : m->hact[head][l + 1];
            AK(gemm(m, B, nout, nin, in, nin, 1, m->P + off[l][0], 1, nin, out, nout, m->P + off[l][1], false),
               "gemm head");
            if (l < 3) {
                k_relu<<<nblk((int64_t)B * nout), 256, 0, m->st>>>(out, (int64_t)B * nout);
                AK(cudaGetLastError(), "relu");
            }
            in = out;
            nin = nout;
        }
    }
    return MD_OK;
}

int heads_backward(md_ai *m, int B)
{
    for (int head = 0; head < 2; ++head) {
        int64_t(*off)[2] = head == 0 ? m->kh : m->lh_;
        const int last = head == 0 ? m->c.n_classes : 1;
        float *d = head == 0 ? m->dlog : m->dlh;
        for (int l = 3; l >= 0; --l) {
            const int nin = m->hd[l], nout = l == 3 ? last : m->hd[l + 1];
            const float *in = l == 0 ? m->Z : m->hact[head][l];
            AK(gemm(m, nout, nin, B, d, 1, nout, in, nin, 1, m->G + off[l][0], nin, nullptr, true), "gemm dW head");
            AK(colsum(m, d, B, nout, nout, m->G + off[l][1]), "db head");
            if (l > 0) {
                float *dn = m->hgrad[head];
                float *dst = (d == dn) ? m->tmp : dn;
                AK(gemm(m, B, nin, nout, d, nout, 1, m->P + off[l][0], nin, 1, dst, nin, nullptr, false), "gemm dX head");
                k_relu_bwd<<<nblk((int64_t)B * nin), 256, 0, m->st>>>(dst, m->hact[head][l], (int64_t)B * nin);
                AK(cudaGetLastError(), "relu bwd");
                d = dst;
            }
        }
    }
    return MD_OK;
}

int stage_windows(md_ai *m, const float *x, int B, int where, bool raw)
{
    const int T = m->c.T, F = m->c.F;
    const int64_t cnt = (int64_t)B * T * F;
    const float *src = x;
    if (where == MD_AI_HOST) {
        AK(cudaMemcpyAsync(m->Y, x, sizeof(float) * cnt, cudaMemcpyHostToDevice, m->st), "upload windows");
        src = m->Y;
    }
    if (raw) {
        if (T > 256 || (T & 1)) { m->err = "window length must be even and <= 256"; return MD_EINVAL; }
        k_denoise<<<nblk((int64_t)B * F, 128), 128, 0, m->st>>>(src, B, T, F, m->has_norm ? m->mean : nullptr,
                                                            m->has_norm ? m->stdv : nullptr, m->X);
    } else {
        k_to_time_major<<<nblk(cnt), 256, 0, m->st>>>(src, B, T, F, m->X);
    }
    AK(cudaGetLastError(), "stage windows");
    return MD_OK;
}

}  // namespace

extern "C" {

int md_ai_config_defaults(md_ai_config *c)
{
    if (!c) return MD_EINVAL;
    c->T = 128; c->F = 12; c->hidden = GH; c->latent = 16; c->n_classes = 5;
    c->head_hidden[0] = 32; c->head_hidden[1] = 16; c->head_hidden[2] = 8;
    c->batch_max = 256;
    return MD_OK;
}

int md_ai_param_count(const md_ai_config *c, int64_t *n)
{
    if (!c || !n || c->hidden != GH) return MD_EINVAL;
    md_ai m;
    m.c = *c;
    size_t off = 0;
    plan_ai(m, nullptr, off);
    *n = m.nparam;
    return MD_OK;
}

int md_ai_workspace_size(const md_ai_config *c, size_t *bytes)
{
    if (!c || !bytes || c->hidden != GH || c->T < 2 || c->F < 1 || c->latent < 1 || c->batch_max < 1 ||
        c->n_classes < 1)
        return MD_EINVAL;
    md_ai m;
    m.c = *c;
    size_t off = 0;
    plan_ai(m, nullptr, off);
    *bytes = off + 256;
    return MD_OK;
}

int md_ai_init(const md_ai_config *c, void *workspace, size_t bytes, void *stream, md_ai **out)
{
    if (!c || !out) return MD_EINVAL;
    size_t need = 0;
    if (md_ai_workspace_size(c, &need) != MD_OK) return MD_EINVAL;
    if (!workspace || bytes < need) return MD_ENOMEM;
    md_ai *m = new (std::nothrow) md_ai();
    if (!m) return MD_ENOMEM;
    m->c = *c;
    m->st = (cudaStream_t)stream;
    size_t off = 0;
    char *base = (char *)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    plan_ai(*m, base, off);
    cudaError_t e = cudaMemsetAsync(m->Am, 0, sizeof(float) * m->nparam, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->Av, 0, sizeof(float) * m->nparam, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) {
        delete m;
        return MD_ECUDA;
    }
    *out = m;
    return MD_OK;
}

void md_ai_destroy(md_ai *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->st);
    delete m;
}

const char *md_ai_last_error(const md_ai *m) { return (m && !m->err.empty()) ? m->err.c_str() : "no error"; }

int md_ai_set_params(md_ai *m, const float *p, int64_t n)
{
    if (!m || !p || n != m->nparam) return MD_EINVAL;
    AK(cudaMemcpyAsync(m->P, p, sizeof(float) * n, cudaMemcpyHostToDevice, m->st), "upload params");
    AK(cudaMemsetAsync(m->Am, 0, sizeof(float) * n, m->st), "reset adam");
    AK(cudaMemsetAsync(m->Av, 0, sizeof(float) * n, m->st), "reset adam");
    AK(cudaStreamSynchronize(m->st), "sync");
    m->adam_t = 0;
    m->adam_t_heads = 0;
    m->has_params = true;
    return MD_OK;
}

int md_ai_get_params(md_ai *m, float *p, int64_t n)
{
    if (!m || !p || n != m->nparam) return MD_EINVAL;
    AK(cudaMemcpyAsync(p, m->P, sizeof(float) * n, cudaMemcpyDeviceToHost, m->st), "download params");
    AK(cudaStreamSynchronize(m->st), "sync");
    return MD_OK;
}

int md_ai_set_norm(md_ai *m, const float *mean, const float *stdv)
{
    if (!m || !mean || !stdv) return MD_EINVAL;
    AK(cudaMemcpyAsync(m->mean, mean, sizeof(float) * m->c.F, cudaMemcpyHostToDevice, m->st), "norm");
    AK(cudaMemcpyAsync(m->stdv, stdv, sizeof(float) * m->c.F, cudaMemcpyHostToDevice, m->st), "norm");
    AK(cudaStreamSynchronize(m->st), "sync");
    m->has_norm = true;
    return MD_OK;
}

}  // extern "C"

namespace {

// Table 2 steps 1-4 on the device: denoised, normalised windows through the
// autoencoder and the heads, then the class probabilities (m->probs), the log
// hold (m->lh) and the reconstruction error (m->rec).
int predict_device(md_ai *m, const float *raw, int32_t B, int32_t where, int strain_col = -1)
{
    int rc = stage_windows(m, raw, B, where, true);
    if (rc) return rc;
    if (strain_col >= 0) {
        // the raw windows (staged in m->Y, or the caller's device array) before
        // the autoencoder reuses m->Y for its reconstruction
        const float *src = where == MD_AI_HOST ? m->Y : raw;
        k_window_max<<<nblk(B, 128), 128, 0, m->st>>>(src, B, m->c.T, m->c.F, strain_col, m->smax);
        AK(cudaGetLastError(), "window max");
    }
    rc = ae_forward(m, B, false);
    if (rc) return rc;
    rc = heads_forward(m, B);
    if (rc) return rc;
    k_heads_loss<<<nblk(B, 128), 128, 0, m->st>>>(m->logits, m->c.n_classes, m->lh, nullptr, nullptr, B, 0.f, nullptr,
                                             nullptr, nullptr, m->probs);
    AK(cudaGetLastError(), "softmax");
    return MD_OK;
}

int check_trust(md_ai *m, const md_ai_trust *tr, const int32_t *k_values)
{
    if (!tr || !k_values || m->c.n_classes > 8) { m->err = "md_ai_decide: bad trust bound or class ratios"; return MD_EINVAL; }
    if (!(tr->hold_min <= tr->hold_max) || tr->fallback_k < 1 || tr->strain_col >= m->c.F) {
        m->err = "md_ai_decide: bad trust bound";
        return MD_EINVAL;
    }
    for (int c = 0; c < m->c.n_classes; ++c)
        if (k_values[c] < 1) { m->err = "md_ai_decide: class ratios must be >= 1"; return MD_EINVAL; }
    return MD_OK;
}

// Steps 5-6 on windows already through predict_device (with the strain
// column's maxima in m->smax); decisions copied to the host arrays.
int decide_device(md_ai *m, int32_t B, const md_ai_trust *tr, const int32_t *k_values, int32_t *k_out,
                  int32_t *hold_out, int32_t *why_out)
{
    decide_args a;
    a.probs = m->probs; a.lh = m->lh; a.rec = m->rec; a.smax = m->smax;
    a.B = B; a.C = m->c.n_classes; a.T = m->c.T; a.F = m->c.F;
    a.p_min = tr->p_min; a.rec_max = tr->rec_max; a.strain_max = tr->strain_max;
    a.hold_min = tr->hold_min; a.hold_max = tr->hold_max;
    a.strain_col = tr->strain_col; a.fallback_k = tr->fallback_k;
    for (int c = 0; c < 8; ++c) a.kv[c] = c < a.C ? k_values[c] : 1;
    a.out = m->dec;
    k_decide<<<nblk(B, 128), 128, 0, m->st>>>(a);
    AK(cudaGetLastError(), "decide");
    std::vector<int32_t> h((size_t)3 * B);
    AK(cudaMemcpyAsync(h.data(), m->dec, sizeof(int32_t) * 3 * B, cudaMemcpyDeviceToHost, m->st), "decisions");
    AK(cudaStreamSynchronize(m->st), "sync");
    for (int b = 0; b < B; ++b) {
        k_out[b] = h[(size_t)b];
        if (hold_out) hold_out[b] = h[(size_t)B + b];
        if (why_out) why_out[b] = h[(size_t)2 * B + b];
    }
    return MD_OK;
}

}  // namespace

extern "C" {

int md_ai_decide(md_ai *m, const float *raw, int32_t B, int32_t where, const md_ai_trust *trust,
                 const int32_t *k_values, int32_t *k_out, int32_t *hold_out, int32_t *why_out)
{
    if (!m || !raw || !k_out || B < 1 || B > m->c.batch_max) return MD_EINVAL;
    if (!m->has_params) return MD_ENOTRAINED;
    int rc = check_trust(m, trust, k_values);
    if (rc) return rc;
    rc = predict_device(m, raw, B, where, trust->strain_col);
    if (rc) return rc;
    return decide_device(m, B, trust, k_values, k_out, hold_out, why_out);
}

int md_ai_decide_system(md_ai *m, md_system *s, const md_ai_trust *trust, const int32_t *k_values, int32_t *k_out,
                        int32_t *hold_out, int32_t *why_out)
{
    if (!m || !s || !k_out) return MD_EINVAL;
    if (!m->has_params) return MD_ENOTRAINED;
    if (s->n_plt == 0 || !s->ring) { m->err = "md_ai_decide_system: the system has no platelets"; return MD_EINVAL; }
    const int P = s->cfg.n_platelets;
    if (P > m->c.batch_max || s->ring_T != m->c.T || m->c.F != 12) {
        m->err = "md_ai_decide_system: controller batch, window length or measurement count does not match the system";
        return MD_EINVAL;
    }
    int rc = check_trust(m, trust, k_values);
    if (rc) return rc;
    // the ring count decides whether a full window exists (one word from the
    // system's pinned mirror after its stream drains)
    AK(cudaMemcpyAsync(s->h_ds, s->ds, sizeof(md_dstate), cudaMemcpyDeviceToHost, s->stream), "ring count");
    AK(cudaStreamSynchronize(s->stream), "sync system");
    if (s->h_ds->ring_count < s->ring_T) {
        m->err = "md_ai_decide_system: fewer recorded steps than one window";
        return MD_EINVAL;
    }
    const int T = m->c.T, F = m->c.F;
    k_gather_ring<<<nblk((int64_t)P * T * F), 256, 0, m->st>>>(s->ring, s->ds, P, T, F, m->Y);
    AK(cudaGetLastError(), "gather ring");
    rc = predict_device(m, m->Y, P, MD_AI_DEVICE, trust->strain_col);
    if (rc) return rc;
    return decide_device(m, P, trust, k_values, k_out, hold_out, why_out);
}

int md_ai_predict(md_ai *m, const float *raw, int32_t B, int32_t where, float *out)
{
    if (!m || !raw || !out || B < 1 || B > m->c.batch_max) return MD_EINVAL;
    if (!m->has_params) return MD_ENOTRAINED;
    int rc = predict_device(m, raw, B, where);
    if (rc) return rc;
    const int C = m->c.n_classes;
    std::vector<float> probs((size_t)B * C), lh((size_t)B), rec((size_t)B);
    AK(cudaMemcpyAsync(probs.data(), m->probs, sizeof(float) * B * C, cudaMemcpyDeviceToHost, m->st), "probs");
    AK(cudaMemcpyAsync(lh.data(), m->lh, sizeof(float) * B, cudaMemcpyDeviceToHost, m->st), "hold");
    AK(cudaMemcpyAsync(rec.data(), m->rec, sizeof(float) * B, cudaMemcpyDeviceToHost, m->st), "rec");
    AK(cudaStreamSynchronize(m->st), "sync");
    for (int b = 0; b < B; ++b) {
        for (int c = 0; c < C; ++c) out[(int64_t)b * (C + 2) + c] = probs[(size_t)b * C + c];
        out[(int64_t)b * (C + 2) + C] = lh[(size_t)b];
        out[(int64_t)b * (C + 2) + C + 1] = rec[(size_t)b];
    }
    return MD_OK;
}

int md_ai_prepare(md_ai *m, const float *raw, int32_t B, int32_t where, float *out)
{
    if (!m || !raw || !out || B < 1 || B > m->c.batch_max) return MD_EINVAL;
    int rc = stage_windows(m, raw, B, where, true);
    if (rc) return rc;
    const int T = m->c.T, F = m->c.F;
    std::vector<float> tm((size_t)T * B * F);
    AK(cudaMemcpyAsync(tm.data(), m->X, sizeof(float) * tm.size(), cudaMemcpyDeviceToHost, m->st), "windows");
    AK(cudaStreamSynchronize(m->st), "sync");
    for (int t = 0; t < T; ++t)          // time-major [T][B][F] -> [B][T][F]
        for (int b = 0; b < B; ++b)
            for (int f = 0; f < F; ++f)
                out[((int64_t)b * T + t) * F + f] = tm[((size_t)t * B + b) * F + f];
    return MD_OK;
}

int md_ai_encode(md_ai *m, const float *x, int32_t B, float *latent_out, float *recon_out)
{
    if (!m || !x || B < 1 || B > m->c.batch_max) return MD_EINVAL;
    if (!m->has_params) return MD_ENOTRAINED;
    int rc = stage_windows(m, x, B, MD_AI_HOST, false);
    if (rc) return rc;
    rc = ae_forward(m, B, false);
    if (rc) return rc;
    if (latent_out)
        AK(cudaMemcpyAsync(latent_out, m->Z, sizeof(float) * B * m->c.latent, cudaMemcpyDeviceToHost, m->st), "Z");
    if (recon_out)   // time-major [T][B][F]
        AK(cudaMemcpyAsync(recon_out, m->Y, sizeof(float) * B * m->c.T * m->c.F, cudaMemcpyDeviceToHost, m->st), "Y");
    AK(cudaStreamSynchronize(m->st), "sync");
    return MD_OK;
}

int md_ai_grads(md_ai *m, const float *x, const int32_t *k_class, const float *log_hold, int32_t B, int32_t what,
                float *grads, float *loss)
{
    if (!m || !x || B < 1 || B > m->c.batch_max || (what != MD_AI_TRAIN_AE && what != MD_AI_TRAIN_HEADS))
        return MD_EINVAL;
    if (what == MD_AI_TRAIN_HEADS && (!k_class || !log_hold)) return MD_EINVAL;
    if (!m->has_params) return MD_ENOTRAINED;
    int rc = stage_windows(m, x, B, MD_AI_HOST, false);
    if (rc) return rc;
    AK(cudaMemsetAsync(m->G, 0, sizeof(float) * m->nparam, m->st), "zero grads");
    rc = ae_forward(m, B, what == MD_AI_TRAIN_AE);
    if (rc) return rc;
    float l = 0.f;
    if (what == MD_AI_TRAIN_AE) {
        rc = ae_backward(m, B);
        if (rc) return rc;
        AK(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st), "loss");
    } else {
        rc = heads_forward(m, B);
        if (rc) return rc;
        AK(cudaMemcpyAsync(m->cls, k_class, sizeof(int32_t) * B, cudaMemcpyHostToDevice, m->st), "labels");
        AK(cudaMemcpyAsync(m->lht, log_hold, sizeof(float) * B, cudaMemcpyHostToDevice, m->st), "labels");
        AK(cudaMemsetAsync(m->loss + 1, 0, sizeof(float), m->st), "zero loss");
        k_heads_loss<<<nblk(B, 128), 128, 0, m->st>>>(m->logits, m->c.n_classes, m->lh, m->cls, m->lht, B, 1.f, m->dlog,
                                                 m->dlh, m->loss + 1, m->probs);
        AK(cudaGetLastError(), "heads loss");
        rc = heads_backward(m, B);
        if (rc) return rc;
        AK(cudaMemcpyAsync(&l, m->loss + 1, sizeof(float), cudaMemcpyDeviceToHost, m->st), "loss");
    }
    if (grads) AK(cudaMemcpyAsync(grads, m->G, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->st), "grads");
    AK(cudaStreamSynchronize(m->st), "sync");
    if (loss) *loss = l;
    return MD_OK;
}

int md_ai_train_step(md_ai *m, const float *x, const int32_t *k_class, const float *log_hold, int32_t B, int32_t what,
                     float lr, float *loss)
{
    int rc = md_ai_grads(m, x, k_class, log_hold, B, what, nullptr, loss);
    if (rc) return rc;
    // Adam on the trained part only (the other part's gradient is zero and
    // its moments stay zero, so it does not move)
    int64_t &t = what == MD_AI_TRAIN_AE ? m->adam_t : m->adam_t_heads;
    t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    const int64_t lo = what == MD_AI_TRAIN_AE ? 0 : m->kh[0][0];
    const int64_t hi = what == MD_AI_TRAIN_AE ? m->kh[0][0] : m->nparam;
    k_adam<<<nblk(hi - lo), 256, 0, m->st>>>(m->P + lo, m->G + lo, m->Am + lo, m->Av + lo, hi - lo, lr, b1, b2, 1e-8f,
                                             c1, c2);
    AK(cudaGetLastError(), "adam");
    AK(cudaStreamSynchronize(m->st), "sync");
    return MD_OK;
}

}  // extern "C"
