// The paper's own controller variant (Sec. 3.3): the last 50 steps of six
// per-platelet measurements, denoised (Table 2 step 2), through a two-layer
// LSTM autoencoder of 16 and 4 units whose latent is the 4-unit layer's final
// hidden and cell state (8 features), a mirrored decoder (LSTM 8 -> 4,
// LSTM 4 -> 16, linear 16 -> 6 at every step, fed the repeated latent), and a
// four-layer FCN (32, 16, 8, 1) whose output is log k, the ratio of the fluid
// step to the platelet step (Table 2 step 4).  Backpropagation through time
// and Adam train it on the device.
//
// The layers are a few units wide, so every kernel is plain FP32 SIMT: one
// block per window, one thread per gate row (4H threads), the recurrence
// stepped inside the block with the state in shared memory.
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "msm_internal.cuh"

namespace {

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + __expf(-x)); }

struct lstm_w {
    const float *Wih, *Whh, *bih, *bhh;
};
struct lstm_g {
    float *Wih, *Whh, *bih, *bhh;
};

// One LSTM layer over T steps for window b = blockIdx.x; gates (i, f, g, o)
// stacked along the rows of W_ih [4H][in] and W_hh [4H][H].  xs: input
// [T][B][in] (tstride = B * in), or one input per window repeated over time
// (tstride = 0, xs [B][in]).  Writes h [T][B][H], c [T][B][H] and the gate
// activations [T][B][4H].
template <int H>
__global__ void k_lstm_fwd(const float *xs, int64_t tstride, int in, int T, int B, lstm_w w, float *Hs, float *Cs,
                           float *Gs)
{
    const int b = blockIdx.x, j = threadIdx.x;
    __shared__ float sx[32], sh[H], sc[H], sa[4 * H];
    if (j < H) { sh[j] = 0.f; sc[j] = 0.f; }
    for (int t = 0; t < T; ++t) {
        if (j < in) sx[j] = xs[t * tstride + (int64_t)b * in + j];
        __syncthreads();
        float a = w.bih[j] + w.bhh[j];
        for (int k = 0; k < in; ++k) a += w.Wih[j * in + k] * sx[k];
#pragma unroll
        for (int k = 0; k < H; ++k) a += w.Whh[j * H + k] * sh[k];
        const float act = (j >= 2 * H && j < 3 * H) ? tanhf(a) : sigm(a);
        sa[j] = act;
        Gs[((int64_t)t * B + b) * 4 * H + j] = act;
        __syncthreads();
        if (j < H) {
            const float c = sa[H + j] * sc[j] + sa[j] * sa[2 * H + j];
            const float h = sa[3 * H + j] * tanhf(c);
            sc[j] = c;
            sh[j] = h;
            Hs[((int64_t)t * B + b) * H + j] = h;
            Cs[((int64_t)t * B + b) * H + j] = c;
        }
        __syncthreads();
    }
}

// Backpropagation through time of one layer for window b = blockIdx.x.
// dHs: dL/dh_t from above [T][B][H] (may be null); dh_last, dc_last: extra
// dL/dh_T, dL/dc_T [B][H] (may be null).  Weight gradients are added to g;
// the input gradient goes to dXs [T][B][in] (tstride > 0) or, for an input
// repeated over time, summed over t into dXs [B][in]; dXs may be null.
template <int H>
__global__ void k_lstm_bwd(const float *xs, int64_t tstride, int in, int T, int B, lstm_w w, const float *Hs,
                           const float *Cs, const float *Gs, const float *dHs, const float *dh_last,
                           const float *dc_last, lstm_g g, float *dXs)
{
    const int b = blockIdx.x, j = threadIdx.x;
    __shared__ float sx[32], shp[H], sdh[H], sdc[H], sda[4 * H];
    if (j < H) {
        sdh[j] = dh_last ? dh_last[(int64_t)b * H + j] : 0.f;
        sdc[j] = dc_last ? dc_last[(int64_t)b * H + j] : 0.f;
    }
    float gih[32], ghh[H], gb = 0.f, dxsum = 0.f;
    for (int k = 0; k < 32; ++k) gih[k] = 0.f;
#pragma unroll
    for (int k = 0; k < H; ++k) ghh[k] = 0.f;
    __syncthreads();
    for (int t = T - 1; t >= 0; --t) {
        if (j < in) sx[j] = xs[t * tstride + (int64_t)b * in + j];
        if (j < H) shp[j] = t > 0 ? Hs[((int64_t)(t - 1) * B + b) * H + j] : 0.f;
        float dc_new = 0.f;
        if (j < H) {
            const float *ga = Gs + ((int64_t)t * B + b) * 4 * H;
            const float i = ga[j], f = ga[H + j], gg = ga[2 * H + j], o = ga[3 * H + j];
            const float c = Cs[((int64_t)t * B + b) * H + j];
            const float cp = t > 0 ? Cs[((int64_t)(t - 1) * B + b) * H + j] : 0.f;
            const float tc = tanhf(c);
            const float dh = sdh[j] + (dHs ? dHs[((int64_t)t * B + b) * H + j] : 0.f);
            const float dct = sdc[j] + dh * o * (1.f - tc * tc);
            sda[j] = dct * gg * i * (1.f - i);
            sda[H + j] = dct * cp * f * (1.f - f);
            sda[2 * H + j] = dct * i * (1.f - gg * gg);
            sda[3 * H + j] = dh * tc * o * (1.f - o);
            dc_new = dct * f;
        }
        __syncthreads();
        const float da = sda[j];
        gb += da;
        for (int k = 0; k < in; ++k) gih[k] += da * sx[k];
#pragma unroll
        for (int k = 0; k < H; ++k) ghh[k] += da * shp[k];
        float dx = 0.f, dhp = 0.f;
        if (j < in) {
            for (int r = 0; r < 4 * H; ++r) dx += sda[r] * w.Wih[r * in + j];
            if (dXs && tstride) dXs[((int64_t)t * B + b) * in + j] = dx;
            dxsum += dx;
        }
        if (j < H)
            for (int r = 0; r < 4 * H; ++r) dhp += sda[r] * w.Whh[r * H + j];
        __syncthreads();
        if (j < H) { sdh[j] = dhp; sdc[j] = dc_new; }
        __syncthreads();
    }
    if (dXs && !tstride && j < in) dXs[(int64_t)b * in + j] = dxsum;
    for (int k = 0; k < in; ++k) atomicAdd(&g.Wih[j * in + k], gih[k]);
#pragma unroll
    for (int k = 0; k < H; ++k) atomicAdd(&g.Whh[j * H + k], ghh[k]);
    atomicAdd(&g.bih[j], gb);
    atomicAdd(&g.bhh[j], gb);
}

// y[r][o] = W[o] . x[r] + b[o] for rows r < R (optionally ReLU)
__global__ void k_dense(const float *x, int R, int nin, const float *W, const float *bias, int nout, int relu,
                        float *y)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)R * nout) return;
    const int64_t r = q / nout;
    const int o = (int)(q % nout);
    float a = bias[o];
    for (int k = 0; k < nin; ++k) a += W[o * nin + k] * x[r * nin + k];
    y[q] = relu ? fmaxf(a, 0.f) : a;
}

// dense layer backward: gW[o][k] += sum_r d[r][o] x[r][k], gb[o] += sum_r d[r][o]
// (one thread per weight), dx[r][k] = sum_o d[r][o] W[o][k] (times the ReLU
// mask of x when relu_x, null dx: skipped)
__global__ void k_dense_wgrad(const float *x, const float *d, int R, int nin, int nout, float *gW, float *gb)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nout * (nin + 1)) return;
    const int o = q / (nin + 1), k = q % (nin + 1);
    float s = 0.f;
    for (int r = 0; r < R; ++r) s += d[(int64_t)r * nout + o] * (k < nin ? x[(int64_t)r * nin + k] : 1.f);
    if (k < nin) gW[o * nin + k] += s;
    else gb[o] += s;
}

__global__ void k_dense_xgrad(const float *d, int R, int nin, int nout, const float *W, const float *x, int relu_x,
                              float *dx)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)R * nin) return;
    const int64_t r = q / nin;
    const int k = (int)(q % nin);
    float s = 0.f;
    for (int o = 0; o < nout; ++o) s += d[r * nout + o] * W[o * nin + k];
    if (relu_x && !(x[q] > 0.f)) s = 0.f;
    dx[q] = s;
}

// reconstruction error: rec[b] = mean over (t, f) of (y - x)^2; with dy:
// dy = 2 (y - x) / (T B F) and loss += mean over all
__global__ void k_lstm_mse(const float *Y, const float *X, int B, int T, int F, float *dY, float *loss, float *rec)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)T * B * F;
    if (q >= n) return;
    const int b = (int)((q / F) % B);
    const float e = Y[q] - X[q];
    if (dY) dY[q] = 2.f * e / (float)n;
    atomicAdd(&rec[b], e * e / (float)(T * F));
    if (loss) atomicAdd(loss, e * e / (float)n);
}

// latent [B][2 H2] = [h_T, c_T] of the 4-unit layer
__global__ void k_latent(const float *Hs, const float *Cs, int T, int B, int H, float *Z)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B * 2 * H) return;
    const int b = q / (2 * H), k = q % (2 * H);
    const int64_t o = ((int64_t)(T - 1) * B + b) * H + (k % H);
    Z[q] = k < H ? Hs[o] : Cs[o];
}

// FCN regression loss on log k: loss = mean (out - target)^2, d = 2 e / B
__global__ void k_fcn_loss(const float *out, const float *target, int B, float *d, float *loss)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float e = out[b] - target[b];
    d[b] = 2.f * e / (float)B;
    atomicAdd(loss, e * e / (float)B);
}

unsigned nb(int64_t n, int t = 256) { return (unsigned)(n > 0 ? (n + t - 1) / t : 1); }

}  // namespace

struct md_lstm {
    md_lstm_config c;
    cudaStream_t st;
    std::string err;
    int64_t nparam = 0;
    int64_t off_l[4][4];             // enc1, enc2, dec1, dec2: W_ih, W_hh, b_ih, b_hh
    int64_t off_out[2], off_fcn[4][2];
    int hd[5];                        // FCN widths: latent, h0, h1, h2, 1
    float *P, *G, *Am, *Av, *mean, *stdv;
    float *Yraw, *X, *Y, *dY;         // staging [B][T][F]; windows, reconstruction, its gradient [T][B][F]
    float *Hs[4], *Cs[4], *Gs[4];     // per layer [T][B][H], [T][B][H], [T][B][4H]
    float *dA, *dB;                   // [T][B][16] input gradients between layers
    float *Z, *dZ, *dh2, *dc2;        // latent [B][8], its gradient, its split [B][4] x 2
    float *act[5], *dact[2];          // FCN activations [B][w], gradients
    float *rec, *loss, *target;
    int64_t adam_t[2] = {0, 0};
    bool has_params = false, has_norm = false;
};

namespace {

int H_of(const md_lstm &m, int l) { return (l == 0 || l == 3) ? m.c.H1 : m.c.H2; }
int in_of(const md_lstm &m, int l)
{
    return l == 0 ? m.c.F : (l == 1 ? m.c.H1 : (l == 2 ? 2 * m.c.H2 : m.c.H2));
}

void plan_lstm(md_lstm &m, char *base, size_t &off)
{
    auto take = [&](int64_t n) -> float * {
        off = (off + 255) & ~(size_t)255;
        float *p = base ? reinterpret_cast<float *>(base + off) : nullptr;
        off += sizeof(float) * (size_t)(n > 0 ? n : 1);
        return p;
    };
    const md_lstm_config &c = m.c;
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
        const int H = H_of(m, l), in = in_of(m, l);
        m.off_l[l][0] = o; o += 4 * H * in;
        m.off_l[l][1] = o; o += 4 * H * H;
        m.off_l[l][2] = o; o += 4 * H;
        m.off_l[l][3] = o; o += 4 * H;
    }
    m.off_out[0] = o; o += c.F * c.H1;
    m.off_out[1] = o; o += c.F;
    m.hd[0] = 2 * c.H2; m.hd[1] = c.fcn[0]; m.hd[2] = c.fcn[1]; m.hd[3] = c.fcn[2]; m.hd[4] = 1;
    for (int l = 0; l < 4; ++l) {
        m.off_fcn[l][0] = o; o += m.hd[l + 1] * m.hd[l];
        m.off_fcn[l][1] = o; o += m.hd[l + 1];
    }
    m.nparam = o;
    const int64_t T = c.T, B = c.batch_max, F = c.F;
    m.P = take(o); m.G = take(o); m.Am = take(o); m.Av = take(o);
    m.mean = take(F); m.stdv = take(F);
    m.Yraw = take(B * T * F); m.X = take(T * B * F); m.Y = take(T * B * F); m.dY = take(T * B * F);
    for (int l = 0; l < 4; ++l) {
        const int H = H_of(m, l);
        m.Hs[l] = take(T * B * H); m.Cs[l] = take(T * B * H); m.Gs[l] = take(T * B * 4 * H);
    }
    m.dA = take(T * B * 16); m.dB = take(T * B * 16);
    m.Z = take(B * 2 * c.H2); m.dZ = take(B * 2 * c.H2); m.dh2 = take(B * c.H2); m.dc2 = take(B * c.H2);
    int wmax = 1;
    for (int l = 0; l < 5; ++l) wmax = wmax > m.hd[l] ? wmax : m.hd[l];
    for (int l = 0; l < 5; ++l) m.act[l] = take(B * wmax);
    m.dact[0] = take(B * wmax); m.dact[1] = take(B * wmax);
    m.rec = take(B); m.loss = take(4); m.target = take(B);
}

int lfail(md_lstm *m, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return MD_OK;
    m->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    return MD_ECUDA;
}
#define LK(expr, where)                          \
    do {                                         \
        int _rc = lfail(m, (expr), where);       \
        if (_rc) return _rc;                     \
    } while (0)

lstm_w weights(md_lstm *m, int l)
{
    return {m->P + m->off_l[l][0], m->P + m->off_l[l][1], m->P + m->off_l[l][2], m->P + m->off_l[l][3]};
}
lstm_g wgrads(md_lstm *m, int l)
{
    return {m->G + m->off_l[l][0], m->G + m->off_l[l][1], m->G + m->off_l[l][2], m->G + m->off_l[l][3]};
}

cudaError_t layer_fwd(md_lstm *m, int l, const float *xs, bool repeated, int B)
{
    const int H = H_of(*m, l), in = in_of(*m, l), T = m->c.T;
    const int64_t ts = repeated ? 0 : (int64_t)B * in;
    if (H == 16) k_lstm_fwd<16><<<B, 64, 0, m->st>>>(xs, ts, in, T, B, weights(m, l), m->Hs[l], m->Cs[l], m->Gs[l]);
    else k_lstm_fwd<4><<<B, 16, 0, m->st>>>(xs, ts, in, T, B, weights(m, l), m->Hs[l], m->Cs[l], m->Gs[l]);
    return cudaGetLastError();
}

cudaError_t layer_bwd(md_lstm *m, int l, const float *xs, bool repeated, int B, const float *dHs, const float *dhl,
                      const float *dcl, float *dX)
{
    const int H = H_of(*m, l), in = in_of(*m, l), T = m->c.T;
    const int64_t ts = repeated ? 0 : (int64_t)B * in;
    if (H == 16)
        k_lstm_bwd<16><<<B, 64, 0, m->st>>>(xs, ts, in, T, B, weights(m, l), m->Hs[l], m->Cs[l], m->Gs[l], dHs, dhl,
                                             dcl, wgrads(m, l), dX);
    else
        k_lstm_bwd<4><<<B, 16, 0, m->st>>>(xs, ts, in, T, B, weights(m, l), m->Hs[l], m->Cs[l], m->Gs[l], dHs, dhl,
                                            dcl, wgrads(m, l), dX);
    return cudaGetLastError();
}

// autoencoder forward on m->X: latent m->Z, reconstruction m->Y, per-window
// error m->rec (and m->dY, m->loss[0] when train)
int ae_fwd(md_lstm *m, int B, bool train)
{
    const int T = m->c.T, F = m->c.F;
    LK(layer_fwd(m, 0, m->X, false, B), "enc1");
    LK(layer_fwd(m, 1, m->Hs[0], false, B), "enc2");
    k_latent<<<nb((int64_t)B * 2 * m->c.H2), 256, 0, m->st>>>(m->Hs[1], m->Cs[1], T, B, m->c.H2, m->Z);
    LK(cudaGetLastError(), "latent");
    LK(layer_fwd(m, 2, m->Z, true, B), "dec1");
    LK(layer_fwd(m, 3, m->Hs[2], false, B), "dec2");
    k_dense<<<nb((int64_t)T * B * F), 256, 0, m->st>>>(m->Hs[3], T * B, m->c.H1, m->P + m->off_out[0],
                                                      m->P + m->off_out[1], F, 0, m->Y);
    LK(cudaGetLastError(), "out");
    LK(cudaMemsetAsync(m->rec, 0, sizeof(float) * B, m->st), "zero rec");
    LK(cudaMemsetAsync(m->loss, 0, sizeof(float) * 4, m->st), "zero loss");
    k_lstm_mse<<<nb((int64_t)T * B * F), 256, 0, m->st>>>(m->Y, m->X, B, T, F, train ? m->dY : nullptr,
                                                          train ? m->loss : nullptr, m->rec);
    LK(cudaGetLastError(), "mse");
    return MD_OK;
}

int ae_bwd(md_lstm *m, int B)
{
    const int T = m->c.T, F = m->c.F, H1 = m->c.H1, H2 = m->c.H2;
    const int TB = T * B;
    k_dense_wgrad<<<nb(F * (H1 + 1), 128), 128, 0, m->st>>>(m->Hs[3], m->dY, TB, H1, F, m->G + m->off_out[0],
                                                      m->G + m->off_out[1]);
    k_dense_xgrad<<<nb((int64_t)TB * H1), 256, 0, m->st>>>(m->dY, TB, H1, F, m->P + m->off_out[0], nullptr, 0,
                                                         m->dA);
    LK(cudaGetLastError(), "out bwd");
    LK(layer_bwd(m, 3, m->Hs[2], false, B, m->dA, nullptr, nullptr, m->dB), "dec2 bwd");
    LK(layer_bwd(m, 2, m->Z, true, B, m->dB, nullptr, nullptr, m->dZ), "dec1 bwd");
    // dZ = [dh_T, dc_T] of the 4-unit encoder layer
    LK(cudaMemcpy2DAsync(m->dh2, sizeof(float) * H2, m->dZ, sizeof(float) * 2 * H2, sizeof(float) * H2, B,
                         cudaMemcpyDeviceToDevice, m->st), "split dZ");
    LK(cudaMemcpy2DAsync(m->dc2, sizeof(float) * H2, m->dZ + H2, sizeof(float) * 2 * H2, sizeof(float) * H2, B,
                         cudaMemcpyDeviceToDevice, m->st), "split dZ");
    LK(layer_bwd(m, 1, m->Hs[0], false, B, nullptr, m->dh2, m->dc2, m->dA), "enc2 bwd");
    LK(layer_bwd(m, 0, m->X, false, B, m->dA, nullptr, nullptr, nullptr), "enc1 bwd");
    return MD_OK;
}

int fcn_fwd(md_lstm *m, int B)
{
    const float *in = m->Z;
    for (int l = 0; l < 4; ++l) {
        k_dense<<<nb((int64_t)B * m->hd[l + 1]), 256, 0, m->st>>>(in, B, m->hd[l], m->P + m->off_fcn[l][0],
                                                                 m->P + m->off_fcn[l][1], m->hd[l + 1], l < 3 ? 1 : 0,
                                                                 m->act[l + 1]);
        LK(cudaGetLastError(), "fcn");
        in = m->act[l + 1];
    }
    return MD_OK;
}

int fcn_bwd(md_lstm *m, int B)
{
    float *d = m->dact[0];
    for (int l = 3; l >= 0; --l) {
        const float *in = l == 0 ? m->Z : m->act[l];
        k_dense_wgrad<<<nb(m->hd[l + 1] * (m->hd[l] + 1), 128), 128, 0, m->st>>>(in, d, B, m->hd[l], m->hd[l + 1],
                                                                           m->G + m->off_fcn[l][0],
                                                                           m->G + m->off_fcn[l][1]);
        LK(cudaGetLastError(), "fcn wgrad");
        if (l > 0) {
            float *dn = d == m->dact[0] ? m->dact[1] : m->dact[0];
            k_dense_xgrad<<<nb((int64_t)B * m->hd[l]), 256, 0, m->st>>>(d, B, m->hd[l], m->hd[l + 1],
                                                                       m->P + m->off_fcn[l][0], m->act[l], 1, dn);
            LK(cudaGetLastError(), "fcn xgrad");
            d = dn;
        }
    }
    return MD_OK;
}

int stage(md_lstm *m, const float *x, int B, int where, bool raw)
{
    const int T = m->c.T, F = m->c.F;
    const int64_t cnt = (int64_t)B * T * F;
    const float *src = x;
    if (where == MD_AI_HOST) {
        LK(cudaMemcpyAsync(m->Yraw, x, sizeof(float) * cnt, cudaMemcpyHostToDevice, m->st), "upload windows");
        src = m->Yraw;
    }
    if (raw) {
        LK(ai_launch_denoise(src, B, T, F, m->has_norm ? m->mean : nullptr, m->has_norm ? m->stdv : nullptr, m->X,
                             m->st), "denoise");
    } else {   // already denoised and normalised, [B][T][F] -> time-major
        std::vector<float> h((size_t)cnt), tm((size_t)cnt);
        if (where != MD_AI_HOST) { m->err = "normalised windows come from the host"; return MD_EINVAL; }
        for (int b = 0; b < B; ++b)
            for (int t = 0; t < T; ++t)
                for (int f = 0; f < F; ++f) tm[((size_t)t * B + b) * F + f] = x[((size_t)b * T + t) * F + f];
        LK(cudaMemcpyAsync(m->X, tm.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice, m->st), "upload x");
        LK(cudaStreamSynchronize(m->st), "sync");
    }
    return MD_OK;
}

}  // namespace

extern "C" {

int md_lstm_config_defaults(md_lstm_config *c)
{
    if (!c) return MD_EINVAL;
    c->T = 50; c->F = 6; c->H1 = 16; c->H2 = 4;
    c->fcn[0] = 32; c->fcn[1] = 16; c->fcn[2] = 8;
    c->batch_max = 256;
    return MD_OK;
}

static bool lstm_cfg_ok(const md_lstm_config *c)
{
    return c && c->H1 == 16 && c->H2 == 4 && c->F >= 1 && c->F <= 16 && c->T >= 2 && c->T <= 256 && !(c->T & 1) &&
           c->batch_max >= 1 && c->fcn[0] >= 1 && c->fcn[1] >= 1 && c->fcn[2] >= 1;
}

int md_lstm_param_count(const md_lstm_config *c, int64_t *n)
{
    if (!lstm_cfg_ok(c) || !n) return MD_EINVAL;
    md_lstm m;
    m.c = *c;
    size_t off = 0;
    plan_lstm(m, nullptr, off);
    *n = m.nparam;
    return MD_OK;
}

int md_lstm_workspace_size(const md_lstm_config *c, size_t *bytes)
{
    if (!lstm_cfg_ok(c) || !bytes) return MD_EINVAL;
    md_lstm m;
    m.c = *c;
    size_t off = 0;
    plan_lstm(m, nullptr, off);
    *bytes = off + 256;
    return MD_OK;
}

int md_lstm_init(const md_lstm_config *c, void *workspace, size_t bytes, void *stream, md_lstm **out)
{
    if (!lstm_cfg_ok(c) || !out) return MD_EINVAL;
    size_t need = 0;
    md_lstm_workspace_size(c, &need);
    if (!workspace || bytes < need) return MD_ENOMEM;
    md_lstm *m = new (std::nothrow) md_lstm();
    if (!m) return MD_ENOMEM;
    m->c = *c;
    m->st = (cudaStream_t)stream;
    size_t off = 0;
    plan_lstm(*m, (char *)(((uintptr_t)workspace + 255) & ~(uintptr_t)255), off);
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

void md_lstm_destroy(md_lstm *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->st);
    delete m;
}

const char *md_lstm_last_error(const md_lstm *m) { return (m && !m->err.empty()) ? m->err.c_str() : "no error"; }

int md_lstm_set_params(md_lstm *m, const float *p, int64_t n)
{
    if (!m || !p || n != m->nparam) return MD_EINVAL;
    LK(cudaMemcpyAsync(m->P, p, sizeof(float) * n, cudaMemcpyHostToDevice, m->st), "params");
    LK(cudaMemsetAsync(m->Am, 0, sizeof(float) * n, m->st), "adam");
    LK(cudaMemsetAsync(m->Av, 0, sizeof(float) * n, m->st), "adam");
    LK(cudaStreamSynchronize(m->st), "sync");
    m->adam_t[0] = m->adam_t[1] = 0;
    m->has_params = true;
    return MD_OK;
}

int md_lstm_get_params(md_lstm *m, float *p, int64_t n)
{
    if (!m || !p || n != m->nparam) return MD_EINVAL;
    LK(cudaMemcpyAsync(p, m->P, sizeof(float) * n, cudaMemcpyDeviceToHost, m->st), "params");
    LK(cudaStreamSynchronize(m->st), "sync");
    return MD_OK;
}

int md_lstm_set_norm(md_lstm *m, const float *mean, const float *stdv)
{
    if (!m || !mean || !stdv) return MD_EINVAL;
    LK(cudaMemcpyAsync(m->mean, mean, sizeof(float) * m->c.F, cudaMemcpyHostToDevice, m->st), "norm");
    LK(cudaMemcpyAsync(m->stdv, stdv, sizeof(float) * m->c.F, cudaMemcpyHostToDevice, m->st), "norm");
    LK(cudaStreamSynchronize(m->st), "sync");
    m->has_norm = true;
    return MD_OK;
}

int md_lstm_predict(md_lstm *m, const float *raw, int32_t B, int32_t where, float *out)
{
    if (!m || !raw || !out || B < 1 || B > m->c.batch_max) return MD_EINVAL;
    if (!m->has_params) return MD_ENOTRAINED;
    int rc = stage(m, raw, B, where, true);
    if (rc) return rc;
    if ((rc = ae_fwd(m, B, false)) || (rc = fcn_fwd(m, B))) return rc;
    std::vector<float> lk((size_t)B), rec((size_t)B);
    LK(cudaMemcpyAsync(lk.data(), m->act[4], sizeof(float) * B, cudaMemcpyDeviceToHost, m->st), "log k");
    LK(cudaMemcpyAsync(rec.data(), m->rec, sizeof(float) * B, cudaMemcpyDeviceToHost, m->st), "rec");
    LK(cudaStreamSynchronize(m->st), "sync");
    for (int b = 0; b < B; ++b) {
        out[2 * b] = lk[(size_t)b];
        out[2 * b + 1] = rec[(size_t)b];
    }
    return MD_OK;
}

int md_lstm_prepare(md_lstm *m, const float *raw, int32_t B, int32_t where, float *out)
{
    if (!m || !raw || !out || B < 1 || B > m->c.batch_max) return MD_EINVAL;
    int rc = stage(m, raw, B, where, true);
    if (rc) return rc;
    const int T = m->c.T, F = m->c.F;
    std::vector<float> tm((size_t)T * B * F);
    LK(cudaMemcpyAsync(tm.data(), m->X, sizeof(float) * tm.size(), cudaMemcpyDeviceToHost, m->st), "windows");
    LK(cudaStreamSynchronize(m->st), "sync");
    for (int t = 0; t < T; ++t)          // time-major [T][B][F] -> [B][T][F]
        for (int b = 0; b < B; ++b)
            for (int f = 0; f < F; ++f) out[((int64_t)b * T + t) * F + f] = tm[((size_t)t * B + b) * F + f];
    return MD_OK;
}

int md_lstm_grads(md_lstm *m, const float *x, const float *log_k, int32_t B, int32_t what, float *grads,
                  float *loss)
{
    if (!m || !x || B < 1 || B > m->c.batch_max || (what != MD_AI_TRAIN_AE && what != MD_AI_TRAIN_HEADS))
        return MD_EINVAL;
    if (what == MD_AI_TRAIN_HEADS && !log_k) return MD_EINVAL;
    if (!m->has_params) return MD_ENOTRAINED;
    int rc = stage(m, x, B, MD_AI_HOST, false);
    if (rc) return rc;
    LK(cudaMemsetAsync(m->G, 0, sizeof(float) * m->nparam, m->st), "zero grads");
    if ((rc = ae_fwd(m, B, what == MD_AI_TRAIN_AE))) return rc;
    float l = 0.f;
    if (what == MD_AI_TRAIN_AE) {
        if ((rc = ae_bwd(m, B))) return rc;
        LK(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st), "loss");
    } else {
        if ((rc = fcn_fwd(m, B))) return rc;
        LK(cudaMemcpyAsync(m->target, log_k, sizeof(float) * B, cudaMemcpyHostToDevice, m->st), "targets");
        LK(cudaMemsetAsync(m->loss + 1, 0, sizeof(float), m->st), "zero loss");
        k_fcn_loss<<<nb(B, 128), 128, 0, m->st>>>(m->act[4], m->target, B, m->dact[0], m->loss + 1);
        LK(cudaGetLastError(), "fcn loss");
        if ((rc = fcn_bwd(m, B))) return rc;
        LK(cudaMemcpyAsync(&l, m->loss + 1, sizeof(float), cudaMemcpyDeviceToHost, m->st), "loss");
    }
    if (grads) LK(cudaMemcpyAsync(grads, m->G, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->st), "grads");
    LK(cudaStreamSynchronize(m->st), "sync");
    if (loss) *loss = l;
    return MD_OK;
}

int md_lstm_train_step(md_lstm *m, const float *x, const float *log_k, int32_t B, int32_t what, float lr,
                       float *loss)
{
    int rc = md_lstm_grads(m, x, log_k, B, what, nullptr, loss);
    if (rc) return rc;
    const int part = what == MD_AI_TRAIN_AE ? 0 : 1;
    const int64_t lo = part == 0 ? 0 : m->off_fcn[0][0];
    const int64_t hi = part == 0 ? m->off_fcn[0][0] : m->nparam;
    LK(ai_launch_adam(m->P + lo, m->G + lo, m->Am + lo, m->Av + lo, hi - lo, lr, ++m->adam_t[part], m->st), "adam");
    LK(cudaStreamSynchronize(m->st), "sync");
    return MD_OK;
}

}  // extern "C"
